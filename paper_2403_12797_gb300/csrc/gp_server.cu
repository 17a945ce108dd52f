// gp_server.cu -- a request server for resident fitted models (C ABI in
// include/gpfagp.h): continuous batching of predict and refit requests.
//
// The server owns a worker thread, `slots` CUDA streams and a device-memory
// budget for request scratch. Models stay resident on the device. Requests
// (predict: X* -> mean, var; refit: new training set for a resident model)
// queue in arrival order; the worker admits the queue head whenever a slot
// is free and the head's scratch estimate fits the budget, so requests that
// arrive while others are on the GPU start as soon as room frees up, and the
// admitted requests run side by side on their own streams. Each request's
// kernels are exactly those of gp_predict_ex / gp_fit_ex (same launch
// plans), so its result does not depend on what else is running.
//
// Host buffers are staged through pinned per-slot memory so that no copy
// blocks the worker; results are copied to the caller's buffers when the
// request's completion event has fired. A refit builds a new model on its
// slot and swaps it in at completion; requests already admitted against the
// old model finish on it, and it is freed when the last of them completes.
// The server owns the models registered with it and frees them at destroy.
#include "gp_internal.cuh"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

using namespace gpi;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// A resident model with a count of admitted requests that still use it.
struct Resident {
    gp_model* model = nullptr;
    int users = 0;
    bool retired = false;  // replaced by a refit: free when users reaches 0
};

// Pinned host staging of one slot, grown on demand.
struct Pinned {
    void* p = nullptr;
    size_t cap = 0;
    int reserve(size_t bytes) {
        if (bytes <= cap) return GP_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = 1 << 16;
        while (want < bytes) want <<= 1;
        if (cudaMallocHost(&p, want) != cudaSuccess) {
            p = nullptr;
            return GP_ENOMEM;
        }
        cap = want;
        return GP_OK;
    }
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
};

struct Request {
    int64_t id = 0;
    int kind = 0;  // 0 predict, 1 refit
    int model = -1;
    // predict
    const double* Xs = nullptr;
    int64_t Ns = 0;
    double* mean = nullptr;
    double* var = nullptr;
    // refit
    const double* X = nullptr;
    const double* y = nullptr;
    int64_t N = 0;
    size_t bytes = 0;  // scratch estimate charged against the budget
    Clock::time_point t_submit, t_start, t_end;
    int status = 1;  // 1 = pending / running, else a GP_* status
    // while running
    int slot = -1;
    gp_model* used = nullptr;  // the model a predict runs against
    gp_model* fresh = nullptr; // the model a refit builds
    Scratch* sc = nullptr;
    GpStatus* st = nullptr;
    FitStage stage;
    // refit: staged device inputs, and the float64-Gram retry
    double* xd = nullptr;
    double* ll = nullptr;
    Scratch* sc2 = nullptr;
    bool escalated = false;
};

}  // namespace

struct gp_server {
    int device = 0;
    int slots = 1;
    size_t budget = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done_ev;
    std::vector<Pinned> pin;
    std::vector<Request*> slot_req;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::vector<Resident> models;
    std::deque<Request*> pending;
    std::map<int64_t, Request*> all;
    int64_t next_id = 1;
    size_t mem_used = 0;
    int inflight = 0;
    int peak_inflight = 0;
    // statistics of finished predicts
    std::vector<double> lat_ms;
    int64_t points = 0;
    int64_t refits_done = 0;
    bool have_first = false;
    Clock::time_point first_submit, last_end;
};

namespace {

size_t predict_bytes(const gp_model* m, int64_t Ns) {
    const GpShape& s = m->shape;
    const size_t Npad = (size_t)gp_round_up(Ns, 128);
    size_t b = (size_t)Ns * s.p * 8 + 2 * (size_t)Ns * 8 + 256;  // X*, mean, var, status
    if (m->prec == GP_PREC_FP64)
        b += (size_t)s.p * s.n * Npad * 8 + predict64_part_elems((int64_t)Npad, s.M) * 8;
    else
        b += (size_t)s.p * s.n * Npad * 4;
    return b + (1 << 20);  // pool granularity slack
}

size_t refit_bytes(const gp_model* m, int64_t N, int sms) {
    const GpShape& s = m->shape;
    const size_t Npad = (size_t)gp_round_up(N, 128);
    const size_t M = (size_t)s.M;
    size_t b = (size_t)N * (s.p + 1) * 8;                        // X, y
    b += (m->prec == GP_PREC_FP64 ? 2 : 1) * M * M * 8 + 5 * M * 8; // new model: L, W (float64 fit), c, b, d
    if (m->prec != GP_PREC_FP64) b += predtc_wpack_bytes((int)M) + predtc_cinfo_ints(s) * 4;
    b += M * M * 8 + solve_refine_work_elems((int)M) * 8 + factor_work_bytes((int)M, true);
    b += (size_t)s.p * s.n * Npad * 8 + Npad * 8;                 // tables, padded y
    b += (Npad / GP_TAB_BLOCK + 1) * (size_t)s.Mpad * 5;          // block maxima and exponents
    b += (size_t)(sms + 1) * 4 * (size_t)s.Mpad * s.Mpad * 4 / 2; // split partial tiles (bound)
    return b + (4 << 20);
}

// Start request r on `slot` (worker thread, lock held).
int launch_request(gp_server* S, Request* r, int slot) {
    cudaStream_t st = S->streams[slot];
    Pinned& pin = S->pin[slot];
    r->slot = slot;
    r->sc = new Scratch(st);
    int rc;
    if ((rc = r->sc->get(&r->st, 1))) return rc;
    cudaMemsetAsync(r->st, 0, sizeof(GpStatus), st);
    if (r->kind == 0) {
        gp_model* m = r->used;
        const int p = m->shape.p;
        const size_t in = (size_t)r->Ns * p * 8, out = (size_t)r->Ns * 8;
        // pinned layout: X* | mean | var | status
        if ((rc = pin.reserve(in + 2 * out + sizeof(GpStatus)))) return set_err(rc);
        memcpy(pin.p, r->Xs, in);
        double *xd = nullptr, *md = nullptr, *vd = nullptr;
        if ((rc = r->sc->get(&xd, (size_t)r->Ns * p))) return rc;
        if ((rc = r->sc->get(&md, (size_t)r->Ns))) return rc;
        if (r->var && (rc = r->sc->get(&vd, (size_t)r->Ns))) return rc;
        cudaMemcpyAsync(xd, pin.p, in, cudaMemcpyHostToDevice, st);
        if ((rc = predict_compute(m, xd, r->Ns, md, vd, r->st, *r->sc, st))) return rc;
        char* hp = (char*)pin.p;
        cudaMemcpyAsync(hp + in, md, out, cudaMemcpyDeviceToHost, st);
        if (vd) cudaMemcpyAsync(hp + in + out, vd, out, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hp + in + 2 * out, r->st, sizeof(GpStatus), cudaMemcpyDeviceToHost, st);
    } else {
        const gp_model* old = S->models[r->model].model;
        const GpShape& s = old->shape;
        gp_model* h = new_model(S->device, old->prec, r->N, s.p, s.n, old->eps, old->alpha, old->sigma2);
        r->fresh = h;
        if ((rc = fit_alloc(h, st))) return rc;
        const size_t in = (size_t)r->N * (s.p + 1) * 8;
        if ((rc = pin.reserve(in + sizeof(GpStatus)))) return set_err(rc);
        memcpy(pin.p, r->X, (size_t)r->N * s.p * 8);
        memcpy((char*)pin.p + (size_t)r->N * s.p * 8, r->y, (size_t)r->N * 8);
        // one device buffer holds X (N x p) followed by y (N), as staged
        double *xd = nullptr, *ll = nullptr;
        if ((rc = r->sc->get(&xd, (size_t)r->N * (s.p + 1)))) return rc;
        if ((rc = r->sc->get(&ll, (size_t)s.p * s.n))) return rc;
        cudaMemcpyAsync(xd, pin.p, in, cudaMemcpyHostToDevice, st);
        const double* yd = xd + (size_t)r->N * s.p;
        r->xd = xd;
        r->ll = ll;
        if ((rc = fit_stage(h, r->stage, ll, st))) return rc;
        if ((rc = fit_compute(h, xd, yd, ll, r->st, 0, *r->sc, st))) return rc;
        cudaMemcpyAsync((char*)pin.p + in, r->st, sizeof(GpStatus), cudaMemcpyDeviceToHost, st);
    }
    cudaEventRecord(S->done_ev[slot], st);
    return GP_OK;
}

// A refit whose mixed Gram met a non-positive pivot: redo the fit on the same
// slot with the float64 Gram (its staged inputs are still on the device).
// Returns false if the retry could not be enqueued.
bool escalate_refit(gp_server* S, Request* r) {
    const int slot = r->slot;
    cudaStream_t st = S->streams[slot];
    const GpShape& s = r->fresh->shape;
    r->escalated = true;
    r->sc2 = new Scratch(st);
    GpStatus* st2 = nullptr;
    if (r->sc2->get(&st2, 1)) return false;
    cudaMemsetAsync(st2, 0, sizeof(GpStatus), st);
    const double* yd = r->xd + (size_t)r->N * s.p;
    if (fit_compute(r->fresh, r->xd, yd, r->ll, st2, 0, *r->sc2, st, GP_PREC_FP64)) return false;
    const size_t in = (size_t)r->N * (s.p + 1) * 8;
    cudaMemcpyAsync((char*)S->pin[slot].p + in, st2, sizeof(GpStatus), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(S->done_ev[slot], st);
    r->st = st2;
    return true;
}

// Request r has completed (or failed to launch): results out, accounting (lock held).
void finish_request(gp_server* S, Request* r, int launch_rc) {
    r->t_end = Clock::now();
    int code = launch_rc;
    Pinned& pin = S->pin[r->slot];
    if (code == GP_OK) {
        if (cudaEventSynchronize(S->done_ev[r->slot]) != cudaSuccess) code = GP_ECUDA;
    } else {
        cudaStreamSynchronize(S->streams[r->slot]);
    }
    if (code == GP_OK) {
        GpStatus hs;
        if (r->kind == 0) {
            const size_t in = (size_t)r->Ns * r->used->shape.p * 8, out = (size_t)r->Ns * 8;
            const char* hp = (const char*)pin.p;
            memcpy(&hs, hp + in + 2 * out, sizeof(hs));
            if (hs.code == GP_OK) {
                memcpy(r->mean, hp + in, out);
                if (r->var) memcpy(r->var, hp + in + out, out);
            }
        } else {
            memcpy(&hs, (const char*)pin.p + (size_t)r->N * (S->models[r->model].model->shape.p + 1) * 8,
                   sizeof(hs));
            if (!r->escalated && mixed_escalates(r->fresh, hs.code) && escalate_refit(S, r))
                return;  // still running: finished when the retry completes
        }
        code = hs.code;
    }
    delete r->sc;  // stream-ordered frees behind the finished work
    r->sc = nullptr;
    delete r->sc2;
    r->sc2 = nullptr;
    r->status = code;
    S->slot_req[r->slot] = nullptr;
    S->mem_used -= r->bytes;
    S->inflight -= 1;
    if (r->kind == 0) {
        // release the user count on the model this request ran against
        for (Resident& res : S->models)
            if (res.model == r->used) {
                res.users -= 1;
                break;
            }
        // a retired model is kept in a side list until its users drain
        if (code == GP_OK) {
            S->lat_ms.push_back(ms_between(r->t_submit, r->t_end));
            S->points += r->Ns;
        }
    } else {
        Resident& res = S->models[r->model];
        if (code == GP_OK) {
            gp_model* old = res.model;
            res.model = r->fresh;
            r->fresh = nullptr;
            S->refits_done += 1;
            if (res.users == 0) {
                free_model(old);
            } else {
                Resident ret;
                ret.model = old;
                ret.users = res.users;
                ret.retired = true;
                res.users = 0;
                S->models.push_back(ret);
            }
        } else if (r->fresh) {
            free_model(r->fresh);
            r->fresh = nullptr;
        }
    }
    // free retired models whose users have drained
    for (Resident& res : S->models)
        if (res.retired && res.users == 0 && res.model) {
            free_model(res.model);
            res.model = nullptr;
        }
    S->last_end = r->t_end;
}

void worker_loop(gp_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // completions
        for (int k = 0; k < S->slots; ++k) {
            Request* r = S->slot_req[k];
            if (r && cudaEventQuery(S->done_ev[k]) == cudaSuccess) finish_request(S, r, GP_OK);
        }
        (void)cudaGetLastError();  // cudaEventQuery's "not ready" is not an error here
        // admissions, in arrival order
        while (!S->pending.empty() && S->inflight < S->slots) {
            Request* r = S->pending.front();
            if (S->inflight > 0 && S->mem_used + r->bytes > S->budget) break;
            int slot = 0;
            while (S->slot_req[slot]) ++slot;
            S->pending.pop_front();
            if (r->kind == 0) {
                r->used = S->models[r->model].model;
                S->models[r->model].users += 1;
            }
            S->slot_req[slot] = r;
            S->mem_used += r->bytes;
            S->inflight += 1;
            S->peak_inflight = std::max(S->peak_inflight, S->inflight);
            r->t_start = Clock::now();
            r->slot = slot;
            const int rc = launch_request(S, r, slot);
            if (rc != GP_OK) finish_request(S, r, rc);
        }
        S->cv_done.notify_all();
        if (S->stop && S->pending.empty() && S->inflight == 0) break;
        if (S->inflight == 0) {
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        } else {
            // poll the running requests
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
    S->cv_done.notify_all();
}

int64_t submit(gp_server* S, Request* r) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    if (!S->have_first) {
        S->have_first = true;
        S->first_submit = r->t_submit;
    }
    S->all[r->id] = r;
    S->pending.push_back(r);
    S->cv_work.notify_one();
    return r->id;
}

}  // namespace

extern "C" {

GPFAGP_API int gp_server_create(int slots, int64_t mem_budget_bytes, gp_server** out) {
    set_err(GP_OK);
    if (!out || slots < 1 || slots > 64) return set_err(GP_EINVAL, 0);
    *out = nullptr;
    int rc, dev;
    if ((rc = check_device(&dev))) return rc;
    gp_server* S = new gp_server();
    S->device = dev;
    S->slots = slots;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    S->budget = mem_budget_bytes > 0 ? (size_t)mem_budget_bytes : freeb / 2;
    S->streams.resize(slots);
    S->done_ev.resize(slots);
    S->pin.resize(slots);
    S->slot_req.assign(slots, nullptr);
    for (int k = 0; k < slots; ++k) {
        cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&S->done_ev[k], cudaEventDisableTiming);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return GP_OK;
}

GPFAGP_API int gp_server_add_model(gp_server* S, gp_model* m, int* model_id) {
    set_err(GP_OK);
    if (!S || !m || !model_id) return set_err(GP_EINVAL, 0);
    if (m->device != S->device) return set_err(GP_EINVAL, 1);
    std::lock_guard<std::mutex> lk(S->mu);
    Resident r;
    r.model = m;
    S->models.push_back(r);
    *model_id = (int)S->models.size() - 1;
    return GP_OK;
}

GPFAGP_API gp_model* gp_server_model(gp_server* S, int model_id) {
    if (!S) return nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    if (model_id < 0 || model_id >= (int)S->models.size() || S->models[model_id].retired) return nullptr;
    return S->models[model_id].model;
}

GPFAGP_API int gp_server_submit_predict(gp_server* S, int model_id, const double* Xs, int64_t Ns,
                                        double* mean, double* var, int64_t* req_id) {
    set_err(GP_OK);
    if (!S || !req_id || !Xs || !mean || Ns < 1) return set_err(GP_EINVAL, 0);
    Request* r = new Request();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (model_id < 0 || model_id >= (int)S->models.size() || S->models[model_id].retired) {
            delete r;
            return set_err(GP_EINVAL, 1);
        }
        r->bytes = predict_bytes(S->models[model_id].model, Ns);
    }
    r->kind = 0;
    r->model = model_id;
    r->Xs = Xs;
    r->Ns = Ns;
    r->mean = mean;
    r->var = var;
    *req_id = submit(S, r);
    return GP_OK;
}

GPFAGP_API int gp_server_submit_refit(gp_server* S, int model_id, const double* X, const double* y,
                                      int64_t N, int64_t* req_id) {
    set_err(GP_OK);
    if (!S || !req_id || !X || !y || N < 1) return set_err(GP_EINVAL, 0);
    Request* r = new Request();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (model_id < 0 || model_id >= (int)S->models.size() || S->models[model_id].retired) {
            delete r;
            return set_err(GP_EINVAL, 1);
        }
        r->bytes = refit_bytes(S->models[model_id].model, N, num_sms(S->device));
    }
    r->kind = 1;
    r->model = model_id;
    r->X = X;
    r->y = y;
    r->N = N;
    *req_id = submit(S, r);
    return GP_OK;
}

GPFAGP_API int gp_server_wait(gp_server* S, int64_t req_id, double timeout_s) {
    set_err(GP_OK);
    if (!S) return set_err(GP_EINVAL, 0);
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(req_id);
    if (it == S->all.end()) return set_err(GP_EINVAL, 1);
    Request* r = it->second;
    const auto until = Clock::now() + std::chrono::microseconds((int64_t)(timeout_s * 1e6));
    while (r->status == 1) {
        if (timeout_s > 0) {
            if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->status == 1)
                return set_err(GP_ETIMEOUT, req_id);
        } else {
            S->cv_done.wait(lk);
        }
    }
    const int code = r->status;
    S->all.erase(it);
    delete r;
    if (code != GP_OK) return set_err(code, req_id);
    return GP_OK;
}

GPFAGP_API int gp_server_stats(gp_server* S, gp_server_report* out) {
    set_err(GP_OK);
    if (!S || !out) return set_err(GP_EINVAL, 0);
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->predicts_done = (int64_t)S->lat_ms.size();
    out->refits_done = S->refits_done;
    out->points = S->points;
    out->peak_inflight = S->peak_inflight;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) {
            const size_t i = (size_t)floor(f * (double)(v.size() - 1) + 0.5);
            return v[i < v.size() ? i : v.size() - 1];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
    }
    if (S->have_first) {
        out->wall_s = ms_between(S->first_submit, S->last_end) / 1e3;
        out->points_per_s = out->wall_s > 0 ? (double)S->points / out->wall_s : 0.0;
    }
    return GP_OK;
}

GPFAGP_API int gp_server_reset_stats(gp_server* S) {
    set_err(GP_OK);
    if (!S) return set_err(GP_EINVAL, 0);
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_ms.clear();
    S->points = 0;
    S->refits_done = 0;
    S->peak_inflight = S->inflight;
    S->have_first = false;
    return GP_OK;
}

GPFAGP_API void gp_server_destroy(gp_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->all) delete kv.second;
    for (Resident& res : S->models)
        if (res.model) free_model(res.model);  // the server owns every model it holds
    for (int k = 0; k < S->slots; ++k) {
        cudaStreamDestroy(S->streams[k]);
        cudaEventDestroy(S->done_ev[k]);
    }
    delete S;
}

}  // extern "C"
