// gp_server.cu -- a request server for resident fitted models (C ABI in
// include/gpfagp.h): continuous batching of predict and refit requests.
//
// The server owns a worker thread, `slots` CUDA streams and a device-memory
// budget for request scratch. Models stay resident on the device. Requests
// (predict: X* -> mean, var; refit: new training set for a resident model)
// queue in arrival order. Whenever a slot is free the worker starts a job
// on it: a refit at the queue head, or every predict queued at the head (up
// to a request and point limit, and within the budget) packed into one
// batch. A batch makes one host-to-device copy of all its test points and
// of a request table, one launch that evaluates all their eigenfunction
// tables, one persistent tensor-core predict launch per basis dimension p
// whose CTAs walk the (request, 128-point tile) items, and one copy of all
// results back (float64 models run their own predict kernels inside the
// batch). So requests that arrive while the GPU is busy leave together
// with little per-request cost, and each request's result is the same as
// gp_predict_ex's on it alone (the same per-point arithmetic and order).
//
// Host buffers are staged through pinned per-slot memory so that no copy
// blocks the worker; results are copied to the caller's buffers when the
// job's completion event has fired. A refit builds a new model on its slot
// and swaps it in at completion; requests already admitted against the old
// model finish on it, and it is freed when the last of them completes. The
// server owns the models registered with it and frees them at destroy.
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
    int64_t xoff = 0, ooff = 0;  // its rows in the batch's packed X* and outputs
    // refit
    const double* X = nullptr;
    const double* y = nullptr;
    int64_t N = 0;
    size_t bytes = 0;  // scratch estimate charged against the budget
    Clock::time_point t_submit, t_start, t_end;
    int status = 1;  // 1 = pending / running, else a GP_* status
    gp_model* used = nullptr;  // the model a predict runs against
};

// What a slot runs: a batch of predicts, or one refit.
struct Job {
    int kind = 0;  // 0 predicts, 1 refit
    std::vector<Request*> reqs;
    size_t bytes = 0;
    Scratch* sc = nullptr;
    // predicts: pinned layout [X* | request table image | mean | var | statuses]
    size_t xbytes = 0, img_bytes = 0;
    int64_t points = 0;
    // refit
    gp_model* fresh = nullptr;
    GpStatus* st = nullptr;
    FitStage stage;
    double* xd = nullptr;  // staged device inputs (X then y) for the float64-Gram retry
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
    std::vector<Job*> slot_job;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::vector<Resident> models;
    std::deque<Request*> pending;
    std::map<int64_t, Request*> all;
    int64_t next_id = 1;
    size_t mem_used = 0;
    int inflight = 0;       // jobs on the slots
    int inflight_reqs = 0;  // requests in those jobs
    int peak_inflight = 0;  // most requests on the device at once
    int peak_batch = 0;     // most predicts in one batch
    int64_t batches = 0;    // predict batches started
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
        b += (size_t)s.p * s.n * Npad * 4 + predtc_vpart_elems((int64_t)Npad, s.M) * 8;
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
    b += (Npad / GP_TAB_BLOCK + 2) * (size_t)s.Mpad * 6 + (size_t)s.Mpad * 4;  // block maxima and exponents
    b += (Npad / GP_TAB_BLOCK + 2 * (size_t)sms + 2) * (size_t)s.Mpad * 4;       // partials of b (bound)
    b += (size_t)(sms + 1) * 4 * (size_t)s.Mpad * s.Mpad * 4 / 2; // split partial tiles (bound)
    return b + (4 << 20);
}

constexpr int kBatchRequests = 256;          // most predicts in one batch
constexpr int64_t kBatchPoints = 1 << 20;      // most test points in one batch (unless one request has more)

// Start a batch of predicts on `slot` (worker thread, lock held).
int launch_predicts(gp_server* S, Job* J, int slot) {
    cudaStream_t st = S->streams[slot];
    Pinned& pin = S->pin[slot];
    J->sc = new Scratch(st);
    Scratch& sc = *J->sc;
    const int cnt = (int)J->reqs.size();
    int64_t xs = 0, pts = 0;
    for (Request* r : J->reqs) {
        r->xoff = xs;
        r->ooff = pts;
        xs += r->Ns * r->used->shape.p;
        pts += r->Ns;
    }
    J->points = pts;
    J->xbytes = (size_t)xs * 8;
    const size_t obytes = 2 * (size_t)pts * 8 + sizeof(GpStatus) * cnt;  // mean | var | statuses
    int rc;
    double* xd = nullptr;
    uint8_t* od = nullptr;
    if ((rc = sc.get(&xd, (size_t)xs))) return rc;
    if ((rc = sc.get(&od, obytes))) return rc;
    double* md = reinterpret_cast<double*>(od);
    double* vd = md + pts;
    GpStatus* sts = reinterpret_cast<GpStatus*>(vd + pts);
    cudaMemsetAsync(sts, 0, sizeof(GpStatus) * cnt, st);
    std::vector<PredEntry> mixed;
    std::vector<int> f64;
    for (int i = 0; i < cnt; ++i) {
        Request* r = J->reqs[i];
        if (r->used->prec == GP_PREC_FP64) {
            f64.push_back(i);
        } else {
            mixed.push_back(PredEntry{r->used, xd + r->xoff, r->Ns, md + r->ooff, r->var ? vd + r->ooff : nullptr,
                                      &sts[i]});
        }
    }
    PredBatch pb;
    uint8_t* up = nullptr;
    if ((rc = pred_batch_build(mixed, sc, pb))) return rc;
    if (pb.total && (rc = sc.get(&up, pb.total))) return rc;
    J->img_bytes = (pb.total + 15) & ~(size_t)15;
    if ((rc = pin.reserve(J->xbytes + J->img_bytes + obytes))) return set_err(rc);
    uint8_t* hp = (uint8_t*)pin.p;
    for (Request* r : J->reqs) memcpy(hp + r->xoff * 8, r->Xs, (size_t)r->Ns * r->used->shape.p * 8);
    if (pb.total) pred_batch_pack(pb, hp + J->xbytes, up);
    cudaMemcpyAsync(xd, hp, J->xbytes, cudaMemcpyHostToDevice, st);
    if (pb.total) cudaMemcpyAsync(up, hp + J->xbytes, pb.total, cudaMemcpyHostToDevice, st);
    if ((rc = pred_batch_enqueue(pb, up, st))) return rc;
    for (int i : f64) {
        Request* r = J->reqs[i];
        if ((rc = predict_compute(r->used, xd + r->xoff, r->Ns, md + r->ooff, r->var ? vd + r->ooff : nullptr,
                                  &sts[i], sc, st)))
            return rc;
    }
    cudaMemcpyAsync(hp + J->xbytes + J->img_bytes, od, obytes, cudaMemcpyDeviceToHost, st);
    cudaEventRecord(S->done_ev[slot], st);
    return GP_OK;
}

// Start a refit on `slot` (worker thread, lock held).
int launch_refit(gp_server* S, Job* J, int slot) {
    cudaStream_t st = S->streams[slot];
    Pinned& pin = S->pin[slot];
    Request* r = J->reqs[0];
    J->sc = new Scratch(st);
    int rc;
    if ((rc = J->sc->get(&J->st, 1))) return rc;
    cudaMemsetAsync(J->st, 0, sizeof(GpStatus), st);
    const gp_model* old = S->models[r->model].model;
    const GpShape& s = old->shape;
    gp_model* h = new_model(S->device, old->prec, r->N, s.p, s.n, old->eps, old->alpha, old->sigma2);
    J->fresh = h;
    if ((rc = fit_alloc(h, st))) return rc;
    const size_t in = (size_t)r->N * (s.p + 1) * 8;
    if ((rc = pin.reserve(in + sizeof(GpStatus)))) return set_err(rc);
    memcpy(pin.p, r->X, (size_t)r->N * s.p * 8);
    memcpy((char*)pin.p + (size_t)r->N * s.p * 8, r->y, (size_t)r->N * 8);
    // one device buffer holds X (N x p) followed by y (N), as staged
    double *xd = nullptr, *ll = nullptr;
    if ((rc = J->sc->get(&xd, (size_t)r->N * (s.p + 1)))) return rc;
    if ((rc = J->sc->get(&ll, (size_t)s.p * s.n))) return rc;
    cudaMemcpyAsync(xd, pin.p, in, cudaMemcpyHostToDevice, st);
    const double* yd = xd + (size_t)r->N * s.p;
    J->xd = xd;
    J->ll = ll;
    if ((rc = fit_stage(h, J->stage, ll, st))) return rc;
    if ((rc = fit_compute(h, xd, yd, ll, J->st, 0, *J->sc, st))) return rc;
    cudaMemcpyAsync((char*)pin.p + in, J->st, sizeof(GpStatus), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(S->done_ev[slot], st);
    return GP_OK;
}

// A refit whose mixed Gram met a non-positive pivot: redo the fit on the same
// slot with the float64 Gram (its staged inputs are still on the device).
// Returns false if the retry could not be enqueued.
bool escalate_refit(gp_server* S, Job* J, int slot) {
    cudaStream_t st = S->streams[slot];
    Request* r = J->reqs[0];
    const GpShape& s = J->fresh->shape;
    J->escalated = true;
    J->sc2 = new Scratch(st);
    GpStatus* st2 = nullptr;
    if (J->sc2->get(&st2, 1)) return false;
    cudaMemsetAsync(st2, 0, sizeof(GpStatus), st);
    const double* yd = J->xd + (size_t)r->N * s.p;
    if (fit_compute(J->fresh, J->xd, yd, J->ll, st2, 0, *J->sc2, st, GP_PREC_FP64)) return false;
    const size_t in = (size_t)r->N * (s.p + 1) * 8;
    cudaMemcpyAsync((char*)S->pin[slot].p + in, st2, sizeof(GpStatus), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(S->done_ev[slot], st);
    J->st = st2;
    return true;
}

// release the user count on the model a predict ran against (lock held)
void release_model(gp_server* S, const gp_model* m) {
    for (Resident& res : S->models)
        if (res.model == m) {
            res.users -= 1;
            break;
        }
}

// The job on `slot` has completed (or failed to launch): results out,
// accounting (lock held).
void finish_job(gp_server* S, int slot, int launch_rc) {
    Job* J = S->slot_job[slot];
    const Clock::time_point now = Clock::now();
    int code = launch_rc;
    if (code == GP_OK) {
        if (cudaEventSynchronize(S->done_ev[slot]) != cudaSuccess) code = GP_ECUDA;
    } else {
        cudaStreamSynchronize(S->streams[slot]);
    }
    const Pinned& pin = S->pin[slot];
    if (J->kind == 0) {
        const uint8_t* hp = (const uint8_t*)pin.p;
        const double* hm = reinterpret_cast<const double*>(hp + J->xbytes + J->img_bytes);
        const double* hv = hm + J->points;
        const GpStatus* hs = reinterpret_cast<const GpStatus*>(hv + J->points);
        for (size_t i = 0; i < J->reqs.size(); ++i) {
            Request* r = J->reqs[i];
            int rc = code;
            if (rc == GP_OK) {
                rc = hs[i].code;
                if (rc == GP_OK) {
                    memcpy(r->mean, hm + r->ooff, (size_t)r->Ns * 8);
                    if (r->var) memcpy(r->var, hv + r->ooff, (size_t)r->Ns * 8);
                }
            }
            r->t_end = now;
            r->status = rc;
            release_model(S, r->used);
            if (rc == GP_OK) {
                S->lat_ms.push_back(ms_between(r->t_submit, r->t_end));
                S->points += r->Ns;
            }
        }
    } else {
        Request* r = J->reqs[0];
        if (code == GP_OK) {
            GpStatus hs;
            memcpy(&hs, (const char*)pin.p + (size_t)r->N * (S->models[r->model].model->shape.p + 1) * 8,
                   sizeof(hs));
            if (!J->escalated && mixed_escalates(J->fresh, hs.code) && escalate_refit(S, J, slot))
                return;  // still running: finished when the retry completes
            code = hs.code;
        }
        r->t_end = now;
        r->status = code;
        Resident& res = S->models[r->model];
        if (code == GP_OK) {
            gp_model* old = res.model;
            res.model = J->fresh;
            J->fresh = nullptr;
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
        } else if (J->fresh) {
            free_model(J->fresh);
            J->fresh = nullptr;
        }
    }
    delete J->sc;  // stream-ordered frees behind the finished work
    delete J->sc2;
    S->slot_job[slot] = nullptr;
    S->mem_used -= J->bytes;
    S->inflight -= 1;
    S->inflight_reqs -= (int)J->reqs.size();
    // free retired models whose users have drained
    for (Resident& res : S->models)
        if (res.retired && res.users == 0 && res.model) {
            free_model(res.model);
            res.model = nullptr;
        }
    S->last_end = now;
    delete J;
}

// The next job from the queue head, or nullptr if the budget does not allow
// one now (lock held).
Job* take_job(gp_server* S) {
    Request* head = S->pending.front();
    const bool idle = S->inflight == 0;
    if (head->kind == 1) {
        if (!idle && S->mem_used + head->bytes > S->budget) return nullptr;
        S->pending.pop_front();
        Job* J = new Job();
        J->kind = 1;
        J->reqs.push_back(head);
        J->bytes = head->bytes;
        return J;
    }
    Job* J = new Job();
    int64_t pts = 0;
    while (!S->pending.empty() && S->pending.front()->kind == 0 && (int)J->reqs.size() < kBatchRequests) {
        Request* r = S->pending.front();
        const bool first = J->reqs.empty();
        if (!first && pts + r->Ns > kBatchPoints) break;
        if (!(first && idle) && S->mem_used + J->bytes + r->bytes > S->budget) break;
        S->pending.pop_front();
        r->used = S->models[r->model].model;
        S->models[r->model].users += 1;
        J->reqs.push_back(r);
        J->bytes += r->bytes;
        pts += r->Ns;
    }
    if (J->reqs.empty()) {
        delete J;
        return nullptr;
    }
    return J;
}

void worker_loop(gp_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // completions
        for (int k = 0; k < S->slots; ++k)
            if (S->slot_job[k] && cudaEventQuery(S->done_ev[k]) == cudaSuccess) finish_job(S, k, GP_OK);
        (void)cudaGetLastError();  // cudaEventQuery's "not ready" is not an error here
        // admissions, in arrival order
        while (!S->pending.empty() && S->inflight < S->slots) {
            Job* J = take_job(S);
            if (J == nullptr) break;
            int slot = 0;
            while (S->slot_job[slot]) ++slot;
            S->slot_job[slot] = J;
            S->mem_used += J->bytes;
            S->inflight += 1;
            S->inflight_reqs += (int)J->reqs.size();
            S->peak_inflight = std::max(S->peak_inflight, S->inflight_reqs);
            const Clock::time_point now = Clock::now();
            for (Request* r : J->reqs) r->t_start = now;
            if (J->kind == 0) {
                S->batches += 1;
                S->peak_batch = std::max(S->peak_batch, (int)J->reqs.size());
            }
            const int rc = J->kind == 0 ? launch_predicts(S, J, slot) : launch_refit(S, J, slot);
            if (rc != GP_OK) finish_job(S, slot, rc);
        }
        S->cv_done.notify_all();
        if (S->stop && S->pending.empty() && S->inflight == 0) break;
        if (S->inflight == 0) {
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        } else {
            // poll the running jobs
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
    S->slot_job.assign(slots, nullptr);
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
    out->peak_batch = S->peak_batch;
    out->batches = S->batches;
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
    S->peak_inflight = S->inflight_reqs;
    S->peak_batch = 0;
    S->batches = 0;
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
