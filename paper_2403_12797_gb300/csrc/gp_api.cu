// gp_api.cu -- the C ABI (include/gpfagp.h): argument checks, device memory,
// and the order of kernel launches for fit and predict.
//
// fit (Sec. 2.2 in the M x M form):
//   eigenfunction tables (Eq. 14-16) -> fused Phi generation + Gram
//   (Phi^T Phi, Phi^T y) -> split reduction + A = G + sigma^2 Lambda^{-1}
//   -> A = L L^T -> W = L^{-1} -> c = A^{-1} b with float64 refinement
// predict (Eq. 11-12, diagonal): tables of X* -> fused Phi_* generation,
//   mean = Phi_* c, var = sigma^2 rowsum((Phi_* W^T)^2).
#include "gp_internal.cuh"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>


namespace gpi {

thread_local int g_err = GP_OK;
thread_local int64_t g_detail = 0;
std::atomic<int> g_fail_after{0};
// which mixed-precision Gram kernel runs: 0 automatic (CTA pairs for M > 384),
// 1 always one CTA per 128 x 128 tile pair, 2 CTA pairs wherever they apply
std::atomic<int> g_gram_kernel{0};
std::mutex g_pool_mu;
std::vector<int> g_pool_ready;

int set_err(int code, int64_t detail) {
    g_err = code;
    g_detail = detail;
    return code;
}

thread_local const char* g_where = "";

int cuda_err(cudaError_t e, const char* where) {
    g_where = where;
    return set_err(GP_ECUDA, (int64_t)e);
}

// Keep the stream-ordered pool's memory across calls (no release at every
// synchronisation), so repeated fits and predicts do not remap memory.
void prepare_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d : g_pool_ready)
        if (d == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_ready.push_back(dev);
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    int k = g_fail_after.load();
    while (k > 0) {
        if (g_fail_after.compare_exchange_weak(k, k - 1)) {
            if (k == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    if (bytes == 0) bytes = 16;
    return cudaMallocAsync(p, bytes, s);
}


int check_device(int* dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_err(GP_ENODEV, (int64_t)e);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return set_err(GP_ENODEV, major * 10 + minor);
    prepare_pool(dev);
    *dev_out = dev;
    return GP_OK;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

int check_hyper(int64_t N, int p, int n, double eps, double alpha, double sigma2) {
    if (N < 1 || p < 1 || p > GP_PMAX || n < 1) return set_err(GP_EINVAL, 1);
    if (!finite_pos(eps) || !finite_pos(alpha) || !finite_pos(sigma2)) return set_err(GP_EINVAL, 2);
    double M = pow((double)n, (double)p);
    if (M > (double)GP_MAX_M) return set_err(GP_EINVAL, 3);
    return GP_OK;
}

// log lambda_k, k = 0..n-1 (Eq. 16 with delta^2 of Eq. 14, rho^2 reading)
void log_eigenvalues(int n, double eps, double alpha, double* out) {
    const double beta = pow(1.0 + (2.0 * eps / alpha) * (2.0 * eps / alpha), 0.25);
    const double delta2 = alpha * alpha * (beta * beta - 1.0) / 2.0;
    const double D = alpha * alpha + delta2 + eps * eps;
    for (int k = 0; k < n; ++k) out[k] = 0.5 * log(alpha * alpha / D) + k * log(eps * eps / D);
}

template <typename T>
__global__ void pad_y_kernel(const double* __restrict__ y, int64_t N, int64_t Npad, T* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Npad) out[i] = i < N ? (T)y[i] : T(0);
}

int read_status(GpStatus* st, cudaStream_t s) {
    PinnedBlock pb = pinned_get(sizeof(GpStatus));
    GpStatus local;
    GpStatus* hp = pb.p ? (GpStatus*)pb.p : &local;
    cudaError_t e = cudaMemcpyAsync(hp, st, sizeof(GpStatus), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const GpStatus h = *hp;
    if (pb.p) pinned_put(pb);
    if (e != cudaSuccess) return cuda_err(e, "status read");
    if (h.code != GP_OK) return set_err(h.code, h.detail);
    return GP_OK;
}

// Split the (padded) rows among CTAs: every split is a multiple of `granule`
// rows, and the split count minimises (waves of tile pairs x splits over
// `target_ctas` resident CTAs) x (rows per split + a fixed cost of one block
// of rows per CTA: pipeline fill, drain, partial tile) -- the time of the
// longest CTA chain -- preferring fewer splits on ties (less partial-tile
// memory to reduce), within eight waves. E.g. 528 tile pairs on 152 CTAs:
// one split takes 4 waves of the whole row range, two splits 7 waves of half
// of it.
void choose_splits(int npairs, int64_t Npad, int target_ctas, int64_t granule, int* nsplit,
                   int64_t* rps, int max_waves = 8) {
    if (target_ctas < 1) target_ctas = 1;
    int64_t maxs = Npad / 256;  // at least 256 rows per split
    if (maxs < 1) maxs = 1;
    if (maxs > 4096) maxs = 4096;
    int64_t best_r = gp_round_up(Npad, granule), best_cost = -1;
    for (int64_t want = 1; want <= maxs; ++want) {
        const int64_t r = gp_round_up((Npad + want - 1) / want, granule);
        const int64_t ns = (Npad + r - 1) / r;
        const int64_t waves = (npairs * ns + target_ctas - 1) / target_ctas;
        if (ns > 1 && ns * npairs > (int64_t)max_waves * target_ctas) break;
        const int64_t cost = waves * (r + 1024);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_r = r;
        }
    }
    *rps = best_r;
    *nsplit = (int)((Npad + best_r - 1) / best_r);
}

// Row splits of the tensor-core Gram per pair class (SyrkSplit). When all
// tile pairs fit in one wave of target_ctas CTAs, each class gets its own
// split count: starting from one split each, the class whose CTAs would take
// longest -- (blocks per split + 1) x its cost per block -- gets one more
// split while the whole grid still fits in the wave. Costs per 1024-row block
// relative to a diagonal pair, measured per CTA on GB300 (p = 2, n = 20):
// 1.24 for the pairs (I, 0), which also form Phi^T y, and 1.17 for the other
// off-diagonal pairs; a diagonal pair generates one operand tile instead of
// two. Otherwise every class takes the uniform choice of choose_splits.
//
// The CTA-pair kernel (tiles of 256) takes the same plan with clusters in
// place of CTAs, class costs `wc`, up to `max_waves` waves and splits of whole
// GP_PAIR_BLOCK-row blocks (`granule`).
const double kClassCost1[3] = {1.0, 1.24, 1.17};
const double kClassCost2[3] = {1.0, 1.05, 1.0};
void choose_splits_tc(int T, int64_t Npad, int target_ctas, SyrkSplit* sp, const double* wc = kClassCost1,
                      int max_waves = 8, int granule = GP_TAB_BLOCK) {
    if (target_ctas < 1) target_ctas = 1;
    const int npairs = T * (T + 1) / 2;
    const int64_t npc[3] = {T, T - 1, (int64_t)(T - 1) * (T - 2) / 2};
    if (npairs > target_ctas) {
        int ns;
        int64_t rps;
        choose_splits(npairs, Npad, target_ctas, granule, &ns, &rps, max_waves);
        for (int c = 0; c < 3; ++c) {
            sp->n[c] = ns;
            sp->rows[c] = rps;
        }
        sp->smax = ns;
        return;
    }
    const int64_t nb = (Npad + granule - 1) / granule;
    const double* w = wc;
    int64_t n[3] = {1, 1, 1};
    auto cost = [&](int c) { return (double)((nb + n[c] - 1) / n[c] + 1) * w[c]; };
    while (true) {
        int cmax = -1;
        for (int c = 0; c < 3; ++c)
            if (npc[c] > 0 && (cmax < 0 || cost(c) > cost(cmax))) cmax = c;
        if ((nb + n[cmax] - 1) / n[cmax] <= 1) break;  // one block per split already
        int64_t ctas = 0;
        for (int c = 0; c < 3; ++c) ctas += npc[c] * n[c];
        if (ctas + npc[cmax] > target_ctas) break;
        ++n[cmax];
    }
    sp->smax = 1;
    for (int c = 0; c < 3; ++c) {
        const int64_t blocks = (nb + n[c] - 1) / n[c];
        sp->rows[c] = blocks * granule;
        sp->n[c] = (int)((Npad + sp->rows[c] - 1) / sp->rows[c]);
        if (npc[c] > 0 && sp->n[c] > sp->smax) sp->smax = sp->n[c];
    }
}

int num_sms(int dev) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// The fused Gram step: A (M x M) = Phi^T Phi [+ diag(d)], b = Phi^T y.
// X, y are device pointers.
// ex (optional, the fit's): the noise diagonal ex->dout from ex->loglam, and
// A's lower triangle in ex->L. The mixed assembly does both in its kernel
// (*l_written = true); the float64 path launches the diagonal kernel first and
// leaves L to the caller.
// The mixed Gram of one problem on the one-CTA kernel (128 x 128 tile
// pairs), in three steps so that a batch can contract many problems in one
// launch: prepare (scratch, split plan, chunk-major tables, column
// exponents), contract (launch_syrk_tc, or a batched launch), assemble.
struct MixedGram {
    GpShape sg;
    SyrkSplit spl;
    float* tabc = nullptr;
    float2* Gpart = nullptr;
    double* bpart = nullptr;
    int* colexp = nullptr;
    signed char* ebx = nullptr;
};

int mixed_gram_prepare(const GpShape& s, int dev, const double* Xd, const double* yd, GpStatus* st, Scratch& sc,
                       cudaStream_t stream, int target_ctas, MixedGram& g, bool exponents) {
    int rc;
    g.sg = s;
    const GpShape& sg = g.sg;
    const int T = sg.Mpad / SYRKTC_TM;
    const int npairs = T * (T + 1) / 2;
    choose_splits_tc(T, sg.Npad, target_ctas > 0 ? target_ctas : num_sms(dev), &g.spl);
    if ((rc = sc.get(&g.tabc, syrktc_table_floats(sg)))) return rc;
    if ((rc = sc.get(&g.Gpart, (size_t)g.spl.smax * npairs * SYRKTC_TM * SYRKTC_TM))) return rc;
    if ((rc = sc.get(&g.bpart, (size_t)g.spl.smax * sg.Mpad))) return rc;
    if ((rc = sc.get(&g.colexp, (size_t)sg.Mpad))) return rc;
    if ((rc = sc.get(&g.ebx, syrktc_ebx_bytes(sg)))) return rc;
    {
        GpProf pf("eig_tables", stream);
        launch_eig_tables_chunked(sg, Xd, yd, g.tabc, st, stream);
        gp_note_launches(1);
    }
    if (exponents) {
        GpProf pf("colexp", stream);
        launch_colexp(sg, g.tabc, g.colexp, g.ebx, stream);
        gp_note_launches(2);
    }
    return GP_OK;
}

void mixed_gram_assemble(const MixedGram& g, int M, const double* d, double* A, double* b, cudaStream_t stream,
                         const AssembleExtra* ex, bool* l_written) {
    GpProf pf("assemble", stream);
    launch_assemble_scaled(g.Gpart, g.bpart, g.colexp, g.spl, SYRKTC_TM, g.sg.Mpad, M, d, A, b, stream, ex);
    gp_note_launches(1);
    if (ex != nullptr && ex->L != nullptr && l_written) *l_written = true;
}

int gram_device(const GpShape& s, int prec, int dev, const double* Xd, const double* yd,
                const double* d, double* A, double* b, GpStatus* st, cudaStream_t stream,
                int target_ctas = 0, const AssembleExtra* ex = nullptr, bool* l_written = nullptr) {
    if (l_written) *l_written = false;
    Scratch sc(stream);
    int rc;
    if (prec == GP_PREC_FP64) {
        double *tab, *ypad, *Gpart, *bpart;
        if ((rc = sc.get(&tab, (size_t)s.p * s.n * s.Npad))) return rc;
        if ((rc = sc.get(&ypad, (size_t)s.Npad))) return rc;
        const int T = s.Mpad / SYRK64_TM;
        const int npairs = T * (T + 1) / 2;
        int nsplit;
        int64_t rps;
        choose_splits(npairs, s.Npad, target_ctas > 0 ? target_ctas : 4 * num_sms(dev), 128, &nsplit, &rps);
        if ((rc = sc.get(&Gpart, (size_t)nsplit * npairs * SYRK64_TM * SYRK64_TM))) return rc;
        if ((rc = sc.get(&bpart, (size_t)nsplit * s.Mpad))) return rc;
        {
            GpProf pf("eig_tables", stream);
            launch_eig_tables_f64(s, Xd, yd, tab, st, stream);
            pad_y_kernel<double><<<(unsigned)((s.Npad + 255) / 256), 256, 0, stream>>>(yd, s.N, s.Npad, ypad);
            gp_note_launches(2);
        }
        {
            GpProf pf("syrk64", stream);
            cudaError_t e = launch_syrk64(s, tab, ypad, nsplit, rps, Gpart, bpart, stream);
            if (e != cudaSuccess) return cuda_err(e, "syrk64 launch");
            gp_note_launches(1);
        }
        {
            GpProf pf("assemble", stream);
            if (ex != nullptr) {
                launch_noise_diag(*ex->shape, ex->loglam, ex->sigma2, ex->dout, stream);
                d = ex->dout;
                gp_note_launches(1);
            }
            launch_assemble_f64(Gpart, bpart, nsplit, SYRK64_TM, s.Mpad, s.M, d, A, b, stream);
            gp_note_launches(1);
        }
    } else {
        // the CTA-pair kernel (256 x 256 tile pairs) for M > 384 where it
        // applies (from there both kernels pad M to the same multiple of 256,
        // or the pairs' padding is outweighed: measured at M = 400, 0.28 ms
        // against 0.31 ms), else one CTA per 128 x 128 tile pair
        GpShape sg = s;
        bool pair = false;
        const int kind = g_gram_kernel.load();
        if (kind != 1 && s.M > (kind == 2 ? 0 : 384)) {
            sg.Mpad = (int)gp_round_up(s.M, 256);
            pair = syrktc2_supported(sg);
            if (!pair) sg.Mpad = s.Mpad;
        }
        if (!pair) {
            MixedGram g;
            if ((rc = mixed_gram_prepare(s, dev, Xd, yd, st, sc, stream, target_ctas, g, true))) return rc;
            {
                GpProf pf("syrk_tc", stream);
                cudaError_t e = launch_syrk_tc(g.sg, g.tabc, g.spl, g.Gpart, g.bpart, g.colexp, g.ebx, st, stream);
                if (e != cudaSuccess) return cuda_err(e, "syrk_tc launch");
                gp_note_launches(1);
            }
            mixed_gram_assemble(g, s.M, d, A, b, stream, ex, l_written);
            cudaError_t e = cudaGetLastError();
            return e == cudaSuccess ? GP_OK : cuda_err(e, "Gram step");
        }
        // CTA pairs: 256 x 256 tile pairs, float64 partial tiles
        constexpr int TT = 256;
        float* tabc;
        double* Gpart2;
        float* bblk = nullptr;  // b's partials per block and row range (the exponent pass forms b)
        if ((rc = sc.get(&tabc, syrktc_table_floats(sg)))) return rc;
        const int T = sg.Mpad / TT;
        const int npairs = T * (T + 1) / 2;
        SyrkSplit spl;
        int clusters = syrktc2_max_clusters(sg, dev);
        if (target_ctas > 0) clusters = std::max(1, std::min(clusters, target_ctas / 2));
        choose_splits_tc(T, sg.Npad, clusters, &spl, kClassCost2, 16, GP_PAIR_BLOCK);
        if ((rc = sc.get(&Gpart2, (size_t)spl.smax * npairs * TT * TT))) return rc;
        if (b != nullptr && (rc = sc.get(&bblk, colexp_b_floats(sg)))) return rc;
        int* colexp;
        signed char* ebx;
        if ((rc = sc.get(&colexp, (size_t)sg.Mpad))) return rc;
        if ((rc = sc.get(&ebx, syrktc_ebx_bytes(sg)))) return rc;
        {
            GpProf pf("eig_tables", stream);
            launch_eig_tables_chunked(sg, Xd, yd, tabc, st, stream);
            gp_note_launches(1);
        }
        {
            GpProf pf("colexp", stream);
            launch_colexp(sg, tabc, colexp, ebx, stream, bblk, b);
            gp_note_launches(b != nullptr ? 3 : 2);
        }
        {
            GpProf pf("syrk_tc", stream);
            cudaError_t e = launch_syrk_tc2(sg, tabc, spl, Gpart2, colexp, ebx, st, stream);
            if (e != cudaSuccess) return cuda_err(e, "syrk_tc2 launch");
            gp_note_launches(1);
        }
        {
            GpProf pf("assemble", stream);
            launch_assemble_pair(Gpart2, nullptr, colexp, spl, sg.Mpad, s.M, d, A, b, stream, ex);
            gp_note_launches(1);
            if (ex != nullptr && ex->L != nullptr && l_written) *l_written = true;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "Gram step");
    return GP_OK;
}

int tile_of(int prec) { return prec == GP_PREC_FP64 ? SYRK64_TM : SYRKTC_TM; }

int check_prec(int prec) {
    if (prec != GP_PREC_FP64 && prec != GP_PREC_MIXED)
        return set_err(GP_EINVAL, 4);
    return GP_OK;
}

void free_model(gp_model* h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    void* ps[] = {h->block};
    for (void* p : ps)
        if (p) cudaFree(p);
    cudaSetDevice(cur);
    delete h;
}

int model_alloc(gp_model* h, size_t bytes, void** p, cudaStream_t s) {
    cudaError_t e = dev_alloc(p, bytes, s);
    if (e == cudaErrorMemoryAllocation) return set_err(GP_ENOMEM, (int64_t)bytes);
    if (e != cudaSuccess) return cuda_err(e, "model allocation");
    return GP_OK;
}

gp_model* new_model(int dev, int prec, int64_t N, int p, int n, const double* eps, const double* alpha,
                    double sigma2) {
    gp_model* h = new gp_model();
    memset(h, 0, sizeof(*h));
    h->device = dev;
    h->prec = prec;
    for (int j = 0; j < p; ++j) {
        h->eps[j] = eps[j];
        h->alpha[j] = alpha[j];
    }
    h->sigma2 = sigma2;
    gp_fill_shape_ard(&h->shape, N, p, n, eps, alpha, tile_of(prec));
    return h;
}

gp_model* new_model(int dev, int prec, int64_t N, int p, int n, double eps, double alpha, double sigma2) {
    double e[GP_PMAX], a[GP_PMAX];
    for (int j = 0; j < GP_PMAX; ++j) {
        e[j] = eps;
        a[j] = alpha;
    }
    return new_model(dev, prec, N, p, n, e, a, sigma2);
}

// The model's own device buffers (kept until gp_free).
// The model's device buffers, carved from one allocation (kept until gp_free).
int fit_alloc(gp_model* h, cudaStream_t stream) {
    const size_t M = (size_t)h->shape.M;
    const bool tc = h->prec != GP_PREC_FP64;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // W = L^{-1} in float64 only for the float64 fit (the mixed one keeps
    // its float32 W packed for the predict kernel)
    const size_t sizes[7] = {sizeof(double) * M * M, tc ? 0 : sizeof(double) * M * M, sizeof(double) * M,
                             sizeof(double) * M,     sizeof(double) * M,
                             tc ? predtc_wpack_bytes((int)M) : 0,
                             tc ? sizeof(int) * predtc_cinfo_ints(h->shape) : 0};
    size_t total = 0;
    for (size_t b : sizes) total += al(b);
    int rc;
    if ((rc = model_alloc(h, total, &h->block, stream))) return rc;
    char* p = (char*)h->block;
    void** dst[7] = {(void**)&h->L, (void**)&h->W, (void**)&h->c, (void**)&h->b,
                     (void**)&h->d, (void**)&h->Wpack, (void**)&h->cinfo};
    for (int i = 0; i < 7; ++i) {
        *dst[i] = sizes[i] ? (void*)p : nullptr;
        p += al(sizes[i]);
    }
    return GP_OK;
}

// ---------------------------------------------------------------- pinned staging pool

namespace {
std::mutex g_pin_mu;
std::multimap<size_t, void*> g_pin_free;  // capacity -> block
}  // namespace

PinnedBlock pinned_get(size_t bytes) {
    size_t cap = 4096;
    while (cap < bytes) cap *= 2;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        auto it = g_pin_free.lower_bound(cap);
        if (it != g_pin_free.end() && it->first <= 4 * cap) {
            PinnedBlock b{it->second, it->first};
            g_pin_free.erase(it);
            return b;
        }
    }
    PinnedBlock b;
    if (cudaHostAlloc(&b.p, cap, cudaHostAllocPortable) == cudaSuccess) {
        b.cap = cap;
    } else {
        cudaGetLastError();
        b.p = nullptr;
    }
    return b;
}

void pinned_put(PinnedBlock b) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.emplace(b.cap, b.p);
}

// Copy the shape-only inputs (log eigenvalues of every dimension, loglam[j n +
// k], and the predict chunk table into the model) to the device, from pinned
// staging memory.
int fit_stage(gp_model* h, FitStage& stage, double* loglam_d, cudaStream_t stream) {
    const GpShape& s = h->shape;
    const size_t nci = h->prec != GP_PREC_FP64 ? predtc_cinfo_ints(s) : 0;
    const size_t lbytes = sizeof(double) * (size_t)s.p * s.n;
    stage.buf = pinned_get(lbytes + sizeof(int) * nci);
    if (!stage.buf.p) return set_err(GP_ENOMEM, (int64_t)(lbytes + sizeof(int) * nci));
    double* ll = (double*)stage.buf.p;
    for (int j = 0; j < s.p; ++j) log_eigenvalues(s.n, h->eps[j], h->alpha[j], ll + (size_t)j * s.n);
    cudaError_t e = cudaMemcpyAsync(loglam_d, ll, lbytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && nci > 0) {
        int* ci = (int*)((char*)stage.buf.p + lbytes);
        predtc_build_cinfo(s, ci);
        e = cudaMemcpyAsync(h->cinfo, ci, sizeof(int) * nci, cudaMemcpyHostToDevice, stream);
    }
    return e == cudaSuccess ? GP_OK : cuda_err(e, "shape-input copies");
}

int fit_factor(gp_model* h, const double* A, double* work, unsigned char* fwork, GpStatus* st,
               cudaStream_t stream, bool l_ready = false, int max_ctas = 0);

__global__ void add_diag_kernel(double* __restrict__ A, const double* __restrict__ d, int M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) A[(int64_t)i * M + i] += d[i];
}

// The exchange layout of a row-sharded Gram: the lower triangle of G row by
// row (entry (i, j), j <= i, at i (i + 1) / 2 + j), then b. One thread per
// element of the packed vector.
__global__ void pack_lower_kernel(const double* __restrict__ G, const double* __restrict__ b, int M,
                                  double* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nl = (int64_t)M * (M + 1) / 2;
    if (q >= nl + M) return;
    if (q >= nl) {
        out[q] = b[q - nl];
        return;
    }
    // row i of the lower triangle holding q: i (i + 1) / 2 <= q
    int64_t i = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    while (i * (i + 1) / 2 > q) --i;
    const int64_t j = q - i * (i + 1) / 2;
    out[q] = G[i * M + j];
}

// The inverse: the full symmetric A (M x M) and b from the packed vector.
__global__ void unpack_lower_kernel(const double* __restrict__ in, int M, double* __restrict__ A,
                                    double* __restrict__ b) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y;
    if (col >= M) return;
    const int64_t r = row >= col ? row : col, c = row >= col ? col : row;
    A[(int64_t)row * M + col] = in[r * (r + 1) / 2 + c];
    if (row == 0) b[col] = in[(int64_t)M * (M + 1) / 2 + col];
}

// Every device step of one fit, enqueued on `stream` with no host
// synchronisation (so that it can be captured into a graph). Inputs are
// device pointers; scratch comes from `sc` (stream-ordered); errors found on
// the device land in *st.
// Test hook: the next k mixed-precision fits report a non-positive pivot on
// their first attempt (exercises the float64 escalation).
std::atomic<int> g_force_escalate{0};

bool mixed_escalates(const gp_model* h, int code) {
    return h->prec == GP_PREC_MIXED && code == GP_ENOTPD && !(h->flags & GP_MODEL_GRAM_FP64);
}

__global__ void force_notpd_kernel(GpStatus* st) { gp_set_status(st, GP_ENOTPD, 0); }

int fit_compute(gp_model* h, const double* Xd, const double* yd, const double* loglam_d, GpStatus* st,
                int gram_ctas, Scratch& sc, cudaStream_t stream, int gram_prec, int factor_ctas) {
    const GpShape& s = h->shape;
    const int M = s.M;
    const int prec = h->prec;
    int rc;
    double *A, *work;
    if ((rc = sc.get(&A, (size_t)M * M))) return rc;
    if ((rc = sc.get(&work, solve_refine_work_elems(M)))) return rc;
    const bool fp32_inverse = (prec != GP_PREC_FP64);
    unsigned char* fwork;
    if ((rc = sc.get(&fwork, factor_work_bytes(M, fp32_inverse)))) return rc;
    const int gp_ = gram_prec < 0 ? prec : gram_prec;
    if (gp_ == GP_PREC_FP64 && prec != GP_PREC_FP64) h->flags |= GP_MODEL_GRAM_FP64;
    // the noise diagonal d (Eq. 16, 20) and the Cholesky's copy of A come out
    // of the assembly
    const AssembleExtra ex{&s, loglam_d, h->sigma2, h->d, h->L};
    bool l_written = false;
    if ((rc = gram_device(s, gp_, h->device, Xd, yd, nullptr, A, h->b, st, stream, gram_ctas, &ex, &l_written)))
        return rc;
    if (prec == GP_PREC_MIXED && gp_ == GP_PREC_MIXED) {
        int k = g_force_escalate.load();
        while (k > 0 && !g_force_escalate.compare_exchange_weak(k, k - 1)) {
        }
        if (k > 0) force_notpd_kernel<<<1, 1, 0, stream>>>(st);
    }
    return fit_factor(h, A, work, fwork, st, stream, l_written, factor_ctas);
}

// The factorisation steps of a fit from the assembled A (device, M x M, kept
// for the refinement residual): L, W = L^{-1}, c, and the predict operand.
// l_ready: h->L already holds A's lower triangle.
int fit_factor(gp_model* h, const double* A, double* work, unsigned char* fwork, GpStatus* st,
               cudaStream_t stream, bool l_ready, int max_ctas) {
    const int M = h->shape.M;
    const int prec = h->prec;
    const bool fp32_inverse = (prec != GP_PREC_FP64);
    if (!l_ready) cudaMemcpyAsync(h->L, A, sizeof(double) * M * M, cudaMemcpyDeviceToDevice, stream);
    cudaError_t e;
    {
        GpProf pf("cholesky", stream);
        // a mixed fit forms the trailing updates in float32, unless its Gram
        // had to be redone in float64 (then the factorisation is float64 too)
        const bool f32 = prec != GP_PREC_FP64 && !(h->flags & GP_MODEL_GRAM_FP64);
        e = launch_cholesky(h->L, M, st, fwork, stream, f32, max_ctas);
    }
    if (e == cudaSuccess) {
        GpProf pf("tri_inverse", stream);
        e = launch_tri_inverse(h->L, h->W, M, fp32_inverse, st, fwork, stream, max_ctas);
    }
    if (e == cudaSuccess) {
        GpProf pf("solve_refine", stream);
        // a mixed fit's solve also packs the predict operand (W and c)
        e = launch_solve_refine(A, h->W, fwork, fp32_inverse, h->b, h->c, work, M, fp32_inverse ? 3 : 2, st,
                                stream, prec != GP_PREC_FP64 ? h->Wpack : nullptr, max_ctas);
    }
    return e == cudaSuccess ? GP_OK : cuda_err(e, "factorisation or solve launch");
}

// Every device step of one predict (tables of X*, then mean and variance),
// enqueued on `stream` without host synchronisation. Device pointers only.
int predict_compute(const gp_model* h, const double* Xd, int64_t Ns, double* md, double* vd, GpStatus* st,
                    Scratch& sc, cudaStream_t stream) {
    GpShape s = h->shape;
    s.N = Ns;
    s.Npad = gp_round_up(Ns, 128);
    int rc;
    cudaError_t e;
    if (h->prec == GP_PREC_FP64) {
        double *tab, *part;
        if ((rc = sc.get(&tab, (size_t)s.p * s.n * s.Npad))) return rc;
        if ((rc = sc.get(&part, predict64_part_elems(s.Npad, s.M)))) return rc;
        {
            GpProf pf("eig_tables", stream);
            launch_eig_tables_f64(s, Xd, nullptr, tab, st, stream);
        }
        GpProf pf("predict64", stream);
        e = launch_predict64(s, tab, h->W, h->c, h->sigma2, part, md, vd, stream);
        gp_note_launches(3);
    } else {
        float* tab;
        double* vpart = nullptr;  // partial variances of the super-tiles
        if ((rc = sc.get(&tab, (size_t)s.p * s.n * s.Npad))) return rc;
        const size_t nv = vd ? predtc_vpart_elems(s.Npad, s.M) : 0;
        if (nv && (rc = sc.get(&vpart, nv))) return rc;
        {
            GpProf pf("eig_tables", stream);
            launch_eig_tables_f32(s, Xd, nullptr, tab, st, stream);
        }
        GpProf pf("predict_tc", stream);
        e = launch_predict_tc(s, tab, h->Wpack, h->cinfo, h->sigma2, md, vd, st, stream, nullptr, vpart);
        gp_note_launches(nv ? 3 : 2);
    }
    return e == cudaSuccess ? GP_OK : cuda_err(e, "predict launch");
}

// ---------------------------------------------------------------- batched predicts

int pred_batch_build(const std::vector<PredEntry>& es, Scratch& sc, PredBatch& pb) {
    pb = PredBatch();
    std::vector<int> order;
    for (int i = 0; i < (int)es.size(); ++i)
        if (es[i].Ns > 0) order.push_back(i);
    // by p (one launch each), heavier models first within a launch
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const GpShape &sa = es[a].m->shape, &sb = es[b].m->shape;
        if (sa.p != sb.p) return sa.p < sb.p;
        return sa.M > sb.M;
    });
    for (int idx : order) {
        const PredEntry& e = es[idx];
        const GpShape& s = e.m->shape;
        PredReq r{};
        r.Ns = e.Ns;
        r.Npad = gp_round_up(e.Ns, 128);
        r.p = s.p;
        r.n = s.n;
        r.M = s.M;
        r.Mpad = (int)gp_round_up(s.M, PREDTC_KB);
        r.maxrows = predtc_window_rows(s);
        r.Xs = e.Xd;
        int rc;
        if ((rc = sc.get(&r.tab, (size_t)s.p * s.n * r.Npad))) return rc;
        r.Wpack = (const uint8_t*)e.m->Wpack;
        r.cf = reinterpret_cast<const float*>((const uint8_t*)e.m->Wpack + 4 * (size_t)r.Mpad * r.Mpad);
        r.cinfo = e.m->cinfo;
        r.sigma2 = e.m->sigma2;
        r.mean = e.md;
        r.var = e.vd;
        r.st = e.st;
        const size_t nv = e.vd ? predtc_vpart_elems(r.Npad, s.M) : 0;
        if (nv && (rc = sc.get(&r.vpart, nv))) return rc;
        if (nv) pb.reduce = true;
        pb.max_npad = std::max(pb.max_npad, r.Npad);
        r.consts = reinterpret_cast<const float*>((uintptr_t)pb.consts.size());  // offset until pack()
        for (int j = 0; j < s.p; ++j) {
            pb.consts.push_back(s.abf[j]);
            pb.consts.push_back(s.sbf[j]);
            pb.consts.push_back(s.d2f[j]);
        }
        const int ridx = (int)pb.reqs.size();
        pb.boff.push_back(pb.nblocks);
        pb.nblocks += (int)((r.Npad + 255) / 256) * s.p;
        pb.max_n = std::max(pb.max_n, s.n);
        if (pb.groups.empty() || pb.groups.back().p != s.p)
            pb.groups.push_back(PredBatch::Group{s.p, (int)pb.items.size(), 0, 0});
        PredBatch::Group& g = pb.groups.back();
        // (tile, super-tile) items, or only the last super-tiles without a
        // variance; each super-tile's cost grows with its W rows' chunks
        const int ns = predtc_nsuper(s.M);
        const int nblocks = (s.M + PREDTC_KB - 1) / PREDTC_KB;
        for (int sp = (e.vd ? 0 : ns - 1); sp < ns; ++sp) {
            const int b0 = sp * PREDTC_SUPER, nblk = std::min(PREDTC_SUPER, nblocks - b0);
            const int mend = std::min(s.M, (b0 + nblk) * PREDTC_KB);
            const int64_t cost = (int64_t)((mend + PREDTC_BK - 1) / PREDTC_BK) * nblk;
            for (int64_t t = 0; t < r.Npad / 128; ++t) {
                pb.items.push_back(make_int2(ridx, (int)(t * ns + sp)));
                pb.cost.push_back(cost);
            }
        }
        g.count = (int)pb.items.size() - g.first;
        g.maxrows = std::max(g.maxrows, r.maxrows);
        pb.reqs.push_back(r);
    }
    pb.boff.push_back(pb.nblocks);
    // costlier items first within each launch (round-robin over the CTAs)
    for (const PredBatch::Group& g : pb.groups) {
        std::vector<int> ord(g.count);
        for (int i = 0; i < g.count; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return pb.cost[g.first + a] > pb.cost[g.first + b]; });
        std::vector<int2> tmp(g.count);
        for (int i = 0; i < g.count; ++i) tmp[i] = pb.items[g.first + ord[i]];
        std::copy(tmp.begin(), tmp.end(), pb.items.begin() + g.first);
    }
    for (const PredBatch::Group& g : pb.groups)
        if (predtc_batch_smem_bytes(g.maxrows, g.p) > (227 - 5) * 1024) return set_err(GP_EINVAL, 7);
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    pb.off_items = al(sizeof(PredReq) * pb.reqs.size());
    pb.off_boff = pb.off_items + al(sizeof(int2) * pb.items.size());
    pb.off_consts = pb.off_boff + al(sizeof(int) * pb.boff.size());
    pb.total = pb.off_consts + al(sizeof(float) * pb.consts.size());
    return GP_OK;
}

void pred_batch_pack(PredBatch& pb, void* host, const uint8_t* dev) {
    uint8_t* h = (uint8_t*)host;
    for (PredReq& r : pb.reqs)
        r.consts = reinterpret_cast<const float*>(dev + pb.off_consts) + (uintptr_t)r.consts;
    memcpy(h, pb.reqs.data(), sizeof(PredReq) * pb.reqs.size());
    memcpy(h + pb.off_items, pb.items.data(), sizeof(int2) * pb.items.size());
    memcpy(h + pb.off_boff, pb.boff.data(), sizeof(int) * pb.boff.size());
    memcpy(h + pb.off_consts, pb.consts.data(), sizeof(float) * pb.consts.size());
}

int pred_batch_enqueue(const PredBatch& pb, const uint8_t* dev, cudaStream_t stream) {
    if (pb.reqs.empty()) return GP_OK;
    const PredReq* dreqs = reinterpret_cast<const PredReq*>(dev);
    const int2* ditems = reinterpret_cast<const int2*>(dev + pb.off_items);
    {
        GpProf pf("eig_tables_batch", stream);
        launch_eig_tables_batch(dreqs, reinterpret_cast<const int*>(dev + pb.off_boff), (int)pb.reqs.size(),
                                pb.nblocks, pb.max_n, stream);
    }
    int nl = 1;
    for (const PredBatch::Group& g : pb.groups) {
        GpProf pf("predict_tc_batch", stream);
        cudaError_t e = launch_predict_tc_batch(dreqs, ditems + g.first, g.count, g.p, g.maxrows, stream);
        if (e != cudaSuccess) return cuda_err(e, "batched predict launch");
        ++nl;
    }
    if (pb.reduce) {
        launch_predict_reduce_batch(dreqs, (int)pb.reqs.size(), pb.max_npad, stream);
        ++nl;
    }
    gp_note_launches(nl);
    return GP_OK;
}

// ---------------------------------------------------------------- batches

// Streams that run the problems of one batch side by side (created per call).
struct StreamSet {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ev;
    explicit StreamSet(int k) {
        st.resize(k);
        ev.resize(k + 1);
        for (int i = 0; i < k; ++i) cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
        for (int i = 0; i <= k; ++i) cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    }
    ~StreamSet() {
        for (cudaStream_t s : st) cudaStreamDestroy(s);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    // every stream waits for the work already on `origin`
    void fork(cudaStream_t origin) {
        cudaEventRecord(ev.back(), origin);
        for (cudaStream_t s : st) cudaStreamWaitEvent(s, ev.back(), 0);
    }
    // `origin` waits for every stream
    void join(cudaStream_t origin) {
        for (size_t i = 0; i < st.size(); ++i) {
            cudaEventRecord(ev[i], st[i]);
            cudaStreamWaitEvent(origin, ev[i], 0);
        }
    }
};

// Gram CTA budget of problem i for the budget factor k: k waves of the GPU
// shared out in proportion to each problem's contraction work. The mixed
// batch contracts all its problems in one launch, so the budgets add up to
// that launch's grid.
std::vector<int> gram_budgets(const std::vector<gp_model*>& hs, int k, int sms) {
    std::vector<double> w(hs.size());
    double tot = 0.0;
    for (size_t i = 0; i < hs.size(); ++i) {
        const GpShape& s = hs[i]->shape;
        const int T = s.Mpad / tile_of(hs[i]->prec);
        w[i] = (double)s.Npad * (double)(T * (T + 1) / 2);
        tot += w[i];
    }
    std::vector<int> out(hs.size());
    for (size_t i = 0; i < hs.size(); ++i) {
        const double c = (double)k * sms * (tot > 0 ? w[i] / tot : 1.0);
        out[i] = c < 1.0 ? 1 : (int)(c + 0.5);
    }
    return out;
}

// ---------------------------------------------------------------- batch plans
//
// A batch's launch plan: the streams its per-problem steps are spread over
// and (mixed precision) the Gram budget factor k; the run is one captured
// CUDA graph. (Enqueued directly instead, a batch is as fast only on a
// process's first call: later calls wait on the scratch pool's
// stream-ordered frees across the streams, 1.2-1.9 times slower measured.)
// The autotuner times candidates on the batch itself, on the host clock from
// call to return, after one untimed run that warms the scratch pool, the
// first time a batch of that kind is seen (the same multiset of p, n, N
// rounded down to a power of two, precision, on the same GPU model), keeps
// the fastest for the process and, when the environment variable
// GPFAGP_TUNE_CACHE names a file, appends it there and reads it back in
// later processes (one line per plan: key, streams, k, ms, graph).

struct BatchPlan {
    int streams = 8;
    int k = 2;
    float ms = 0.f;
    int graph = 1;
    int fcap = 0;         // factorisation grids capped at max(4, SMs / streams) CTAs (1) or not (0)
    bool cached = false;  // taken from the cache (this process's or the file's)
};
int plan_factor_ctas(const BatchPlan& p, int sms) {
    if (!p.fcap) return 0;
    const int c = sms / (p.streams > 0 ? p.streams : 1);
    return c < 4 ? 4 : c;
}

std::mutex g_tune_mu;
std::map<std::string, BatchPlan> g_tune;
bool g_tune_loaded = false;
thread_local int g_batch_graph = 0;
thread_local BatchPlan g_last_plan;

const char* tune_file() {
    const char* e = getenv("GPFAGP_TUNE_CACHE");
    return (e != nullptr && e[0] != '\0') ? e : nullptr;
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = tune_file();
    if (path == nullptr) return;
    FILE* f = fopen(path, "r");
    if (f == nullptr) return;
    char line[512];
    while (fgets(line, sizeof(line), f) != nullptr) {
        char key[384];
        BatchPlan p;
        const int nf = sscanf(line, "%383s %d %d %f %d %d", key, &p.streams, &p.k, &p.ms, &p.graph, &p.fcap);
        if (nf >= 4 && p.streams >= 1 && p.k >= 0) {
            if (nf < 5) p.graph = 1;
            if (nf < 6) p.fcap = 0;
            g_tune[key] = p;  // later lines win
        }
    }
    fclose(f);
}

void tune_store_locked(const std::string& key, const BatchPlan& p) {
    g_tune[key] = p;
    const char* path = tune_file();
    if (path == nullptr) return;
    FILE* f = fopen(path, "a");
    if (f == nullptr) return;
    fprintf(f, "%s %d %d %.4f %d %d\n", key.c_str(), p.streams, p.k, p.ms, p.graph, p.fcap);
    fclose(f);
}

// device model + library version + FNV-1a hash of the sorted problem kinds
std::string batch_key(const std::vector<gp_model*>& hs, int dev) {
    std::vector<std::string> parts;
    for (gp_model* h : hs) {
        int lg = 0;
        while ((int64_t)1 << (lg + 1) <= h->shape.N) ++lg;
        char buf[64];
        snprintf(buf, sizeof(buf), "%d.%d.%d.%d", h->shape.p, h->shape.n, lg, h->prec);
        parts.push_back(buf);
    }
    std::sort(parts.begin(), parts.end());
    uint64_t hsh = 1469598103934665603ull;
    for (auto& x : parts)
        for (char ch : x + ";") {
            hsh ^= (unsigned char)ch;
            hsh *= 1099511628211ull;
        }
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        name = prop.name;
        for (char& ch : name)
            if (ch == ' ' || ch == '\t') ch = '_';
        name += "_" + std::to_string(prop.multiProcessorCount);
    }
    char buf[128];
    snprintf(buf, sizeof(buf), "batch/%s/%s/n%zu/%016llx", name.c_str(), gp_version(), hs.size(),
             (unsigned long long)hsh);
    std::string key = buf;
    for (char& ch : key)
        if (ch == ' ') ch = '_';
    return key;
}

// Everything one enqueue of the batch needs.
struct BatchCtx {
    std::vector<gp_model*>* hs;
    std::vector<const double*>* Xd;
    std::vector<const double*>* yd;
    std::vector<double*>* loglam;
    GpStatus* sts;
    int dev, sms;
    cudaStream_t origin;
    StreamSet* ss;                     // the largest stream set; a plan uses its first `streams`
    std::vector<PinnedBlock> pinned;   // host images read by copies not yet run
};

void fork_n(StreamSet& ss, cudaStream_t origin, int n) {
    cudaEventRecord(ss.ev.back(), origin);
    for (int i = 0; i < n; ++i) cudaStreamWaitEvent(ss.st[i], ss.ev.back(), 0);
}
void join_n(StreamSet& ss, cudaStream_t origin, int n) {
    for (int i = 0; i < n; ++i) {
        cudaEventRecord(ss.ev[i], ss.st[i]);
        cudaStreamWaitEvent(origin, ss.ev[i], 0);
    }
}

void maybe_force_notpd(GpStatus* st, cudaStream_t stream) {
    int k = g_force_escalate.load();
    while (k > 0 && !g_force_escalate.compare_exchange_weak(k, k - 1)) {
    }
    if (k > 0) force_notpd_kernel<<<1, 1, 0, stream>>>(st);
}

// Enqueue every problem's fit under a plan, behind and ahead of `origin`.
// Float64: each problem's own steps on stream i mod S. Mixed (stage-major):
// every problem's tables and column exponents on its stream, then the Grams
// of all problems in one launch per p on `origin` (a device table of the
// problems; launch_syrk_tc_batch), then every problem's assembly and
// factorisation on its stream.
int enqueue_batch(BatchCtx& c, const BatchPlan& plan) {
    std::vector<gp_model*>& hs = *c.hs;
    const int count = (int)hs.size();
    const int S = std::min(plan.streams, (int)c.ss->st.size());
    StreamSet& ss = *c.ss;
    fork_n(ss, c.origin, S);
    int rc = GP_OK;
    if (hs[0]->prec == GP_PREC_FP64) {
        std::vector<Scratch*> scs;
        for (int i = 0; i < count && rc == GP_OK; ++i) {
            cudaStream_t s = ss.st[i % S];
            Scratch* sc = new Scratch(s);
            scs.push_back(sc);
            rc = fit_compute(hs[i], (*c.Xd)[i], (*c.yd)[i], (*c.loglam)[i], &c.sts[i], 0, *sc, s, -1,
                             plan_factor_ctas(plan, c.sms));
        }
        for (Scratch* sc : scs) delete sc;  // scratch frees are stream-ordered
        join_n(ss, c.origin, S);
        return rc;
    }
    const std::vector<int> bud = gram_budgets(hs, plan.k, c.sms);
    std::vector<Scratch*> scs(count, nullptr);
    std::vector<MixedGram> gs(count);
    std::vector<double*> A(count), work(count);
    std::vector<unsigned char*> fw(count);
    for (int i = 0; i < count && rc == GP_OK; ++i) {
        cudaStream_t s = ss.st[i % S];
        scs[i] = new Scratch(s);
        const GpShape& sh = hs[i]->shape;
        if ((rc = scs[i]->get(&A[i], (size_t)sh.M * sh.M))) break;
        if ((rc = scs[i]->get(&work[i], solve_refine_work_elems(sh.M)))) break;
        if ((rc = scs[i]->get(&fw[i], factor_work_bytes(sh.M, true)))) break;
        rc = mixed_gram_prepare(sh, c.dev, (*c.Xd)[i], (*c.yd)[i], &c.sts[i], *scs[i], s, bud[i], gs[i], true);
    }
    join_n(ss, c.origin, S);
    if (rc == GP_OK) {
        // the problem table, grouped by p (one launch each)
        std::map<int, std::vector<int>> byp;
        for (int i = 0; i < count; ++i) byp[hs[i]->shape.p].push_back(i);
        std::vector<SyrkBatchProb> probs;
        struct Launch {
            int p, first, n, maxrows;
            int64_t items;
        };
        std::vector<Launch> launches;
        for (auto& kv : byp) {
            Launch L{kv.first, (int)probs.size(), 0, 0, 0};
            for (int i : kv.second) {
                SyrkBatchProb b{};
                b.s = gs[i].sg;
                b.tabc = gs[i].tabc;
                b.ebx = gs[i].ebx;
                b.colexp = gs[i].colexp;
                b.sp = gs[i].spl;
                b.T = gs[i].sg.Mpad / SYRKTC_TM;
                b.Gpart = gs[i].Gpart;
                b.bpart = gs[i].bpart;
                b.st = &c.sts[i];
                b.item0 = L.items;
                L.items += syrktc_items(gs[i].sg, gs[i].spl);
                L.maxrows = std::max(L.maxrows, gp_max_window_rows(gs[i].sg, SYRKTC_TM));
                probs.push_back(b);
                ++L.n;
            }
            launches.push_back(L);
        }
        const size_t bytes = sizeof(SyrkBatchProb) * probs.size();
        PinnedBlock pb = pinned_get(bytes);
        Scratch tsc(c.origin);
        SyrkBatchProb* dprobs = nullptr;
        if (pb.p == nullptr) rc = set_err(GP_ENOMEM, (int64_t)bytes);
        if (rc == GP_OK) rc = tsc.get(&dprobs, probs.size());
        if (rc == GP_OK) {
            c.pinned.push_back(pb);
            memcpy(pb.p, probs.data(), bytes);
            cudaMemcpyAsync(dprobs, pb.p, bytes, cudaMemcpyHostToDevice, c.origin);
            for (const Launch& L : launches) {
                GpProf pf("syrk_tc", c.origin);
                cudaError_t e = launch_syrk_tc_batch(dprobs + L.first, L.n, L.items, L.p, L.maxrows, c.origin);
                if (e != cudaSuccess) {
                    rc = cuda_err(e, "batched Gram launch");
                    break;
                }
                gp_note_launches(1);
            }
        } else if (pb.p != nullptr) {
            pinned_put(pb);
        }
    }
    fork_n(ss, c.origin, S);
    for (int i = 0; i < count; ++i) {
        cudaStream_t s = ss.st[i % S];
        if (rc == GP_OK) {
            gp_model* h = hs[i];
            const AssembleExtra ex{&h->shape, (*c.loglam)[i], h->sigma2, h->d, h->L};
            bool lw = false;
            mixed_gram_assemble(gs[i], h->shape.M, nullptr, A[i], h->b, s, &ex, &lw);
            maybe_force_notpd(&c.sts[i], s);
            rc = fit_factor(h, A[i], work[i], fw[i], &c.sts[i], s, lw, plan_factor_ctas(plan, c.sms));
        }
        delete scs[i];  // stream-ordered frees behind this problem's steps
    }
    join_n(ss, c.origin, S);
    return rc;
}

// One run of the batch under `plan`: captured into one CUDA graph and
// launched if plan.graph (if capture or instantiation is refused, enqueued
// directly), else enqueued directly; then synchronised. *ms = the host time
// from the call to the synchronisation, *graph = whether a graph ran.
int run_batch(BatchCtx& c, const BatchPlan& plan, float* ms, int* graph) {
    const auto h0 = std::chrono::steady_clock::now();
    cudaMemsetAsync(c.sts, 0, sizeof(GpStatus) * c.hs->size(), c.origin);
    const int prof = gp_prof_suspend();
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ran = false;
    int rc = GP_OK;
    if (plan.graph && cudaStreamBeginCapture(c.origin, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const int erc = enqueue_batch(c, plan);
        const cudaError_t ce = cudaStreamEndCapture(c.origin, &g);
        if (erc == GP_OK && ce == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess &&
            cudaGraphLaunch(exec, c.origin) == cudaSuccess)
            ran = true;
        if (!ran) {
            (void)cudaGetLastError();
            set_err(GP_OK);
        }
    } else {
        (void)cudaGetLastError();
    }
    if (!ran) rc = enqueue_batch(c, plan);
    cudaError_t e = cudaStreamSynchronize(c.origin);
    gp_prof_resume(prof);
    for (PinnedBlock& b : c.pinned) pinned_put(b);
    c.pinned.clear();
    const float t = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - h0).count();
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    if (ms) *ms = t;
    if (graph) *graph = ran ? 1 : 0;
    if (rc != GP_OK) return rc;
    return e == cudaSuccess ? GP_OK : cuda_err(e, "batch synchronise");
}

// The plan for this batch: from the cache, or timed over the candidates
// (streams 8, 16, 32 -- at most the problem count -- and, for mixed
// precision, k = 1, 2, 4); each candidate runs the whole batch once, after
// one untimed run.
int plan_batch(BatchCtx& c, BatchPlan* out) {
    const std::string key = batch_key(*c.hs, c.dev);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *out = it->second;
            out->cached = true;
            return GP_OK;
        }
    }
    {
        // warm the scratch pool, so that the first candidate is not charged for it
        BatchPlan w;
        w.streams = std::min(8, (int)c.hs->size());
        w.k = (*c.hs)[0]->prec != GP_PREC_FP64 ? 2 : 0;
        const int rc = run_batch(c, w, nullptr, nullptr);
        if (rc != GP_OK) return rc;
    }
    const int count = (int)c.hs->size();
    const bool mixed = (*c.hs)[0]->prec != GP_PREC_FP64;
    BatchPlan best;
    best.ms = 1e30f;
    bool any = false;
    for (int S : {8, 16, 32}) {
        if (S > count && S != 8) break;
        for (int k : {1, 2, 4}) {
            if (!mixed && k != 1) break;
            for (int fcap : {0, 1}) {
                BatchPlan cand;
                cand.streams = std::min(S, count);
                cand.k = mixed ? k : 0;
                cand.fcap = fcap;
                float ms = 0.f;
                const int rc = run_batch(c, cand, &ms, nullptr);
                if (rc != GP_OK) return rc;
                if (ms < best.ms) {
                    best = cand;
                    best.ms = ms;
                    any = true;
                }
            }
        }
    }
    if (!any) best = BatchPlan();
    best.cached = false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store_locked(key, best);
    *out = best;
    return GP_OK;
}

}  // namespace gpi

using namespace gpi;

int gp_fill_shape_ard(GpShape* s, int64_t N, int p, int n, const double* eps, const double* alpha, int tile) {
    memset(s, 0, sizeof(*s));
    s->N = N;
    s->Npad = gp_round_up(N > 0 ? N : 1, 128);
    s->p = p;
    s->n = n;
    int64_t M = 1;
    for (int j = 0; j < p; ++j) M *= n;
    s->M = (int)M;
    s->Mpad = (int)gp_round_up(M, tile);
    int64_t st = 1;
    for (int j = p - 1; j >= 0; --j) {
        s->stride[j] = (int)st;
        st *= n;
    }
    // Eq. 14 per dimension (delta^2 with the rho^2 reading)
    for (int j = 0; j < p && j < GP_PMAX; ++j) {
        const double e = eps[j], a = alpha[j];
        const double beta = pow(1.0 + (2.0 * e / a) * (2.0 * e / a), 0.25);
        s->ab[j] = a * beta;
        s->d2[j] = a * a * (beta * beta - 1.0) / 2.0;
        s->sb[j] = sqrt(beta);
        s->abf[j] = (float)s->ab[j];
        s->d2f[j] = (float)s->d2[j];
        s->sbf[j] = (float)s->sb[j];
    }
    return GP_OK;
}

int gp_fill_shape(GpShape* s, int64_t N, int p, int n, double eps, double alpha, int tile) {
    double e[GP_PMAX], a[GP_PMAX];
    for (int j = 0; j < GP_PMAX; ++j) {
        e[j] = eps;
        a[j] = alpha;
    }
    return gp_fill_shape_ard(s, N, p, n, e, a, tile);
}

extern "C" {

GPFAGP_API const char* gp_version(void) { return "gpfagp 0.3 sm_103a"; }

GPFAGP_API int gp_last_error(void) { return g_err; }
GPFAGP_API int64_t gp_last_error_detail(void) { return g_detail; }

GPFAGP_API const char* gp_last_error_where(void) { return g_err == GP_ECUDA ? g_where : ""; }

GPFAGP_API const char* gp_strerror(int status) {
    switch (status) {
        case GP_OK: return "ok";
        case GP_EINVAL: return "invalid argument";
        case GP_ENOMEM: return "device allocation failed";
        case GP_ENOTPD: return "matrix A is not positive definite";
        case GP_ECUDA: return "CUDA runtime error";
        case GP_ETIMEOUT: return "bounded device wait timed out";
        case GP_ENODEV: return "no sm_103 device";
        default: return "unknown status";
    }
}

GPFAGP_API void gp_debug_fail_alloc_after(int k) { g_fail_after.store(k > 0 ? k : 0); }

GPFAGP_API void gp_debug_force_escalation(int k) { g_force_escalate.store(k > 0 ? k : 0); }

GPFAGP_API void gp_debug_gram_kernel(int kind) { g_gram_kernel.store(kind >= 0 && kind <= 2 ? kind : 0); }

GPFAGP_API void gp_debug_barrier_timeout(double limit_s, int skip_cta) {
    factor_debug_barrier_timeout(limit_s, skip_cta);
}

GPFAGP_API int gp_debug_gram_splits(int T, int64_t Npad, int target_ctas, int64_t* out) {
    if (T < 1 || Npad < 1 || target_ctas < 1 || !out) return set_err(GP_EINVAL, 0);
    SyrkSplit sp;
    choose_splits_tc(T, Npad, target_ctas, &sp);
    const int64_t npc[3] = {T, T - 1, (int64_t)(T - 1) * (T - 2) / 2};
    int64_t ctas = 0;
    for (int c = 0; c < 3; ++c) {
        out[c] = sp.n[c];
        out[3 + c] = sp.rows[c];
        ctas += npc[c] * sp.n[c];
    }
    out[6] = ctas;
    return GP_OK;
}

GPFAGP_API int gp_debug_column_exponents(const double* X, int64_t N, int p, int n, double eps, double alpha,
                                         signed char* ebx, signed char* ebx4, int* colexp) {
    set_err(GP_OK);
    int rc, dev;
    if (!X || !ebx || !ebx4 || !colexp) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, 1.0))) return rc;
    if ((rc = check_device(&dev))) return rc;
    GpShape s;
    gp_fill_shape(&s, N, p, n, eps, alpha, SYRKTC_TM);
    cudaStream_t stream = 0;
    Scratch sc(stream);
    GpStatus* st;
    double* xd;
    float* tabc;
    int* ce;
    signed char* eb;
    if ((rc = sc.get(&st, 1))) return rc;
    if ((rc = sc.get(&xd, (size_t)N * p))) return rc;
    if ((rc = sc.get(&tabc, syrktc_table_floats(s)))) return rc;
    if ((rc = sc.get(&ce, (size_t)s.Mpad))) return rc;
    if ((rc = sc.get(&eb, syrktc_ebx_bytes(s)))) return rc;
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    cudaMemcpyAsync(xd, X, sizeof(double) * N * p, cudaMemcpyHostToDevice, stream);
    launch_eig_tables_chunked(s, xd, nullptr, tabc, st, stream);
    launch_colexp(s, tabc, ce, eb, stream);
    const int64_t nblk = (s.Npad + GP_TAB_BLOCK - 1) / GP_TAB_BLOCK, nblk4 = (s.Npad + GP_PAIR_BLOCK - 1) / GP_PAIR_BLOCK;
    std::vector<signed char> h1((size_t)nblk * s.Mpad), h4((size_t)nblk4 * s.Mpad);
    std::vector<int> hc(s.Mpad);
    cudaMemcpyAsync(h1.data(), eb, h1.size(), cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(h4.data(), syrktc_pair_exponents(s, eb), h4.size(), cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(hc.data(), ce, sizeof(int) * s.Mpad, cudaMemcpyDeviceToHost, stream);
    if ((rc = read_status(st, stream))) return rc;  // synchronises the stream
    for (int64_t b = 0; b < nblk; ++b)
        for (int m = 0; m < s.M; ++m) ebx[b * s.M + m] = h1[(size_t)b * s.Mpad + m];
    for (int64_t b = 0; b < nblk4; ++b)
        for (int m = 0; m < s.M; ++m) ebx4[b * s.M + m] = h4[(size_t)b * s.Mpad + m];
    for (int m = 0; m < s.M; ++m) colexp[m] = hc[m];
    return GP_OK;
}

GPFAGP_API int gp_model_flags(const gp_model* h) { return h ? h->flags : 0; }

GPFAGP_API int gp_gram_ex(const double* X, const double* y, int64_t N, int p, int n, double eps,
                          double alpha, int prec, double* G, double* b, void* cuda_stream,
                          int dev_ptrs) {
    set_err(GP_OK);
    int rc, dev;
    if (!X || !y || !G || !b) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, 1.0))) return rc;
    if ((rc = check_prec(prec))) return rc;
    if ((rc = check_device(&dev))) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    GpShape s;
    gp_fill_shape(&s, N, p, n, eps, alpha, tile_of(prec));
    Scratch sc(stream);
    const double *Xd = X, *yd = y;
    double *Gd = G, *bd = b;
    GpStatus* st;
    if ((rc = sc.get(&st, 1))) return rc;
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    if (!dev_ptrs) {
        double *xx, *yy;
        if ((rc = sc.get(&xx, (size_t)N * p))) return rc;
        if ((rc = sc.get(&yy, (size_t)N))) return rc;
        if ((rc = sc.get(&Gd, (size_t)s.M * s.M))) return rc;
        if ((rc = sc.get(&bd, (size_t)s.M))) return rc;
        cudaMemcpyAsync(xx, X, sizeof(double) * N * p, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(yy, y, sizeof(double) * N, cudaMemcpyHostToDevice, stream);
        Xd = xx;
        yd = yy;
    }
    if ((rc = gram_device(s, prec, dev, Xd, yd, nullptr, Gd, bd, st, stream))) return rc;
    if (!dev_ptrs) {
        cudaMemcpyAsync(G, Gd, sizeof(double) * s.M * s.M, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(b, bd, sizeof(double) * s.M, cudaMemcpyDeviceToHost, stream);
    }
    return read_status(st, stream);
}

GPFAGP_API int gp_gram_packed_ex(const double* X, const double* y, int64_t N, int p, int n, double eps,
                                 double alpha, int prec, double* packed, void* cuda_stream, int dev_ptrs) {
    set_err(GP_OK);
    int rc, dev;
    if (!X || !y || !packed) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, 1.0))) return rc;
    if ((rc = check_prec(prec))) return rc;
    if ((rc = check_device(&dev))) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    GpShape s;
    gp_fill_shape(&s, N, p, n, eps, alpha, tile_of(prec));
    const int M = s.M;
    const size_t np = (size_t)M * (M + 1) / 2 + M;
    Scratch sc(stream);
    const double *Xd = X, *yd = y;
    double *Gd, *bd, *pd = packed;
    GpStatus* st;
    if ((rc = sc.get(&st, 1))) return rc;
    if ((rc = sc.get(&Gd, (size_t)M * M))) return rc;
    if ((rc = sc.get(&bd, (size_t)M))) return rc;
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    if (!dev_ptrs) {
        double *xx, *yy;
        if ((rc = sc.get(&xx, (size_t)N * p))) return rc;
        if ((rc = sc.get(&yy, (size_t)N))) return rc;
        if ((rc = sc.get(&pd, np))) return rc;
        cudaMemcpyAsync(xx, X, sizeof(double) * N * p, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(yy, y, sizeof(double) * N, cudaMemcpyHostToDevice, stream);
        Xd = xx;
        yd = yy;
    }
    if ((rc = gram_device(s, prec, dev, Xd, yd, nullptr, Gd, bd, st, stream))) return rc;
    pack_lower_kernel<<<(unsigned)((np + 255) / 256), 256, 0, stream>>>(Gd, bd, M, pd);
    gp_note_launches(1);
    if (!dev_ptrs) cudaMemcpyAsync(packed, pd, sizeof(double) * np, cudaMemcpyDeviceToHost, stream);
    return read_status(st, stream);
}

GPFAGP_API int gp_gram_static(const double* X, const double* y, int64_t N, int p, int n, double eps,
                              double alpha, double* G, double* b, void* cuda_stream) {
    set_err(GP_OK);
    int rc, dev;
    if (!X || !y || !G || !b) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, 1.0))) return rc;
    if ((rc = check_device(&dev))) return rc;
    int64_t detail = 0;
    rc = gp_static_gram(X, y, N, p, n, eps, alpha, G, b, (cudaStream_t)cuda_stream, &detail);
    if (rc != GP_OK) return set_err(rc, detail);
    return GP_OK;
}

namespace {
// gp_fit_ex with eps_j, alpha_j per dimension (already validated)
int fit_ex_impl(const double* X, const double* y, int64_t N, int p, int n, const double* eps, const double* alpha,
                double sigma2, int prec, void* cuda_stream, int dev_ptrs, gp_model** out) {
    int rc, dev;
    if ((rc = check_prec(prec))) return rc;
    if ((rc = check_device(&dev))) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    gp_model* h = new_model(dev, prec, N, p, n, eps, alpha, sigma2);
    Scratch sc(stream);
    FitStage stage;
    auto fail = [&](int code) {
        int64_t det = g_detail;
        cudaStreamSynchronize(stream);
        free_model(h);
        set_err(code, det);
        return code;
    };
    if ((rc = fit_alloc(h, stream))) return fail(rc);
    GpStatus* st;
    double* loglam;
    if ((rc = sc.get(&st, 1))) return fail(rc);
    if ((rc = sc.get(&loglam, (size_t)p * n))) return fail(rc);
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    const double *Xd = X, *yd = y;
    if (!dev_ptrs) {
        double *xx, *yy;
        if ((rc = sc.get(&xx, (size_t)N * p))) return fail(rc);
        if ((rc = sc.get(&yy, (size_t)N))) return fail(rc);
        cudaMemcpyAsync(xx, X, sizeof(double) * N * p, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(yy, y, sizeof(double) * N, cudaMemcpyHostToDevice, stream);
        Xd = xx;
        yd = yy;
    }
    if ((rc = fit_stage(h, stage, loglam, stream))) return fail(rc);
    if ((rc = fit_compute(h, Xd, yd, loglam, st, 0, sc, stream))) return fail(rc);
    // the staged host vectors live until this read synchronises the stream
    rc = read_status(st, stream);
    if (mixed_escalates(h, rc)) {
        // the mixed Gram was not accurate enough for this A: redo it in float64
        set_err(GP_OK);
        cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
        Scratch sc2(stream);
        if ((rc = fit_compute(h, Xd, yd, loglam, st, 0, sc2, stream, GP_PREC_FP64))) return fail(rc);
        rc = read_status(st, stream);
    }
    if (rc) return fail(rc);
    *out = h;
    return GP_OK;
}
}  // namespace

GPFAGP_API int gp_fit_ex(const double* X, const double* y, int64_t N, int p, int n, double eps,
                         double alpha, double sigma2, int prec, void* cuda_stream, int dev_ptrs,
                         gp_model** out) {
    set_err(GP_OK);
    int rc;
    if (!out) return set_err(GP_EINVAL, 0);
    *out = nullptr;
    if (!X || !y) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, sigma2))) return rc;
    double e[GP_PMAX], a[GP_PMAX];
    for (int j = 0; j < GP_PMAX; ++j) {
        e[j] = eps;
        a[j] = alpha;
    }
    return fit_ex_impl(X, y, N, p, n, e, a, sigma2, prec, cuda_stream, dev_ptrs, out);
}

GPFAGP_API int gp_fit_ard_ex(const double* X, const double* y, int64_t N, int p, int n, const double* eps,
                             const double* alpha, double sigma2, int prec, void* cuda_stream, int dev_ptrs,
                             gp_model** out) {
    set_err(GP_OK);
    int rc;
    if (!out) return set_err(GP_EINVAL, 0);
    *out = nullptr;
    if (!X || !y || !eps || !alpha) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, 1.0, 1.0, sigma2))) return rc;
    for (int j = 0; j < p; ++j)
        if (!finite_pos(eps[j]) || !finite_pos(alpha[j])) return set_err(GP_EINVAL, 2);
    return fit_ex_impl(X, y, N, p, n, eps, alpha, sigma2, prec, cuda_stream, dev_ptrs, out);
}

namespace {
// The device steps of a predict on a fitted model into device or host
// outputs (host: staged through scratch and copied back on the stream).
int predict_enqueue(const gp_model* h, const double* Xs, int64_t Ns, double* mean, double* var, int dev_ptrs,
                    GpStatus* st, Scratch& sc, cudaStream_t stream) {
    if (Ns == 0) return GP_OK;
    const double* Xd = Xs;
    double *md = mean, *vd = var;
    int rc;
    if (!dev_ptrs) {
        double* xx;
        if ((rc = sc.get(&xx, (size_t)Ns * h->shape.p))) return rc;
        if ((rc = sc.get(&md, (size_t)Ns))) return rc;
        if (var && (rc = sc.get(&vd, (size_t)Ns))) return rc;
        cudaMemcpyAsync(xx, Xs, sizeof(double) * Ns * h->shape.p, cudaMemcpyHostToDevice, stream);
        Xd = xx;
    }
    if ((rc = predict_compute(h, Xd, Ns, md, vd, st, sc, stream))) return rc;
    if (!dev_ptrs) {
        cudaMemcpyAsync(mean, md, sizeof(double) * Ns, cudaMemcpyDeviceToHost, stream);
        if (var) cudaMemcpyAsync(var, vd, sizeof(double) * Ns, cudaMemcpyDeviceToHost, stream);
    }
    return GP_OK;
}
}  // namespace

GPFAGP_API int gp_fit_predict_ex(const double* X, const double* y, int64_t N, int p, int n, double eps,
                                 double alpha, double sigma2, int prec, const double* Xs, int64_t Ns,
                                 double* mean, double* var, void* cuda_stream, int dev_ptrs, gp_model** out) {
    set_err(GP_OK);
    int rc, dev;
    if (!out) return set_err(GP_EINVAL, 0);
    *out = nullptr;
    if (!X || !y || Ns < 0 || (Ns > 0 && (!Xs || !mean))) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, sigma2))) return rc;
    if ((rc = check_prec(prec))) return rc;
    if ((rc = check_device(&dev))) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    gp_model* h = new_model(dev, prec, N, p, n, eps, alpha, sigma2);
    Scratch sc(stream);
    FitStage stage;
    auto fail = [&](int code) {
        int64_t det = g_detail;
        cudaStreamSynchronize(stream);
        free_model(h);
        set_err(code, det);
        return code;
    };
    if ((rc = fit_alloc(h, stream))) return fail(rc);
    GpStatus* st;
    double* loglam;
    if ((rc = sc.get(&st, 1))) return fail(rc);
    if ((rc = sc.get(&loglam, (size_t)p * n))) return fail(rc);
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    const double *Xd = X, *yd = y;
    if (!dev_ptrs) {
        double *xx, *yy;
        if ((rc = sc.get(&xx, (size_t)N * p))) return fail(rc);
        if ((rc = sc.get(&yy, (size_t)N))) return fail(rc);
        cudaMemcpyAsync(xx, X, sizeof(double) * N * p, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(yy, y, sizeof(double) * N, cudaMemcpyHostToDevice, stream);
        Xd = xx;
        yd = yy;
    }
    if ((rc = fit_stage(h, stage, loglam, stream))) return fail(rc);
    if ((rc = fit_compute(h, Xd, yd, loglam, st, 0, sc, stream))) return fail(rc);
    // the predict reads the model the fit leaves; if the fit failed, what it
    // computes is discarded below
    if ((rc = predict_enqueue(h, Xs, Ns, mean, var, dev_ptrs, st, sc, stream))) return fail(rc);
    // the staged host vectors live until this read synchronises the stream
    rc = read_status(st, stream);
    if (mixed_escalates(h, rc)) {
        set_err(GP_OK);
        cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
        Scratch sc2(stream);
        if ((rc = fit_compute(h, Xd, yd, loglam, st, 0, sc2, stream, GP_PREC_FP64))) return fail(rc);
        if ((rc = predict_enqueue(h, Xs, Ns, mean, var, dev_ptrs, st, sc2, stream))) return fail(rc);
        rc = read_status(st, stream);
    }
    if (rc) return fail(rc);
    *out = h;
    return GP_OK;
}

namespace {
// A fit continued from a Gram: full G and b (packed == false) or the packed
// lower triangle and b of gp_gram_packed_ex (packed == true, in G).
int fit_from_gram(const double* G, const double* b, bool packed, int64_t N, int p, int n, double eps, double alpha,
                  double sigma2, int prec, void* cuda_stream, int dev_ptrs, gp_model** out) {
    set_err(GP_OK);
    int rc, dev;
    if (!out) return set_err(GP_EINVAL, 0);
    *out = nullptr;
    if (!G || (!packed && !b)) return set_err(GP_EINVAL, 0);
    if ((rc = check_hyper(N, p, n, eps, alpha, sigma2))) return rc;
    if ((rc = check_prec(prec))) return rc;
    if ((rc = check_device(&dev))) return rc;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    gp_model* h = new_model(dev, prec, N, p, n, eps, alpha, sigma2);
    const int M = h->shape.M;
    Scratch sc(stream);
    FitStage stage;
    auto fail = [&](int code) {
        int64_t det = g_detail;
        cudaStreamSynchronize(stream);
        free_model(h);
        set_err(code, det);
        return code;
    };
    if ((rc = fit_alloc(h, stream))) return fail(rc);
    GpStatus* st;
    double *loglam, *A, *work;
    unsigned char* fwork;
    if ((rc = sc.get(&st, 1))) return fail(rc);
    if ((rc = sc.get(&loglam, (size_t)p * n))) return fail(rc);
    if ((rc = sc.get(&A, (size_t)M * M))) return fail(rc);
    if ((rc = sc.get(&work, solve_refine_work_elems(M)))) return fail(rc);
    if ((rc = sc.get(&fwork, factor_work_bytes(M, prec != GP_PREC_FP64)))) return fail(rc);
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    const cudaMemcpyKind kind = dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (packed) {
        const size_t np = (size_t)M * (M + 1) / 2 + M;
        const double* pd = G;
        if (!dev_ptrs) {
            double* tmp;
            if ((rc = sc.get(&tmp, np))) return fail(rc);
            cudaMemcpyAsync(tmp, G, sizeof(double) * np, kind, stream);
            pd = tmp;
        }
        dim3 grid((unsigned)((M + 255) / 256), (unsigned)M);
        unpack_lower_kernel<<<grid, 256, 0, stream>>>(pd, M, A, h->b);
        gp_note_launches(1);
    } else {
        cudaMemcpyAsync(A, G, sizeof(double) * M * M, kind, stream);
        cudaMemcpyAsync(h->b, b, sizeof(double) * M, kind, stream);
    }
    if ((rc = fit_stage(h, stage, loglam, stream))) return fail(rc);
    launch_noise_diag(h->shape, loglam, sigma2, h->d, stream);
    add_diag_kernel<<<(M + 255) / 256, 256, 0, stream>>>(A, h->d, M);
    gp_note_launches(2);
    if ((rc = fit_factor(h, A, work, fwork, st, stream))) return fail(rc);
    if ((rc = read_status(st, stream))) return fail(rc);
    *out = h;
    return GP_OK;
}
}  // namespace

GPFAGP_API int gp_fit_gram_ex(const double* G, const double* b, int64_t N, int p, int n, double eps,
                              double alpha, double sigma2, int prec, void* cuda_stream, int dev_ptrs,
                              gp_model** out) {
    return fit_from_gram(G, b, false, N, p, n, eps, alpha, sigma2, prec, cuda_stream, dev_ptrs, out);
}

GPFAGP_API int gp_fit_gram_packed_ex(const double* packed, int64_t N, int p, int n, double eps, double alpha,
                                     double sigma2, int prec, void* cuda_stream, int dev_ptrs, gp_model** out) {
    return fit_from_gram(packed, nullptr, true, N, p, n, eps, alpha, sigma2, prec, cuda_stream, dev_ptrs, out);
}

GPFAGP_API gp_model* gp_fit(const double* X, const double* y, int64_t N, int p, int n, double eps,
                            double alpha, double sigma2) {
    gp_model* h = nullptr;
    gp_fit_ex(X, y, N, p, n, eps, alpha, sigma2, GP_PREC_MIXED, nullptr, 0, &h);
    return h;
}

GPFAGP_API int gp_predict_ex(const gp_model* h, const double* Xs, int64_t Ns, double* mean,
                             double* var, void* cuda_stream, int dev_ptrs) {
    set_err(GP_OK);
    int rc, dev;
    if (!h || Ns < 0) return set_err(GP_EINVAL, 0);
    if (Ns == 0) return GP_OK;
    if (!Xs || !mean) return set_err(GP_EINVAL, 0);
    if ((rc = check_device(&dev))) return rc;
    if (dev != h->device) return set_err(GP_EINVAL, 5);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    Scratch sc(stream);
    GpStatus* st;
    if ((rc = sc.get(&st, 1))) return rc;
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    const double* Xd = Xs;
    double *md = mean, *vd = var;
    if (!dev_ptrs) {
        double* xx;
        if ((rc = sc.get(&xx, (size_t)Ns * h->shape.p))) return rc;
        if ((rc = sc.get(&md, (size_t)Ns))) return rc;
        if (var && (rc = sc.get(&vd, (size_t)Ns))) return rc;
        cudaMemcpyAsync(xx, Xs, sizeof(double) * Ns * h->shape.p, cudaMemcpyHostToDevice, stream);
        Xd = xx;
    }
    if ((rc = predict_compute(h, Xd, Ns, md, vd, st, sc, stream))) return rc;
    if (!dev_ptrs) {
        cudaMemcpyAsync(mean, md, sizeof(double) * Ns, cudaMemcpyDeviceToHost, stream);
        if (var) cudaMemcpyAsync(var, vd, sizeof(double) * Ns, cudaMemcpyDeviceToHost, stream);
    }
    return read_status(st, stream);
}

GPFAGP_API int gp_predict_cov_ex(const gp_model* h, const double* Xs, int64_t Ns, double* mean, double* cov,
                                 int noisy, void* cuda_stream, int dev_ptrs) {
    set_err(GP_OK);
    int rc, dev;
    if (!h || Ns < 0) return set_err(GP_EINVAL, 0);
    if (Ns == 0) return GP_OK;
    if (!Xs || !cov) return set_err(GP_EINVAL, 0);
    if (Ns > GP_COV_MAX_NS) return set_err(GP_EINVAL, 6);
    if ((rc = check_device(&dev))) return rc;
    if (dev != h->device) return set_err(GP_EINVAL, 5);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    Scratch sc(stream);
    GpStatus* st;
    if ((rc = sc.get(&st, 1))) return rc;
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    GpShape s = h->shape;
    s.N = Ns;
    s.Npad = gp_round_up(Ns, 128);
    const double* Xd = Xs;
    double *md = mean, *cd = cov;
    const size_t ncov = (size_t)Ns * (size_t)Ns;
    if (!dev_ptrs) {
        double* xx;
        if ((rc = sc.get(&xx, (size_t)Ns * s.p))) return rc;
        if ((rc = sc.get(&cd, ncov))) return rc;
        cudaMemcpyAsync(xx, Xs, sizeof(double) * Ns * s.p, cudaMemcpyHostToDevice, stream);
        Xd = xx;
        md = nullptr;
    }
    if (md == nullptr && (rc = sc.get(&md, (size_t)Ns))) return rc;  // the kernels always form the mean
    cudaError_t e;
    if (h->prec == GP_PREC_FP64) {
        double *tab, *part, *z;
        if ((rc = sc.get(&tab, (size_t)s.p * s.n * s.Npad))) return rc;
        if ((rc = sc.get(&part, predict64_part_elems(s.Npad, s.M)))) return rc;
        if ((rc = sc.get(&z, predict64_z_elems(s.Npad, s.M)))) return rc;
        launch_eig_tables_f64(s, Xd, nullptr, tab, st, stream);
        e = launch_predict64(s, tab, h->W, h->c, h->sigma2, part, md, nullptr, stream, z);
        if (e == cudaSuccess) {
            GpProf pf("cov64", stream);
            e = launch_cov64(z, Ns, (int)(predict64_z_elems(s.Npad, s.M) / (size_t)s.Npad), h->sigma2, noisy, cd,
                             stream);
        }
        gp_note_launches(4);
    } else {
        float* tab;
        uint8_t* zpack;
        if ((rc = sc.get(&tab, (size_t)s.p * s.n * s.Npad))) return rc;
        if ((rc = sc.get(&zpack, predtc_zpack_bytes(s.Npad, s.M)))) return rc;
        launch_eig_tables_f32(s, Xd, nullptr, tab, st, stream);
        e = launch_predict_tc(s, tab, h->Wpack, h->cinfo, h->sigma2, md, nullptr, st, stream, zpack);
        if (e == cudaSuccess) {
            GpProf pf("cov_tc", stream);
            e = launch_cov_tc(zpack, Ns, s.Npad, s.M, h->sigma2, noisy, cd, st, stream);
        }
        gp_note_launches(3);
    }
    if (e != cudaSuccess) return cuda_err(e, "covariance launch");
    if (!dev_ptrs) {
        if (mean) cudaMemcpyAsync(mean, md, sizeof(double) * Ns, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(cov, cd, sizeof(double) * ncov, cudaMemcpyDeviceToHost, stream);
    }
    return read_status(st, stream);
}

GPFAGP_API int gp_predict(const gp_model* h, const double* Xs, int64_t Ns, double* mean, double* var) {
    return gp_predict_ex(h, Xs, Ns, mean, var, nullptr, 0);
}

GPFAGP_API void gp_free(gp_model* h) { free_model(h); }

GPFAGP_API int gp_model_log_marginal(const gp_model* h, const double* y, int64_t N, double* out,
                                     void* cuda_stream, int dev_ptrs) {
    set_err(GP_OK);
    int rc, dev;
    if (!h || !y || !out) return set_err(GP_EINVAL, 0);
    if (N != h->shape.N) return set_err(GP_EINVAL, 1);
    if ((rc = check_device(&dev))) return rc;
    if (dev != h->device) return set_err(GP_EINVAL, 5);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int M = h->shape.M;
    const int nparts = lml_partial_count(num_sms(dev));
    Scratch sc(stream);
    double *part, *terms;
    if ((rc = sc.get(&part, (size_t)4 * nparts))) return rc;
    if ((rc = sc.get(&terms, 4))) return rc;
    const double* yd = y;
    if (!dev_ptrs) {
        double* yy;
        if ((rc = sc.get(&yy, (size_t)N))) return rc;
        cudaMemcpyAsync(yy, y, sizeof(double) * N, cudaMemcpyHostToDevice, stream);
        yd = yy;
    }
    launch_lml_terms(yd, N, h->L, h->b, h->c, h->d, M, nparts, part, terms, stream);
    gp_note_launches(2);
    double t[4];
    cudaError_t e = cudaMemcpyAsync(t, terms, sizeof(t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_err(e, "log marginal likelihood");
    const double s2 = h->sigma2;
    const double two_pi = 6.283185307179586476925286766559;
    *out = -0.5 * ((t[0] - t[1]) / s2 + (double)N * log(s2) + 2.0 * t[2] - t[3] + (double)N * log(two_pi));
    return GP_OK;
}

GPFAGP_API int gp_model_log_marginal_grad(const gp_model* h, const double* y, int64_t N, double* lml,
                                          double* dlml_dsigma2, void* cuda_stream, int dev_ptrs) {
    set_err(GP_OK);
    int rc, dev;
    if (!h || !y || !lml || !dlml_dsigma2) return set_err(GP_EINVAL, 0);
    if (N != h->shape.N) return set_err(GP_EINVAL, 1);
    if ((rc = check_device(&dev))) return rc;
    if (dev != h->device) return set_err(GP_EINVAL, 5);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int M = h->shape.M;
    const int nparts = lml_partial_count(num_sms(dev));
    Scratch sc(stream);
    double *part, *terms, *ainv;
    GpStatus* st;
    if ((rc = sc.get(&part, (size_t)4 * nparts))) return rc;
    if ((rc = sc.get(&terms, 8))) return rc;
    if ((rc = sc.get(&ainv, (size_t)M))) return rc;
    if ((rc = sc.get(&st, 1))) return rc;
    cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);
    const double* yd = y;
    if (!dev_ptrs) {
        double* yy;
        if ((rc = sc.get(&yy, (size_t)N))) return rc;
        cudaMemcpyAsync(yy, y, sizeof(double) * N, cudaMemcpyHostToDevice, stream);
        yd = yy;
    }
    // diag(A^{-1}) from W = L^{-1}: the float64 model keeps W; for the mixed
    // model it is formed again from L in float64 (in a factor workspace whose
    // barrier header is zeroed here). Not in float32 as its variance does:
    // where d_m nears its clamp, L_mm reaches 1e100 and 1/L_mm underflows in
    // float32, and tr(A^{-1} E) weights (A^{-1})_mm ~ 1/d_m by e_m = d_m/sigma^2,
    // so each such column would lose a whole 1/sigma^2 from the gradient.
    const double* Wsrc = h->W;
    if (Wsrc == nullptr) {
        unsigned char* fwork;
        double* Wd;
        if ((rc = sc.get(&fwork, factor_work_bytes(M, false)))) return rc;
        if ((rc = sc.get(&Wd, (size_t)M * M))) return rc;
        cudaMemsetAsync(fwork, 0, 256, stream);
        cudaError_t e = launch_tri_inverse(h->L, Wd, M, false, st, fwork, stream);
        if (e != cudaSuccess) return cuda_err(e, "inverse for the likelihood gradient");
        gp_note_launches(1);
        Wsrc = Wd;
    }
    launch_ainv_diag(Wsrc, false, M, ainv, stream);
    gp_note_launches(1);
    launch_lml_terms(yd, N, h->L, h->b, h->c, h->d, M, nparts, part, terms, stream);
    launch_lml_grad_terms(h->c, h->d, ainv, h->sigma2, M, nparts, part, terms + 4, stream);
    gp_note_launches(4);
    double t[8];
    cudaError_t e = cudaMemcpyAsync(t, terms, sizeof(t), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_err(e, "log marginal likelihood gradient");
    if ((rc = read_status(st, stream))) return rc;
    const double s2 = h->sigma2;
    const double two_pi = 6.283185307179586476925286766559;
    const double quad = t[0] - t[1];  // y^T y - b^T c
    *lml = -0.5 * (quad / s2 + (double)N * log(s2) + 2.0 * t[2] - t[3] + (double)N * log(two_pi));
    // d log p / d sigma^2 = -1/2 [ c^T E c / s2 - quad / s2^2 + N / s2 + tr(A^{-1} E) - n_u / s2 ]
    *dlml_dsigma2 = -0.5 * (t[4] / s2 - quad / (s2 * s2) + (double)N / s2 + t[5] - t[6] / s2);
    return GP_OK;
}

GPFAGP_API int gp_model_info(const gp_model* h, int64_t* M, int* p, int* n, int* prec) {
    if (!h) return set_err(GP_EINVAL, 0);
    if (M) *M = h->shape.M;
    if (p) *p = h->shape.p;
    if (n) *n = h->shape.n;
    if (prec) *prec = h->prec;
    return GP_OK;
}

GPFAGP_API int gp_model_read(const gp_model* h, int field, double* dst) {
    set_err(GP_OK);
    if (!h || !dst) return set_err(GP_EINVAL, 0);
    const size_t M = (size_t)h->shape.M;
    const double* src = nullptr;
    size_t cnt = M;
    switch (field) {
        case GP_FIELD_L: src = h->L; cnt = M * M; break;
        case GP_FIELD_C: src = h->c; break;
        case GP_FIELD_B: src = h->b; break;
        case GP_FIELD_D: src = h->d; break;
        default: return set_err(GP_EINVAL, field);
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaError_t e = cudaMemcpy(dst, src, cnt * sizeof(double), cudaMemcpyDeviceToHost);
    cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_err(e, "model read");
    return GP_OK;
}

GPFAGP_API int gp_fit_batch(int count, const gp_fit_args* args, int prec, void* cuda_stream,
                            int dev_ptrs, gp_model** out) {
    set_err(GP_OK);
    g_batch_graph = 0;
    g_last_plan = BatchPlan();
    int rc, dev;
    if (count < 0 || (count > 0 && (!args || !out))) return set_err(GP_EINVAL, 0);
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    if (count == 0) return GP_OK;
    if ((rc = check_prec(prec))) return rc;
    for (int i = 0; i < count; ++i) {
        const gp_fit_args& a = args[i];
        if (!a.X || !a.y) return set_err(GP_EINVAL, i);
        if (check_hyper(a.N, a.p, a.n, a.eps, a.alpha, a.sigma2)) return set_err(GP_EINVAL, i);
    }
    if ((rc = check_device(&dev))) return rc;
    // The legacy default stream cannot be captured: the batch then runs on a
    // stream of its own, ordered after the work already queued there.
    struct OwnStream {
        cudaStream_t s = nullptr;
        ~OwnStream() {
            if (s) cudaStreamDestroy(s);
        }
    } own;
    cudaStream_t origin = (cudaStream_t)cuda_stream;
    if (origin == nullptr) {
        cudaEvent_t ev;
        cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaEventRecord(ev, nullptr);
        cudaStreamWaitEvent(own.s, ev, 0);
        cudaEventDestroy(ev);
        origin = own.s;
    }
    const int sms = num_sms(dev);

    // models, inputs on the device, shape-only inputs: all before any capture
    std::vector<gp_model*> hs(count, nullptr);
    std::vector<FitStage> stages(count);
    std::vector<const double*> Xd(count), yd(count);
    Scratch keep(origin);  // inputs and statuses, freed after the batch has run
    GpStatus* sts = nullptr;
    auto fail_all = [&](int code, int idx) {
        int64_t det = g_detail;
        cudaStreamSynchronize(origin);
        for (gp_model* h : hs) free_model(h);
        set_err(code, idx >= 0 ? idx : det);
        return code;
    };
    if ((rc = keep.get(&sts, (size_t)count))) return fail_all(rc, -1);
    cudaMemsetAsync(sts, 0, sizeof(GpStatus) * count, origin);
    std::vector<double*> loglam(count);
    for (int i = 0; i < count; ++i) {
        const gp_fit_args& a = args[i];
        hs[i] = new_model(dev, prec, a.N, a.p, a.n, a.eps, a.alpha, a.sigma2);
        if ((rc = fit_alloc(hs[i], origin))) return fail_all(rc, i);
        if ((rc = keep.get(&loglam[i], (size_t)a.p * a.n))) return fail_all(rc, i);
        if ((rc = fit_stage(hs[i], stages[i], loglam[i], origin))) return fail_all(rc, i);
        Xd[i] = a.X;
        yd[i] = a.y;
        if (!dev_ptrs) {
            double *xx, *yy;
            if ((rc = keep.get(&xx, (size_t)a.N * a.p))) return fail_all(rc, i);
            if ((rc = keep.get(&yy, (size_t)a.N))) return fail_all(rc, i);
            cudaMemcpyAsync(xx, a.X, sizeof(double) * a.N * a.p, cudaMemcpyHostToDevice, origin);
            cudaMemcpyAsync(yy, a.y, sizeof(double) * a.N, cudaMemcpyHostToDevice, origin);
            Xd[i] = xx;
            yd[i] = yy;
        }
    }
    cudaError_t e = cudaStreamSynchronize(origin);  // staged host inputs have been read
    if (e != cudaSuccess) return fail_all(cuda_err(e, "batch input staging"), -1);

    StreamSet ss(std::min(count, 32));
    BatchCtx ctx{&hs, &Xd, &yd, &loglam, sts, dev, sms, origin, &ss, {}};
    BatchPlan plan;
    if ((rc = plan_batch(ctx, &plan))) return fail_all(rc, -1);
    int graph = 0;
    if ((rc = run_batch(ctx, plan, nullptr, &graph))) return fail_all(rc, -1);
    g_batch_graph = graph;
    g_last_plan = plan;

    std::vector<GpStatus> hst(count);
    e = cudaMemcpy(hst.data(), sts, sizeof(GpStatus) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_all(cuda_err(e, "batch status read"), -1);
    // members whose mixed Gram was not accurate enough: float64 Gram, one by one
    for (int i = 0; i < count; ++i) {
        if (!mixed_escalates(hs[i], hst[i].code)) continue;
        cudaMemsetAsync(&sts[i], 0, sizeof(GpStatus), origin);
        Scratch sc2(origin);
        rc = fit_compute(hs[i], Xd[i], yd[i], loglam[i], &sts[i], 0, sc2, origin, GP_PREC_FP64);
        if (rc != GP_OK) return fail_all(rc, i);
        e = cudaMemcpyAsync(&hst[i], &sts[i], sizeof(GpStatus), cudaMemcpyDeviceToHost, origin);
        if (e == cudaSuccess) e = cudaStreamSynchronize(origin);
        if (e != cudaSuccess) return fail_all(cuda_err(e, "batch status read"), -1);
    }
    set_err(GP_OK);
    int first = GP_OK;
    int64_t first_idx = 0;
    for (int i = 0; i < count; ++i) {
        if (hst[i].code != GP_OK) {
            if (first == GP_OK) {
                first = hst[i].code;
                first_idx = i;
            }
            free_model(hs[i]);
            hs[i] = nullptr;
        }
        out[i] = hs[i];
    }
    if (first != GP_OK) return set_err(first, first_idx);
    return GP_OK;
}

GPFAGP_API int gp_batch_info(int* used_graph, int* tuned_k) {
    if (used_graph) *used_graph = g_batch_graph;
    if (tuned_k) *tuned_k = g_last_plan.k;
    return GP_OK;
}

GPFAGP_API int gp_batch_plan(int* streams, int* k, int* factor_ctas, int* from_cache, double* tuned_ms) {
    if (streams) *streams = g_last_plan.streams;
    if (k) *k = g_last_plan.k;
    if (factor_ctas) {
        int dev = 0;
        cudaGetDevice(&dev);
        *factor_ctas = plan_factor_ctas(g_last_plan, num_sms(dev));
    }
    if (from_cache) *from_cache = g_last_plan.cached ? 1 : 0;
    if (tuned_ms) *tuned_ms = g_last_plan.ms;
    return GP_OK;
}

GPFAGP_API int gp_predict_batch(int count, const gp_predict_args* args, void* cuda_stream) {
    set_err(GP_OK);
    if (count < 0 || (count > 0 && !args)) return set_err(GP_EINVAL, 0);
    if (count == 0) return GP_OK;
    int rc, dev;
    for (int i = 0; i < count; ++i) {
        const gp_predict_args& a = args[i];
        if (!a.model || a.Ns < 0 || (a.Ns > 0 && (!a.Xs || !a.mean))) return set_err(GP_EINVAL, i);
    }
    if ((rc = check_device(&dev))) return rc;
    for (int i = 0; i < count; ++i)
        if (args[i].model->device != dev) return set_err(GP_EINVAL, i);
    cudaStream_t origin = (cudaStream_t)cuda_stream;
    Scratch keep(origin);
    GpStatus* sts;
    if ((rc = keep.get(&sts, (size_t)count))) return rc;
    cudaMemsetAsync(sts, 0, sizeof(GpStatus) * count, origin);
    // mixed-precision models: one batched launch sequence on `origin`;
    // float64 models: their own kernels, side by side on a few streams
    std::vector<PredEntry> mixed;
    std::vector<int> f64;
    for (int i = 0; i < count; ++i) {
        const gp_predict_args& a = args[i];
        if (a.Ns == 0) continue;
        if (a.model->prec == GP_PREC_FP64) f64.push_back(i);
        else mixed.push_back(PredEntry{a.model, a.Xs, a.Ns, a.mean, a.var, &sts[i]});
    }
    int first = GP_OK;
    int64_t first_idx = 0;
    if (!mixed.empty()) {
        PredBatch pb;
        uint8_t* up = nullptr;
        rc = pred_batch_build(mixed, keep, pb);
        if (rc == GP_OK) rc = keep.get(&up, pb.total);
        if (rc == GP_OK) {
            std::vector<uint8_t> img(pb.total);
            pred_batch_pack(pb, img.data(), up);
            // from pageable memory: returns once the image is staged
            cudaError_t e = cudaMemcpyAsync(up, img.data(), pb.total, cudaMemcpyHostToDevice, origin);
            rc = e == cudaSuccess ? pred_batch_enqueue(pb, up, origin) : cuda_err(e, "batch upload");
        }
        if (rc != GP_OK) {
            first = rc;
            first_idx = 0;
        }
    }
    if (!f64.empty() && first == GP_OK) {
        StreamSet ss(f64.size() < 8 ? (int)f64.size() : 8);
        ss.fork(origin);
        std::vector<Scratch*> scs;
        for (size_t k = 0; k < f64.size(); ++k) {
            const int i = f64[k];
            const gp_predict_args& a = args[i];
            cudaStream_t s = ss.st[k % ss.st.size()];
            Scratch* sc = new Scratch(s);
            scs.push_back(sc);
            rc = predict_compute(a.model, a.Xs, a.Ns, a.mean, a.var, &sts[i], *sc, s);
            if (rc != GP_OK && first == GP_OK) {
                first = rc;
                first_idx = i;
            }
        }
        for (Scratch* sc : scs) delete sc;
        ss.join(origin);
    }
    cudaError_t e = cudaStreamSynchronize(origin);
    if (e != cudaSuccess) return cuda_err(e, "batch synchronise");
    if (first != GP_OK) return set_err(first, first_idx);
    std::vector<GpStatus> hst(count);
    e = cudaMemcpy(hst.data(), sts, sizeof(GpStatus) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "batch status read");
    for (int i = 0; i < count; ++i)
        if (hst[i].code != GP_OK) return set_err(hst[i].code, i);
    return GP_OK;
}

}  // extern "C"
