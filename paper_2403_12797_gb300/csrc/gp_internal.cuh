// gp_internal.cuh -- library-internal interface shared by the C ABI
// (gp_api.cu) and the request server (gp_server.cu): the model record,
// stream-ordered scratch memory, and the enqueue-only fit and predict steps.
#pragma once

#include "gp_kernels.cuh"

#include <vector>

struct gp_model {
    int device;
    int prec;
    GpShape shape;          // N / Npad of the training set (informational)
    double eps[GP_PMAX];    // eps_j and alpha_j (rho_j) per input dimension (equal: isotropic)
    double alpha[GP_PMAX];
    double sigma2;
    double* L;              // M x M lower Cholesky factor of A
    double* W;              // M x M, L^{-1}
    double* c;              // M, A^{-1} b
    double* b;              // M, Phi^T y
    double* d;              // M, sigma^2 / lambda_m (clamped)
    uint16_t* Wpack;        // bf16 hi/lo operand layout of W (GP_PREC_MIXED only)
    int* cinfo;             // chunk table of the tensor-core predict (GP_PREC_MIXED only)
    int flags;              // GP_MODEL_GRAM_FP64: Gram recomputed in float64 (mixed mode)
    void* block;            // the one device allocation the buffers above are carved from
};

namespace gpi {

// thread-local status of the last ABI call (gp_last_error / _detail)
int set_err(int code, int64_t detail = 0);
// GP_ECUDA with detail = the CUDA error code; `where` names the failing step
int cuda_err(cudaError_t e, const char* where = "");
// stream-ordered allocation (honours gp_debug_fail_alloc_after)
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);

// Stream-ordered scratch: requests are carved (256-byte aligned) from chunks
// of at least 1 MiB, so a fit makes a few allocations instead of one per
// buffer; every chunk is freed on the stream when the object goes out of
// scope.
struct Scratch {
    static constexpr size_t kChunk = (size_t)1 << 20;
    cudaStream_t s;
    std::vector<void*> ptrs;  // chunks
    char* cur = nullptr;
    size_t left = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
    template <typename T>
    int get(T** p, size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        if (bytes > left) {
            const size_t sz = bytes > kChunk ? bytes : kChunk;
            void* v = nullptr;
            cudaError_t e = dev_alloc(&v, sz, s);
            if (e == cudaErrorMemoryAllocation) return set_err(GP_ENOMEM, (int64_t)sz);
            if (e != cudaSuccess) return cuda_err(e, "scratch allocation");
            ptrs.push_back(v);
            if (bytes >= kChunk) {  // a large request takes its chunk alone
                *p = (T*)v;
                return GP_OK;
            }
            cur = (char*)v;
            left = sz;
        }
        *p = (T*)cur;
        cur += bytes;
        left -= bytes;
        return GP_OK;
    }
};

int check_device(int* dev_out);
int num_sms(int dev);
int tile_of(int prec);
void free_model(gp_model* h);

gp_model* new_model(int dev, int prec, int64_t N, int p, int n, double eps, double alpha, double sigma2);
// eps[j], alpha[j] for the p input dimensions (ARD)
gp_model* new_model(int dev, int prec, int64_t N, int p, int n, const double* eps, const double* alpha, double sigma2);
// the model's own device buffers
int fit_alloc(gp_model* h, cudaStream_t stream);

// Host inputs of one fit that its asynchronous copies read: kept alive by
// the caller until the stream (or graph) has run.
// Page-locked host memory from a process-wide pool (allocated on first need,
// reused afterwards): copies from it are asynchronous, where a copy from
// pageable memory first waits for the whole stream.
struct PinnedBlock {
    void* p = nullptr;
    size_t cap = 0;
};
PinnedBlock pinned_get(size_t bytes);  // p == nullptr if the allocation failed
void pinned_put(PinnedBlock b);

// Host staging of a fit's shape-only inputs, in pinned memory that stays
// valid until the object is destroyed (after the stream has been synchronised
// or the captured graph has run).
struct FitStage {
    PinnedBlock buf;
    FitStage() = default;
    FitStage(const FitStage&) = delete;
    FitStage& operator=(const FitStage&) = delete;
    ~FitStage() {
        if (buf.p) pinned_put(buf);
    }
};

// shape-only inputs to the device (log eigenvalues; predict chunk table into the model)
int fit_stage(gp_model* h, FitStage& stage, double* loglam_d, cudaStream_t stream);
// every device step of a fit / of a predict, enqueued without host synchronisation
// gram_prec: precision of the Gram step (-1: the model's); factor_ctas > 0
// caps the factorisation kernels' grids (batched fits); the mixed mode
// escalates to GP_PREC_FP64 after a non-positive pivot (see mixed_escalates)
int fit_compute(gp_model* h, const double* Xd, const double* yd, const double* loglam_d, GpStatus* st,
                int gram_ctas, Scratch& sc, cudaStream_t stream, int gram_prec = -1, int factor_ctas = 0);
// whether a fit that ended with `code` is redone with the float64 Gram: a
// mixed-precision fit whose Cholesky met a non-positive pivot
bool mixed_escalates(const gp_model* h, int code);
int predict_compute(const gp_model* h, const double* Xd, int64_t Ns, double* md, double* vd, GpStatus* st,
                    Scratch& sc, cudaStream_t stream);

// ---- batched predicts ----------------------------------------------------
// Predicts against mixed-precision models, laid out for one upload and run
// as one table launch plus one persistent predict launch per basis
// dimension p among them. Each request's results are those of
// predict_compute (the same per-point arithmetic and summation order).
struct PredEntry {
    const gp_model* m;  // GP_PREC_MIXED
    const double* Xd;   // Ns x p test points (device)
    int64_t Ns;
    double* md;         // device outputs
    double* vd;         // or NULL
    GpStatus* st;       // this request's status word (device)
};
struct PredBatch {
    std::vector<PredReq> reqs;
    std::vector<int2> items;    // (request, tile * nsuper + super-tile), grouped by p, costlier first
    std::vector<int64_t> cost;  // per item while building
    std::vector<int> boff;      // table blocks of each request (nreq + 1)
    std::vector<float> consts;  // 3p per request; PredReq::consts holds the float offset until pack()
    struct Group {
        int p, first, count, maxrows;
    };
    std::vector<Group> groups;
    int max_n = 0, nblocks = 0;
    bool reduce = false;        // some request sums partial variances (launch_predict_reduce_batch)
    int64_t max_npad = 0;
    size_t off_items = 0, off_boff = 0, off_consts = 0, total = 0;  // upload layout (bytes)
};
// Lays out the entries (tables of X* taken from sc) and sizes the upload.
int pred_batch_build(const std::vector<PredEntry>& es, Scratch& sc, PredBatch& pb);
// Writes the upload image for device address dev into host (pb.total bytes).
void pred_batch_pack(PredBatch& pb, void* host, const uint8_t* dev);
// The launches, once the image is on the device at dev (stream-ordered).
int pred_batch_enqueue(const PredBatch& pb, const uint8_t* dev, cudaStream_t stream);

}  // namespace gpi
