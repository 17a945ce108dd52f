// gp_static.cu -- the allocation-free Gram entry point gp_gram_static().
//
// Some callers cannot allocate device memory while they call into this
// library: code running under a custom or fixed device-memory budget (an
// inference server that carves all of HBM up front, a real-time loop that
// must not touch the allocator), or a framework whose allocator hook must
// not be re-entered. For them this file provides a variant of the float64
// Gram step whose scratch (eigenfunction tables, padded y, per-split partial
// tiles, status word) lives in one file-scope __device__ array of
// GP_STATIC_SCRATCH_BYTES bytes instead of memory obtained from
// cudaMallocAsync. The caller still passes the inputs and outputs.
//
// The array exists once per device that loads the library and stays
// allocated until the process exits. Host code cannot use the array's name
// as a device address: the first call on each device (with that device
// current) asks the runtime for the address with cudaGetSymbolAddress and
// keeps it; later calls reuse it. That first call must not happen inside a
// stream capture. The kept address belongs to the device's current context:
// after cudaDeviceReset the module is loaded anew and the address is stale,
// so this entry point must not be used again in a process that reset the
// device. All calls share the array and its contents persist
// between calls, so calls that overlap on the GPU (different streams or
// threads at the same time) race with each other; serialise them.
#include "gp_kernels.cuh"

#include <mutex>

namespace {

constexpr size_t kStaticBytes = GP_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_gram_scratch[kStaticBytes];

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of g_gram_scratch on the current device (set up once).
cudaError_t static_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = (unsigned char*)g_static_addr[dev];
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct StaticPlan {
    int nsplit;
    int64_t rps;
    size_t off_tab, off_y, off_G, off_b, total;
};

// Scratch layout for nsplit splits: status | tables | y | G partials | b partials.
StaticPlan plan_for(const GpShape& s, int npairs, int nsplit) {
    StaticPlan P;
    P.nsplit = nsplit;
    P.rps = gp_round_up((s.Npad + nsplit - 1) / nsplit, 128);
    P.nsplit = (int)((s.Npad + P.rps - 1) / P.rps);
    size_t o = align256(sizeof(GpStatus));
    P.off_tab = o;
    o = align256(o + sizeof(double) * (size_t)s.p * s.n * s.Npad);
    P.off_y = o;
    o = align256(o + sizeof(double) * (size_t)s.Npad);
    P.off_G = o;
    o = align256(o + sizeof(double) * (size_t)P.nsplit * npairs * SYRK64_TM * SYRK64_TM);
    P.off_b = o;
    o = align256(o + sizeof(double) * (size_t)P.nsplit * s.Mpad);
    P.total = o;
    return P;
}

__global__ void static_pad_y_kernel(const double* __restrict__ y, int64_t N, int64_t Npad,
                                    double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Npad) out[i] = i < N ? y[i] : 0.0;
}

}  // namespace

int gp_static_gram(const double* X, const double* y, int64_t N, int p, int n, double eps,
                   double alpha, double* G, double* b, cudaStream_t stream, int64_t* detail) {
    *detail = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *detail = e;
        return GP_ENODEV;
    }
    GpShape s;
    gp_fill_shape(&s, N, p, n, eps, alpha, SYRK64_TM);
    const int T = s.Mpad / SYRK64_TM;
    const int npairs = T * (T + 1) / 2;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // as many splits as fill the GPU, fewer if the scratch array is too small
    int want = (4 * sms + npairs - 1) / npairs;
    if (want > (int)(s.Npad / 256)) want = (int)(s.Npad / 256);
    if (want < 1) want = 1;
    StaticPlan P = plan_for(s, npairs, want);
    while (P.total > kStaticBytes && want > 1) {
        want = want / 2;
        P = plan_for(s, npairs, want);
    }
    if (P.total > kStaticBytes) {
        *detail = (int64_t)P.total;  // bytes this problem would need
        return GP_EINVAL;
    }
    unsigned char* base = nullptr;
    e = static_scratch(dev, &base);
    if (e != cudaSuccess) {
        *detail = e;
        return GP_ECUDA;
    }
    GpStatus* st = (GpStatus*)base;
    double* tab = (double*)(base + P.off_tab);
    double* ypad = (double*)(base + P.off_y);
    double* Gpart = (double*)(base + P.off_G);
    double* bpart = (double*)(base + P.off_b);
    e = cudaMemsetAsync(st, 0, sizeof(GpStatus), stream);  // the array keeps the last call's status
    if (e != cudaSuccess) {
        *detail = e;
        return GP_ECUDA;
    }
    launch_eig_tables_f64(s, X, y, tab, st, stream);
    static_pad_y_kernel<<<(unsigned)((s.Npad + 255) / 256), 256, 0, stream>>>(y, s.N, s.Npad, ypad);
    e = launch_syrk64(s, tab, ypad, P.nsplit, P.rps, Gpart, bpart, stream);
    if (e == cudaSuccess) {
        launch_assemble_f64(Gpart, bpart, P.nsplit, SYRK64_TM, s.Mpad, s.M, nullptr, G, b, stream);
        e = cudaGetLastError();
    }
    gp_note_launches(4);
    if (e != cudaSuccess) {
        *detail = e;
        return GP_ECUDA;
    }
    GpStatus h;
    e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        *detail = e;
        return GP_ECUDA;
    }
    if (h.code != GP_OK) {
        *detail = h.detail;
        return h.code;
    }
    return GP_OK;
}
