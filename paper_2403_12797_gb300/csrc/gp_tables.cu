// gp_tables.cu -- per-dimension eigenfunction tables (Sec. 2.3, Eq. 14-15).
//
// For every point i and input dimension j the kernel evaluates the n SE
// eigenfunctions phi_k(x_ij) = gamma_k exp(-delta^2 x^2) H_{k-1}(rho beta x)
// through the normalised Hermite recurrence (the quantity gamma_{k+1} H_k(t)
// satisfies q_{k+1} = sqrt(2/(k+1)) t q_k - sqrt(k/(k+1)) q_{k-1},
// q_0 = sqrt(beta), q_1 = sqrt(2) t q_0), so nothing overflows for large n.
//
// Layouts: T[(j * n + k) * Npad + i] (float64 Gram, predictions), or chunk-major
// for the mixed-precision Gram (below); rows i >= N are zero. A column of Phi
// (Eq. 19) is the product of one row per dimension of this table, formed
// later inside the contraction kernels: Phi itself is never stored.
#include "gp_kernels.cuh"

#include <math.h>

namespace {

// up to this n the recurrence coefficients are staged in shared memory
constexpr int COEF_SMEM_N = 2048;

template <typename T>
__device__ __forceinline__ T gp_exp(T v);
template <>
__device__ __forceinline__ float gp_exp<float>(float v) { return expf(v); }
template <>
__device__ __forceinline__ double gp_exp<double>(double v) { return exp(v); }

template <typename T>
__device__ __forceinline__ T gp_sqrt(T v);
template <>
__device__ __forceinline__ float gp_sqrt<float>(float v) { return sqrtf(v); }
template <>
__device__ __forceinline__ double gp_sqrt<double>(double v) { return sqrt(v); }

// float64 -> T without the float64 pipe (T = float: integer rounding)
__device__ __forceinline__ float to_tab(double x, float*) { return gp_d2f_rn(x); }
__device__ __forceinline__ double to_tab(double x, double*) { return x; }

// The shape constants of dimension j (rho_j beta_j, sqrt(beta_j), delta_j^2),
// in T: the float ones were rounded on the host (on GB300 the conversion
// instruction, like every float64 operation, holds its scheduler's float64
// pipe for 64 cycles a warp).
__device__ __forceinline__ void shape_consts(const GpShape& s, int j, double& ab, double& sb, double& d2) {
    ab = s.ab[j];
    sb = s.sb[j];
    d2 = s.d2[j];
}
__device__ __forceinline__ void shape_consts(const GpShape& s, int j, float& ab, float& sb, float& d2) {
    ab = s.abf[j];
    sb = s.sbf[j];
    d2 = s.d2f[j];
}
// Table column i (one point) of dimension j: out[k * Npad] = phi_k(x_ij),
// k = 0 .. n-1 (zero for padding rows i >= N and for non-finite input, which
// also records GP_EINVAL with the row). ca, cb: the recurrence coefficients
// when staged.
template <typename T>
__device__ __forceinline__ void eig_column(const double* __restrict__ X, const double* __restrict__ y, int64_t i,
                                           int j, int64_t N, int64_t Npad, int p, int n, T abT, T sbT, T d2T,
                                           const T* ca, const T* cb, bool staged, T* __restrict__ out,
                                           GpStatus* st) {
    if (i >= N) {
        for (int k = 0; k < n; ++k) out[(int64_t)k * Npad] = T(0);
        return;
    }
    const double xd = X[i * p + j];
    if (!gp_isfinite_bits(xd) || (j == 0 && y != nullptr && !gp_isfinite_bits(y[i]))) {
        gp_set_status(st, GP_EINVAL, i);
        for (int k = 0; k < n; ++k) out[(int64_t)k * Npad] = T(0);
        return;
    }
    const T x = to_tab(xd, (T*)nullptr);
    const T t = abT * x;
    T q0 = sbT * gp_exp<T>(-d2T * x * x);
    out[0] = q0;
    if (n == 1) return;
    T q1 = gp_sqrt<T>(T(2)) * t * q0;
    out[Npad] = q1;
    for (int k = 1; k + 1 < n; ++k) {
        const T a = staged ? ca[k] : gp_sqrt<T>(T(2) / T(k + 1));
        const T b = staged ? cb[k] : gp_sqrt<T>(T(k) / T(k + 1));
        const T q2 = a * t * q1 - b * q0;
        out[(int64_t)(k + 1) * Npad] = q2;
        q0 = q1;
        q1 = q2;
    }
}

template <typename T>
__device__ __forceinline__ void stage_coefs(int n, T* ca, T* cb) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        ca[k] = gp_sqrt<T>(T(2) / T(k + 1));
        cb[k] = gp_sqrt<T>(T(k) / T(k + 1));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) eig_tables_kernel(GpShape s, const double* __restrict__ X,
                                                         const double* __restrict__ y,
                                                         T* __restrict__ tab, GpStatus* st) {
    // recurrence coefficients sqrt(2/(k+1)), sqrt(k/(k+1)), once per block
    extern __shared__ __align__(16) unsigned char coef_raw[];
    T* ca = reinterpret_cast<T*>(coef_raw);
    T* cb = ca + s.n;
    const bool staged = s.n <= COEF_SMEM_N;
    if (staged) {
        stage_coefs<T>(s.n, ca, cb);
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= s.Npad) return;
    T abT, sbT, d2T;
    shape_consts(s, j, abT, sbT, d2T);
    eig_column<T>(X, y, i, j, s.N, s.Npad, s.p, s.n, abT, sbT, d2T, ca, cb, staged,
                  tab + (int64_t)j * s.n * s.Npad + i, st);
}

// Every request of a predict batch: block b belongs to the request r with
// boff[r] <= b < boff[r + 1]; within it, dimension j = (b - boff[r]) % p and
// points 256 ((b - boff[r]) / p) + threadIdx.x. The per-point work is
// eig_column, as in eig_tables_kernel, so a request's tables are the same
// bits either way.
__global__ void __launch_bounds__(256) eig_tables_batch_kernel(const PredReq* __restrict__ reqs,
                                                               const int* __restrict__ boff, int nreq) {
    extern __shared__ __align__(16) unsigned char coef_raw[];
    const int b = blockIdx.x;
    int lo = 0, hi = nreq - 1;  // the last r with boff[r] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(boff + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    const PredReq& R = reqs[lo];
    const int p = R.p, n = R.n;
    const int local = b - __ldg(boff + lo);
    const int j = local % p;
    float* ca = reinterpret_cast<float*>(coef_raw);
    float* cb = ca + n;
    const bool staged = n <= COEF_SMEM_N;
    if (staged) {
        stage_coefs<float>(n, ca, cb);
        __syncthreads();
    }
    const int64_t i = (int64_t)(local / p) * blockDim.x + threadIdx.x;
    if (i >= R.Npad) return;
    const float abT = R.consts[3 * j], sbT = R.consts[3 * j + 1], d2T = R.consts[3 * j + 2];
    eig_column<float>(R.Xs, nullptr, i, j, R.Ns, R.Npad, p, n, abT, sbT, d2T, ca, cb, staged,
                      R.tab + (int64_t)j * n * R.Npad + i, R.st);
}

// The same recurrence, written in the chunk-major layout of the mixed-precision
// Gram: for chunk q = i / 32 of the rows, table row R = j * n + k at
// T[q * RC + R * WS + i % 32] (WS = 36 floats, the last 4 zero) and y in row
// R = p * n, RC = (p * n + 1) * WS. One chunk's rows of every table row are
// thus one contiguous block that a single bulk copy can move.
__global__ void __launch_bounds__(256) eig_tables_chunked_kernel(GpShape s, const double* __restrict__ X,
                                                                 const double* __restrict__ y,
                                                                 float* __restrict__ tab, GpStatus* st) {
    constexpr int WS = SYRKTC_WS, CW = SYRKTC_BK;
    extern __shared__ __align__(16) unsigned char coef_raw[];
    float* ca = reinterpret_cast<float*>(coef_raw);
    float* cb = ca + s.n;
    const bool staged = s.n <= COEF_SMEM_N;
    if (staged) {
        for (int k = threadIdx.x; k < s.n; k += blockDim.x) {
            ca[k] = sqrtf(2.f / (float)(k + 1));
            cb[k] = sqrtf((float)k / (float)(k + 1));
        }
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= s.Npad) return;  // whole warps: Npad is a multiple of 128
    const float abf = s.abf[j], sbf = s.sbf[j], d2f = s.d2f[j];
    const int rows = s.p * s.n + 1;
    float* chunk = tab + (i / CW) * (int64_t)rows * WS;
    const int k0 = (int)(i % CW);
    float* out = chunk + (int64_t)j * s.n * WS + k0;
    if (k0 < WS - CW) {  // zero the padding of this thread's share of the rows
        for (int k = 0; k < s.n; ++k) out[k * WS + CW] = 0.f;
        if (j == 0) chunk[(int64_t)(rows - 1) * WS + CW + k0] = 0.f;
    }
    bool zero = i >= s.N;
    double xd = 0.0;
    if (!zero) {
        xd = X[i * s.p + j];
        if (!gp_isfinite_bits(xd) || (j == 0 && y != nullptr && !gp_isfinite_bits(y[i]))) {
            gp_set_status(st, GP_EINVAL, i);
            zero = true;
        }
    }
    if (j == 0) chunk[(int64_t)(rows - 1) * WS + k0] = (zero || y == nullptr) ? 0.f : gp_d2f_rn(y[i]);
    // rows beyond N or with bad input are zero from q0 on
    auto emit = [&](int k, float v) { out[k * WS] = v; };
    const float x = zero ? 0.f : gp_d2f_rn(xd);
    const float t = abf * x;
    float q0 = zero ? 0.f : sbf * expf(-d2f * x * x);
    emit(0, q0);
    if (s.n == 1) return;
    float q1 = sqrtf(2.f) * t * q0;
    emit(1, q1);
    for (int k = 1; k + 1 < s.n; ++k) {
        const float a = staged ? ca[k] : sqrtf(2.f / (float)(k + 1));
        const float b = staged ? cb[k] : sqrtf((float)k / (float)(k + 1));
        const float q2 = a * t * q1 - b * q0;
        emit(k + 1, q2);
        q0 = q1;
        q1 = q2;
    }
}

template <typename T>
size_t coef_bytes(const GpShape& s) {
    return s.n <= COEF_SMEM_N ? 2 * sizeof(T) * (size_t)s.n : 0;
}

}  // namespace

void launch_eig_tables_f64(const GpShape& s, const double* X, const double* y, double* tab,
                           GpStatus* st, cudaStream_t stream) {
    dim3 grid((unsigned)((s.Npad + 255) / 256), (unsigned)s.p);
    eig_tables_kernel<double><<<grid, 256, coef_bytes<double>(s), stream>>>(s, X, y, tab, st);
}

void launch_eig_tables_f32(const GpShape& s, const double* X, const double* y, float* tab,
                           GpStatus* st, cudaStream_t stream) {
    dim3 grid((unsigned)((s.Npad + 255) / 256), (unsigned)s.p);
    eig_tables_kernel<float><<<grid, 256, coef_bytes<float>(s), stream>>>(s, X, y, tab, st);
}

void launch_eig_tables_batch(const PredReq* reqs, const int* boff, int nreq, int nblocks, int max_n,
                             cudaStream_t stream) {
    if (nblocks <= 0) return;
    const size_t smem = max_n <= COEF_SMEM_N ? 2 * sizeof(float) * (size_t)max_n : 0;
    eig_tables_batch_kernel<<<(unsigned)nblocks, 256, smem, stream>>>(reqs, boff, nreq);
}

size_t syrktc_table_floats(const GpShape& s) {
    return (size_t)(s.Npad / SYRKTC_BK) * (size_t)(s.p * s.n + 1) * SYRKTC_WS;
}

void launch_eig_tables_chunked(const GpShape& s, const double* X, const double* y, float* tabc, GpStatus* st,
                               cudaStream_t stream) {
    dim3 grid((unsigned)((s.Npad + 255) / 256), (unsigned)s.p);
    eig_tables_chunked_kernel<<<grid, 256, coef_bytes<float>(s), stream>>>(s, X, y, tabc, st);
}
