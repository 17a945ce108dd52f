// gp_assemble.cu -- split-N reduction and assembly of A = Phi^T Phi + sigma^2 Lambda^{-1}.
//
// A is sigma^2 times the Lambda-bar of Sec. 2.2 (with Sigma_n = sigma^2 I);
// its diagonal term d_m = sigma^2 / lambda_m uses the tensor-product
// eigenvalues lambda_m = prod_j lambda_{m_j} of Eq. 20 with lambda_k of
// Eq. 16, evaluated in log space and clamped at 1e200 so that eigenvalues
// that underflow stay finite.
//
// The partial Gram tiles of the N splits are summed in float64 in split
// order, so the result does not depend on scheduling.
#include "gp_kernels.cuh"

#include <math.h>

namespace {

// a partial value as float64 (float pairs hold hi + lo)
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float2 v) { return (double)v.x + (double)v.y; }

template <typename P, typename PB = P>
__global__ void __launch_bounds__(256) assemble_kernel(const P* __restrict__ Gpart,
                                                       const PB* __restrict__ bpart,
                                                       const PB* __restrict__ dpart,
                                                       const int* __restrict__ colexp, int nsplit,
                                                       int tile, int Mpad, int M,
                                                       const double* __restrict__ d,
                                                       double* __restrict__ A,
                                                       double* __restrict__ b) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y;
    if (col >= M) return;
    const int T = Mpad / tile;
    const int npairs = T * (T + 1) / 2;
    // read the lower-triangle element (r >= c), so A is exactly symmetric
    const int r = row >= col ? row : col;
    const int c = row >= col ? col : row;
    const int I = r / tile, J = c / tile;
    const int q = I * (I + 1) / 2 + J;
    const int64_t off = (int64_t)q * tile * tile + (int64_t)(r % tile) * tile + (c % tile);
    const int64_t sstride = (int64_t)npairs * tile * tile;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += to_f64(Gpart[off + s * sstride]);
    if (row == col && dpart != nullptr)
        for (int s = 0; s < nsplit; ++s) acc += to_f64(dpart[(int64_t)s * Mpad + row]);
    if (colexp != nullptr) acc = ldexp(acc, colexp[r] + colexp[c] - 14);
    if (row == col && d != nullptr) acc += d[row];
    A[(int64_t)row * M + col] = acc;
    if (row == 0) {
        double bb = 0.0;
        for (int s = 0; s < nsplit; ++s) bb += to_f64(bpart[(int64_t)s * Mpad + col]);
        b[col] = bb;
    }
}

__global__ void noise_diag_kernel(GpShape s, const double* __restrict__ loglam, double log_sigma2,
                                  double* __restrict__ d) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= s.M) return;
    double ll = 0.0;
    for (int j = 0; j < s.p; ++j) ll += loglam[(m / s.stride[j]) % s.n];
    const double logd = log_sigma2 - ll;
    const double lclamp = 460.51701859880913680;  // log(1e200)
    d[m] = logd >= lclamp ? 1e200 : exp(logd);
}

}  // namespace

void launch_assemble_f64(const double* Gpart, const double* bpart, int nsplit, int tile, int Mpad,
                         int M, const double* d, double* A, double* b, cudaStream_t stream) {
    dim3 grid((unsigned)((M + 255) / 256), (unsigned)M);
    assemble_kernel<double, double><<<grid, 256, 0, stream>>>(Gpart, bpart, nullptr, nullptr, nsplit, tile,
                                                      Mpad, M, d, A, b);
}

void launch_assemble_f32(const float* Gpart, const float* bpart, const float* dpart,
                         const int* colexp, int nsplit, int tile, int Mpad, int M, const double* d,
                         double* A, double* b, cudaStream_t stream) {
    dim3 grid((unsigned)((M + 255) / 256), (unsigned)M);
    assemble_kernel<float, float><<<grid, 256, 0, stream>>>(Gpart, bpart, dpart, colexp, nsplit, tile, Mpad,
                                                     M, d, A, b);
}

void launch_assemble_scaled(const float2* Gpart, const double* bpart, const int* colexp, int nsplit,
                            int tile, int Mpad, int M, const double* d, double* A, double* b,
                            cudaStream_t stream) {
    dim3 grid((unsigned)((M + 255) / 256), (unsigned)M);
    assemble_kernel<float2, double><<<grid, 256, 0, stream>>>(Gpart, bpart, nullptr, colexp, nsplit, tile,
                                                              Mpad, M, d, A, b);
}

void launch_noise_diag(const GpShape& s, const double* loglam, double sigma2, double* d,
                       cudaStream_t stream) {
    noise_diag_kernel<<<(s.M + 255) / 256, 256, 0, stream>>>(s, loglam, log(sigma2), d);
}
