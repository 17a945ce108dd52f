// gp_chol.cu -- the solve c = A^{-1} b of the fit (Eq. 11 in the M x M form).
//
// With W = L^{-1} from gp_factor.cu, c = W^T (W b); it is then refined
// against the float64 residual r = b - A c: c += W^T W r. In the mixed mode
// W is computed in float32, and the refinement steps bring c to float64
// accuracy. Every kernel returns early once the status word holds an error
// (e.g. GP_ENOTPD from the factorisation).
#include "gp_kernels.cuh"

#include <math.h>

namespace {


// ---------------------------------------------------------------- matrix-vector products

// y[i] = sum_{j < lim(i)} A[i][j] x[j]  (lim = i+1 if lower, else M); if bsub: y = bsub - y
__global__ void gemv_rows_kernel(const double* __restrict__ A, int M, const double* __restrict__ x,
                                 double* __restrict__ y, int lower, const double* __restrict__ bsub,
                                 const GpStatus* st) {
    if (st->code != 0) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= M) return;
    const int lim = lower ? warp + 1 : M;
    const double* row = A + (int64_t)warp * M;
    double s = 0.0;
    for (int j = lane; j < lim; j += 32) s += row[j] * x[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[warp] = bsub ? bsub[warp] - s : s;
}

// part[ch][j] = sum_{i in chunk ch, i >= j} W[i][j] x[i]
__global__ void gemv_lowerT_part_kernel(const double* __restrict__ W, int M,
                                        const double* __restrict__ x, double* __restrict__ part,
                                        int rows_per_chunk, const GpStatus* st) {
    if (st->code != 0) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    if (j >= M) return;
    int i0 = ch * rows_per_chunk;
    const int i1 = min(M, i0 + rows_per_chunk);
    if (i0 < j) i0 = j;
    double s = 0.0;
    for (int i = i0; i < i1; ++i) s += W[(int64_t)i * M + j] * x[i];
    part[(int64_t)ch * M + j] = s;
}

// y[j] = sum_ch part[ch][j]  (+ y[j] if accumulate)
__global__ void sum_parts_kernel(const double* __restrict__ part, int nch, int M,
                                 double* __restrict__ y, int accumulate, const GpStatus* st) {
    if (st->code != 0) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(int64_t)c * M + j];
    y[j] = accumulate ? y[j] + s : s;
}

constexpr int LT_CHUNK = 32;

// y = W^T (W v)  using tmp (M) and part (ceil(M/LT_CHUNK) * M)
void wtw_apply(const double* W, int M, const double* v, double* tmp, double* part, double* y,
               int accumulate, const GpStatus* st, cudaStream_t stream) {
    gemv_rows_kernel<<<(M * 32 + 255) / 256, 256, 0, stream>>>(W, M, v, tmp, 1, nullptr, st);
    const int nch = (M + LT_CHUNK - 1) / LT_CHUNK;
    dim3 g((M + 127) / 128, nch);
    gemv_lowerT_part_kernel<<<g, 128, 0, stream>>>(W, M, tmp, part, LT_CHUNK, st);
    sum_parts_kernel<<<(M + 255) / 256, 256, 0, stream>>>(part, nch, M, y, accumulate, st);
}

}  // namespace

cudaError_t launch_solve_refine(const double* A, const double* W, const double* b, double* c,
                                double* work, int M, int refine, const GpStatus* st,
                                cudaStream_t stream) {
    // work: tmp (M) | r (M) | part (ceil(M/LT_CHUNK) * M)
    double* tmp = work;
    double* r = work + M;
    double* part = work + 2 * (int64_t)M;
    wtw_apply(W, M, b, tmp, part, c, 0, st, stream);
    gp_note_launches(3 + 4 * refine);
    for (int it = 0; it < refine; ++it) {
        gemv_rows_kernel<<<(M * 32 + 255) / 256, 256, 0, stream>>>(A, M, c, r, 0, b, st);
        wtw_apply(W, M, r, tmp, part, c, 1, st, stream);
    }
    return cudaGetLastError();
}

size_t solve_refine_work_elems(int M) {
    const int nch = (M + LT_CHUNK - 1) / LT_CHUNK;
    return 2 * (size_t)M + (size_t)nch * M;
}
