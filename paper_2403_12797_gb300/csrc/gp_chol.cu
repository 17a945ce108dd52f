// gp_chol.cu -- float64 factorisation of A and the solves of the fit.
//
// Sec. 3 of the paper inverts Lambda-bar with an LU factorisation; A =
// sigma^2 Lambda-bar is symmetric positive definite, so it is factored here
// as A = L L^T (right-looking blocked Cholesky, 64-column panels). The
// fit then forms W = L^{-1} (blocked triangular inverse): it serves both the
// predictive variance, var = sigma^2 |W phi_*|^2 (diagonal of Eq. 12), and
// the solve c = A^{-1} b = W^T W b (Eq. 11), which is refined against the
// float64 residual b - A c.
//
// A non-positive (or NaN) pivot sets GP_ENOTPD with the column index in the
// status word; every later kernel of the chain sees the status and returns,
// so nothing traps.
#include "gp_kernels.cuh"

#include <math.h>

namespace {

constexpr int NB = CHOL_NB;

// ---------------------------------------------------------------- Cholesky

__global__ void __launch_bounds__(256) chol_diag_kernel(double* __restrict__ L, int M, int kb, int w,
                                                        GpStatus* st) {
    __shared__ double a[NB][NB + 1];
    __shared__ int bad;
    if (st->code != 0) return;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < w * w; e += blockDim.x) {
        int i = e / w, j = e % w;
        a[i][j] = (j <= i) ? L[(int64_t)(kb + i) * M + kb + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (tid == 0) {
            double piv = a[j][j];
            if (!(piv > 0.0) || !isfinite(piv)) {
                bad = 1;
                gp_set_status(st, GP_ENOTPD, kb + j);
            } else {
                a[j][j] = sqrt(piv);
            }
        }
        __syncthreads();
        if (bad) return;
        const double djj = a[j][j];
        for (int i = j + 1 + tid; i < w; i += blockDim.x) a[i][j] /= djj;
        __syncthreads();
        const int r = w - j - 1;
        for (int e = tid; e < r * r; e += blockDim.x) {
            int i = j + 1 + e / r, l = j + 1 + e % r;
            if (l <= i) a[i][l] -= a[i][j] * a[l][j];
        }
        __syncthreads();
    }
    for (int e = tid; e < w * w; e += blockDim.x) {
        int i = e / w, j = e % w;
        if (j <= i) L[(int64_t)(kb + i) * M + kb + j] = a[i][j];
    }
}

// rows below the diagonal block: X = A21 L11^{-T}
__global__ void __launch_bounds__(64) chol_panel_kernel(double* __restrict__ L, int M, int kb, int w,
                                                        GpStatus* st) {
    extern __shared__ double shp[];
    double(*l11)[NB + 1] = (double(*)[NB + 1])shp;
    double(*x)[NB + 1] = (double(*)[NB + 1])(shp + NB * (NB + 1));
    if (st->code != 0) return;
    const int tid = threadIdx.x;
    const int row0 = kb + w + blockIdx.x * NB;
    for (int e = tid; e < w * w; e += blockDim.x) {
        int i = e / w, j = e % w;
        l11[i][j] = (j <= i) ? L[(int64_t)(kb + i) * M + kb + j] : 0.0;
    }
    for (int e = tid; e < NB * w; e += blockDim.x) {
        int r = e / w, j = e % w;
        x[r][j] = (row0 + r < M) ? L[(int64_t)(row0 + r) * M + kb + j] : 0.0;
    }
    __syncthreads();
    if (row0 + tid < M) {
        for (int j = 0; j < w; ++j) {
            double s = x[tid][j];
            for (int l = 0; l < j; ++l) s -= x[tid][l] * l11[j][l];
            x[tid][j] = s / l11[j][j];
        }
    }
    __syncthreads();
    for (int e = tid; e < NB * w; e += blockDim.x) {
        int r = e / w, j = e % w;
        if (row0 + r < M) L[(int64_t)(row0 + r) * M + kb + j] = x[r][j];
    }
}

// trailing update A22 -= L21 L21^T on the lower 64 x 64 tiles
__global__ void __launch_bounds__(256) chol_update_kernel(double* __restrict__ L, int M, int kb, int w,
                                                          GpStatus* st) {
    __shared__ double li[32][NB + 1];
    __shared__ double lj[32][NB + 1];
    if (st->code != 0) return;
    const int t0 = kb + w;
    int I, J;
    tri_pair(blockIdx.x, &I, &J);
    const int rI = t0 + I * NB, rJ = t0 + J * NB;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double acc[4][4] = {};
    for (int kc = 0; kc < w; kc += 32) {
        const int kw = min(32, w - kc);
        for (int e = tid; e < NB * 32; e += blockDim.x) {
            int r = e / 32, k = e % 32;
            double vi = 0.0, vj = 0.0;
            if (k < kw) {
                if (rI + r < M) vi = L[(int64_t)(rI + r) * M + kb + kc + k];
                if (rJ + r < M) vj = L[(int64_t)(rJ + r) * M + kb + kc + k];
            }
            li[k][r] = vi;
            lj[k][r] = vj;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = li[k][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = lj[k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int i = rI + ty + 16 * a, l = rJ + tx + 16 * b;
            if (i < M && l < M && l <= i) L[(int64_t)i * M + l] -= acc[a][b];
        }
}

__global__ void zero_upper_kernel(double* __restrict__ L, int M) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y;
    if (col < M && col > row) L[(int64_t)row * M + col] = 0.0;
}

// ---------------------------------------------------------------- triangular inverse

// CTA (I, J = blockIdx.x <= I) computes the block W_IJ of W = L^{-1}:
//   W_II = L_II^{-1},  W_IJ = -L_II^{-1} sum_{K=J}^{I-1} L_IK W_KJ  (J < I).
__global__ void __launch_bounds__(256) trinv_row_kernel(const double* __restrict__ L,
                                                        double* __restrict__ W, int M, int I,
                                                        GpStatus* st) {
    extern __shared__ double sh[];
    double(*lb)[NB + 1] = (double(*)[NB + 1])sh;                   // L_II
    double(*dinv)[NB + 1] = (double(*)[NB + 1])(sh + NB * (NB + 1));  // L_II^{-1}
    double(*ta)[NB + 1] = (double(*)[NB + 1])(sh + 2 * NB * (NB + 1));
    double(*tb)[NB + 1] = (double(*)[NB + 1])(sh + 3 * NB * (NB + 1));
    if (st->code != 0) return;
    const int J = blockIdx.x;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int r0 = I * NB;
    const int wI = min(NB, M - r0);
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        lb[i][j] = (i < wI && j <= i) ? L[(int64_t)(r0 + i) * M + r0 + j] : 0.0;
        dinv[i][j] = 0.0;
    }
    __syncthreads();
    // column j of L_II^{-1} by forward substitution (one thread per column)
    if (tid < wI) {
        const int j = tid;
        dinv[j][j] = 1.0 / lb[j][j];
        for (int i = j + 1; i < wI; ++i) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s += lb[i][k] * dinv[k][j];
            dinv[i][j] = -s / lb[i][i];
        }
    }
    __syncthreads();
    const int c0 = J * NB;
    const int wJ = min(NB, M - c0);
    if (J == I) {
        for (int e = tid; e < NB * NB; e += blockDim.x) {
            int i = e / NB, j = e % NB;
            if (i < wI && j < wJ) W[(int64_t)(r0 + i) * M + c0 + j] = dinv[i][j];
        }
        return;
    }
    // T = sum_K L_IK W_KJ
    double acc[4][4] = {};
    for (int K = J; K < I; ++K) {
        const int k0 = K * NB;
        for (int e = tid; e < NB * NB; e += blockDim.x) {
            int i = e / NB, k = e % NB;
            ta[k][i] = (i < wI) ? L[(int64_t)(r0 + i) * M + k0 + k] : 0.0;  // L_IK^T
            tb[i][k] = (k < wJ) ? W[(int64_t)(k0 + i) * M + c0 + k] : 0.0;  // W_KJ
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < NB; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = ta[k][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = tb[k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    // W_IJ = -dinv * T
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) tb[ty + 16 * a][tx + 16 * b] = acc[a][b];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = ty + 16 * a, j = tx + 16 * b;
            double s = 0.0;
            for (int k = 0; k <= i; ++k) s += dinv[i][k] * tb[k][j];
            if (i < wI && j < wJ) W[(int64_t)(r0 + i) * M + c0 + j] = -s;
        }
}

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

constexpr int LT_CHUNK = 128;

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

cudaError_t launch_cholesky(double* L, int M, GpStatus* st, cudaStream_t stream) {
    const size_t psmem = 2 * NB * (NB + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(chol_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)psmem);
    if (e != cudaSuccess) return e;
    for (int kb = 0; kb < M; kb += NB) {
        const int w = min(NB, M - kb);
        chol_diag_kernel<<<1, 256, 0, stream>>>(L, M, kb, w, st);
        gp_note_launches(1);
        const int rest = M - kb - w;
        if (rest > 0) {
            chol_panel_kernel<<<(rest + NB - 1) / NB, 64, psmem, stream>>>(L, M, kb, w, st);
            const int T = (rest + NB - 1) / NB;
            chol_update_kernel<<<T * (T + 1) / 2, 256, 0, stream>>>(L, M, kb, w, st);
            gp_note_launches(2);
        }
    }
    dim3 g((M + 255) / 256, M);
    zero_upper_kernel<<<g, 256, 0, stream>>>(L, M);
    gp_note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tri_inverse(const double* L, double* W, int M, GpStatus* st,
                               cudaStream_t stream) {
    const size_t smem = 4 * NB * (NB + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(trinv_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(W, 0, (size_t)M * M * sizeof(double), stream);
    const int nb = (M + NB - 1) / NB;
    for (int I = 0; I < nb; ++I) trinv_row_kernel<<<I + 1, 256, smem, stream>>>(L, W, M, I, st);
    gp_note_launches(nb);
    return cudaGetLastError();
}

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
