// gp_factor.cu -- factorisation of A = L L^T and the inverse W = L^{-1}.
//
// Sec. 3 of the paper inverts Lambda-bar with an LU factorisation; A =
// sigma^2 Lambda-bar is symmetric positive definite, so it is factored by
// Cholesky. On GB300 the float64 pipe retires about 2 FMAs per clock per SM,
// so an M x M factorisation only runs at speed when every SM works on it and
// no time is lost between launches. Both kernels here are therefore single
// persistent cooperative launches (one CTA per SM) that walk the block
// algorithm step by step, separated by grid barriers whose waits are bounded
// (GP_ETIMEOUT after GP_WAIT_NS; nothing can hang):
//
//   Cholesky (float64, right-looking, 32-column panels, look-ahead), per step k:
//     B  one warp per row below the factored diagonal block solves
//        x L_kk^T = a (lane j owns x_j);
//     C  16 x 16 tiles of the trailing lower triangle subtract L_ik L_jk^T;
//        CTA 0 updates the next diagonal block's tiles first and factors it
//        (32 x 32, in shared memory) while the other CTAs finish C.
//   A non-positive or NaN pivot sets GP_ENOTPD (detail = column); every CTA
//   sees it after the next barrier and returns.
//
//   W = L^{-1} (right-looking block forward substitution on R = I, 32-row
//   blocks), in float32 or float64 arithmetic:
//     0  invert every 32 x 32 diagonal block (D_I = L_II^{-1}); R = I;
//     for each block row I:  1  W_IJ = D_I R_IJ        (J <= I)
//                            2  R_KJ -= L_KI W_IJ      (K > I, J <= I)
//   The mixed-precision fit uses float32 here: W feeds the bf16 hi/lo
//   variance contraction, and as the preconditioner of c = A^{-1} b its
//   error is removed by the float64 iterative refinement.
#include "gp_kernels.cuh"
#include "gp_tc.cuh"

#include <math.h>

namespace {

constexpr int CB = 32;  // Cholesky panel width
constexpr int UT = 16;  // Cholesky trailing-update tile
constexpr int IB = 32;  // inverse block size
constexpr int NT = 256; // threads per CTA

struct GridBar {
    unsigned int count;
    unsigned int gen;
};

// Bounded grid-wide barrier for a cooperative launch. Returns false (and
// sets GP_ETIMEOUT) if the other CTAs do not arrive within GP_WAIT_NS.
__device__ bool grid_sync(GridBar* gb, GpStatus* st) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_fail = 0;
        unsigned int g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&gb->gen) : "memory");
        __threadfence();
        const unsigned int arrived = atomicAdd(&gb->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            gb->count = 0u;
            __threadfence();
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gb->gen) : "memory");
        } else {
            const uint64_t t0 = globaltimer_ns();
            uint32_t it = 0;
            while (true) {
                unsigned int cur;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&gb->gen) : "memory");
                if (cur != g) break;
                if ((++it & 1023u) == 0 && globaltimer_ns() - t0 > GP_WAIT_NS) {
                    gp_set_status(st, GP_ETIMEOUT, 100);
                    s_fail = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_fail == 0;
}

__device__ __forceinline__ int status_code(const GpStatus* st) { return *(volatile const int*)&st->code; }

// ---------------------------------------------------------------- Cholesky

// Factor the w x w diagonal block at (kb, kb) in shared memory (one CTA).
__device__ void chol_diag_block(double* __restrict__ L, int M, int kb, int w, GpStatus* st,
                                double (*a)[CB + 1]) {
    __shared__ int bad;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < w * w; e += NT) {
        const int i = e / w, j = e % w;
        a[i][j] = (j <= i) ? L[(int64_t)(kb + i) * M + kb + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (tid == 0) {
            const double piv = a[j][j];
            if (!(piv > 0.0) || !isfinite(piv)) {
                bad = 1;
                gp_set_status(st, GP_ENOTPD, kb + j);
            } else {
                a[j][j] = sqrt(piv);
            }
        }
        __syncthreads();
        if (bad) break;
        const double djj = a[j][j];
        for (int i = j + 1 + tid; i < w; i += NT) a[i][j] /= djj;
        __syncthreads();
        const int r = w - j - 1;
        for (int e = tid; e < r * r; e += NT) {
            const int i = j + 1 + e / r, l = j + 1 + e % r;
            if (l <= i) a[i][l] -= a[i][j] * a[l][j];
        }
        __syncthreads();
    }
    if (!bad)
        for (int e = tid; e < w * w; e += NT) {
            const int i = e / w, j = e % w;
            if (j <= i) L[(int64_t)(kb + i) * M + kb + j] = a[i][j];
        }
    __syncthreads();
}

// L[r0.., c0..] -= L[r0.., kb..kb+w) L[c0.., kb..kb+w)^T on one 16 x 16 lower tile.
__device__ void chol_update_tile(double* __restrict__ L, int M, int kb, int w, int r0, int c0,
                                 double (*ti)[CB + 1], double (*tj)[CB + 1]) {
    const int tid = threadIdx.x;
    for (int e = tid; e < UT * w; e += NT) {
        const int r = e / w, l = e % w;
        ti[r][l] = (r0 + r < M) ? L[(int64_t)(r0 + r) * M + kb + l] : 0.0;
        tj[r][l] = (c0 + r < M) ? L[(int64_t)(c0 + r) * M + kb + l] : 0.0;
    }
    __syncthreads();
    const int ty = tid / UT, tx = tid % UT;
    double s = 0.0;
    for (int l = 0; l < w; ++l) s = fma(ti[ty][l], tj[tx][l], s);
    const int i = r0 + ty, j = c0 + tx;
    if (i < M && j <= i) L[(int64_t)i * M + j] -= s;
    __syncthreads();
}

// Right-looking Cholesky with look-ahead: while the other CTAs apply step
// k's trailing update, CTA 0 updates the tiles of the next diagonal block
// first and factors it, so each step costs two grid barriers.
__global__ void __launch_bounds__(NT) chol_coop_kernel(double* __restrict__ L, int M, GpStatus* st,
                                                       GridBar* gb) {
    __shared__ double a[CB][CB + 1];
    __shared__ double ti[UT][CB + 1];
    __shared__ double tj[UT][CB + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = (M + CB - 1) / CB;
    const int G = gridDim.x;
    if (blockIdx.x == 0) chol_diag_block(L, M, 0, min(CB, M), st, a);
    if (!grid_sync(gb, st)) return;
    if (status_code(st) != 0) return;
    for (int k = 0; k < nb; ++k) {
        const int kb = k * CB, w = min(CB, M - kb);
        const int rest = M - kb - w;
        if (rest == 0) break;
        // ---- B: panel rows, one warp per row
        const int rows_here = G * (NT / 32);
        if ((int)blockIdx.x * (NT / 32) < rest) {
            for (int e = tid; e < w * w; e += NT) {
                const int i = e / w, j = e % w;
                a[i][j] = (j <= i) ? L[(int64_t)(kb + i) * M + kb + j] : 0.0;
            }
            __syncthreads();
            for (int rr = blockIdx.x * (NT / 32) + warp; rr < rest; rr += rows_here) {
                const int i = kb + w + rr;
                double* row = L + (int64_t)i * M + kb;
                const double av = lane < w ? row[lane] : 0.0;
                double acc = 0.0, x = 0.0;
                for (int l = 0; l < w; ++l) {
                    if (lane == l) x = (av - acc) / a[l][l];
                    const double xl = __shfl_sync(0xffffffffu, x, l);
                    if (lane > l && lane < w) acc = fma(xl, a[lane][l], acc);
                }
                if (lane < w) row[lane] = x;
            }
            __syncthreads();
        }
        if (!grid_sync(gb, st)) return;
        // ---- C: trailing update; CTA 0 takes the next diagonal block's tiles and factors it
        const int ntr = (rest + UT - 1) / UT;
        const int ntiles = ntr * (ntr + 1) / 2;
        const int wn = min(CB, rest);              // width of the next diagonal block
        const int nd = (wn + UT - 1) / UT;
        const int ndiag = nd * (nd + 1) / 2;       // its tiles come first in tile order
        if (blockIdx.x == 0) {
            for (int t = 0; t < ndiag; ++t) {
                int I, J;
                tri_pair(t, &I, &J);
                chol_update_tile(L, M, kb, w, kb + w + I * UT, kb + w + J * UT, ti, tj);
            }
            chol_diag_block(L, M, kb + w, wn, st, a);
        }
        const int first = (G > 1) ? (int)blockIdx.x - 1 : 0;
        const int stride = (G > 1) ? G - 1 : 1;
        if (G == 1 || blockIdx.x > 0)
            for (int t = ndiag + first; t < ntiles; t += stride) {
                int I, J;
                tri_pair(t, &I, &J);
                chol_update_tile(L, M, kb, w, kb + w + I * UT, kb + w + J * UT, ti, tj);
            }
        if (!grid_sync(gb, st)) return;
        if (status_code(st) != 0) return;
    }
    // upper triangle = 0
    const int64_t total = (int64_t)M * M;
    for (int64_t e = (int64_t)blockIdx.x * NT + tid; e < total; e += (int64_t)G * NT) {
        const int i = (int)(e / M), j = (int)(e % M);
        if (j > i) L[e] = 0.0;
    }
}

// ---------------------------------------------------------------- W = L^{-1}

template <typename T>
__device__ __forceinline__ T tload(const double* p) { return (T)(*p); }

template <typename T>
__global__ void __launch_bounds__(NT) trinv_coop_kernel(const double* __restrict__ L,
                                                        double* __restrict__ W, int M,
                                                        T* __restrict__ R, T* __restrict__ Dinv,
                                                        GpStatus* st, GridBar* gb) {
    __shared__ T sa[IB][IB + 1];
    __shared__ T sb[IB][IB + 1];
    const int tid = threadIdx.x;
    const int nb = (M + IB - 1) / IB;
    const int ty = tid / IB, tx = tid % IB;   // 8 x 32 threads: rows ty + 8q
    // ---- 0: diagonal block inverses, R = I (lower), W = 0 above the diagonal
    for (int I = blockIdx.x; I < nb; I += gridDim.x) {
        const int r0 = I * IB, wI = min(IB, M - r0);
        for (int e = tid; e < IB * IB; e += NT) {
            const int i = e / IB, j = e % IB;
            sa[i][j] = (i < wI && j <= i) ? tload<T>(L + (int64_t)(r0 + i) * M + r0 + j) : T(0);
            sb[i][j] = T(0);
        }
        __syncthreads();
        if (tid < wI) {  // column j of L_II^{-1} by forward substitution
            const int j = tid;
            sb[j][j] = T(1) / sa[j][j];
            for (int i = j + 1; i < wI; ++i) {
                T s = T(0);
                for (int k = j; k < i; ++k) s += sa[i][k] * sb[k][j];
                sb[i][j] = -s / sa[i][i];
            }
        }
        __syncthreads();
        for (int e = tid; e < IB * IB; e += NT) Dinv[(int64_t)I * IB * IB + e] = sb[e / IB][e % IB];
        __syncthreads();
    }
    const int64_t total = (int64_t)M * M;
    for (int64_t e = (int64_t)blockIdx.x * NT + tid; e < total; e += (int64_t)gridDim.x * NT) {
        const int i = (int)(e / M), j = (int)(e % M);
        R[e] = (i == j) ? T(1) : T(0);  // whole matrix: diagonal blocks are read in full
        if (j > i) W[e] = 0.0;
    }
    if (!grid_sync(gb, st)) return;
    for (int I = 0; I < nb; ++I) {
        const int r0 = I * IB, wI = min(IB, M - r0);
        // ---- 1: W_IJ = D_I R_IJ, J <= I
        for (int J = blockIdx.x; J <= I; J += gridDim.x) {
            const int c0 = J * IB, wJ = min(IB, M - c0);
            for (int e = tid; e < IB * IB; e += NT) {
                const int i = e / IB, j = e % IB;
                sa[i][j] = Dinv[(int64_t)I * IB * IB + e];
                sb[i][j] = (i < wI && j < wJ) ? R[(int64_t)(r0 + i) * M + c0 + j] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < IB / 8; ++q) {
                const int i = ty + 8 * q;
                T s = T(0);
                for (int k = 0; k <= i; ++k) s += sa[i][k] * sb[k][tx];
                if (i < wI && tx < wJ) W[(int64_t)(r0 + i) * M + c0 + tx] = (double)s;
            }
            __syncthreads();
        }
        if (!grid_sync(gb, st)) return;
        // ---- 2: R_KJ -= L_KI W_IJ, K > I, J <= I
        const int nK = nb - I - 1, nJ = I + 1;
        for (int t = blockIdx.x; t < nK * nJ; t += gridDim.x) {
            const int K = I + 1 + t / nJ, J = t % nJ;
            const int k0 = K * IB, wK = min(IB, M - k0);
            const int c0 = J * IB, wJ = min(IB, M - c0);
            for (int e = tid; e < IB * IB; e += NT) {
                const int i = e / IB, j = e % IB;
                sa[i][j] = (i < wK && j < wI) ? tload<T>(L + (int64_t)(k0 + i) * M + r0 + j) : T(0);
                sb[i][j] = (i < wI && j < wJ) ? (T)W[(int64_t)(r0 + i) * M + c0 + j] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < IB / 8; ++q) {
                const int i = ty + 8 * q;
                T s = T(0);
#pragma unroll 8
                for (int k = 0; k < IB; ++k) s += sa[i][k] * sb[k][tx];
                if (i < wK && tx < wJ) R[(int64_t)(k0 + i) * M + c0 + tx] -= s;
            }
            __syncthreads();
        }
        if (!grid_sync(gb, st)) return;
    }
}

int coop_grid(const void* kern, int dev) {
    int sms = 1, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0);
    if (occ < 1) occ = 1;
    return sms * (occ < 2 ? occ : 1);
}

}  // namespace

size_t factor_work_bytes(int M, bool fp32_inverse) {
    const size_t nb = (M + IB - 1) / IB;
    const size_t el = fp32_inverse ? sizeof(float) : sizeof(double);
    return 256 + el * ((size_t)M * M + nb * IB * IB);
}

cudaError_t launch_cholesky(double* L, int M, GpStatus* st, void* work, cudaStream_t stream) {
    int dev = 0;
    cudaGetDevice(&dev);
    GridBar* gb = (GridBar*)work;
    cudaMemsetAsync(gb, 0, sizeof(GridBar), stream);
    dim3 grid((unsigned)coop_grid((const void*)chol_coop_kernel, dev)), block(NT);
    void* args[] = {&L, &M, &st, &gb};
    gp_note_launches(1);
    return cudaLaunchCooperativeKernel((const void*)chol_coop_kernel, grid, block, args, 0, stream);
}

cudaError_t launch_tri_inverse(const double* L, double* W, int M, bool fp32, GpStatus* st, void* work,
                               cudaStream_t stream) {
    int dev = 0;
    cudaGetDevice(&dev);
    GridBar* gb = (GridBar*)work;
    cudaMemsetAsync(gb, 0, sizeof(GridBar), stream);
    char* base = (char*)work + 256;
    const size_t nb = (M + IB - 1) / IB;
    gp_note_launches(1);
    if (fp32) {
        float* R = (float*)base;
        float* D = R + (size_t)M * M;
        const void* k = (const void*)trinv_coop_kernel<float>;
        dim3 grid((unsigned)coop_grid(k, dev)), block(NT);
        void* args[] = {(void*)&L, &W, &M, &R, &D, &st, &gb};
        (void)nb;
        return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
    }
    double* R = (double*)base;
    double* D = R + (size_t)M * M;
    const void* k = (const void*)trinv_coop_kernel<double>;
    dim3 grid((unsigned)coop_grid(k, dev)), block(NT);
    void* args[] = {(void*)&L, &W, &M, &R, &D, &st, &gb};
    return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
}
