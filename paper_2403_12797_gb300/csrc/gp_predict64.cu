// gp_predict64.cu -- float64 predictive mean and variance (CUDA cores).
//
// mean_i = phi(x*_i)^T c                         (Eq. 11 in the M x M form)
// var_i  = sigma^2 |W phi(x*_i)|^2, W = L^{-1}   (diagonal of Eq. 12)
//
// CTA (test tile of 64 points, column tile kt of 64): Z = Phi_* W^T restricted
// to those 64 columns, with W lower triangular so only m <= k contributes.
// Phi_* is regenerated in shared memory from the test points' eigenfunction
// tables. Each CTA writes the partial sum of squares of its Z tile and the
// partial mean over its 64 values of m; a second kernel adds the partials
// in column-tile order (deterministic). With zout given, the Z tile itself is
// also stored (row-major, zld = 64 x column tiles doubles per test point) for
// the covariance block of Eq. 12 (gp_cov.cu).
#include "gp_kernels.cuh"

namespace {

constexpr int TT = PRED64_TT;
constexpr int TK = PRED64_TK;
constexpr int CK = 16;  // m columns per chunk

__global__ void __launch_bounds__(256) predict64_kernel(GpShape s, const double* __restrict__ tab,
                                                        const double* __restrict__ W,
                                                        const double* __restrict__ cvec, int maxrows,
                                                        double* __restrict__ part, double* __restrict__ zout) {
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ TileWindow wv;
    double* win = (double*)smem_raw;                       // maxrows x TT
    double* phis = win + (size_t)maxrows * TT;             // TT x (CK+1)
    double* wt = phis + TT * (CK + 1);                     // CK x TK
    int* tr = (int*)(wt + CK * TK);                        // maxrows
    unsigned short* cr = (unsigned short*)(tr + maxrows);  // CK x p

    const int tt = blockIdx.x, kt = blockIdx.y;
    const int nkt = gridDim.y;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t t0 = (int64_t)tt * TT;
    const int k0 = kt * TK;
    const int mend = min(s.M, k0 + TK);

    double acc[4][4] = {};
    double macc = 0.0;
    for (int m0 = 0; m0 < mend; m0 += CK) {
        if (tid == 0) tile_window(s, m0, CK, &wv);
        __syncthreads();
        for (int r = tid; r < wv.nrows; r += blockDim.x) tr[r] = window_table_row(s, wv, r);
        for (int e = tid; e < CK * s.p; e += blockDim.x) {
            int c = e / s.p, j = e % s.p;
            cr[e] = (unsigned short)(m0 + c < s.M ? window_row(s, wv, j, m0 + c) : 0);
        }
        __syncthreads();
        for (int e = tid; e < wv.nrows * TT; e += blockDim.x) {
            int r = e / TT, t = e % TT;
            win[e] = __ldg(tab + (int64_t)tr[r] * s.Npad + t0 + t);
        }
        for (int e = tid; e < CK * TK; e += blockDim.x) {
            int k = e / CK, c = e % CK;
            int kk = k0 + k, mm = m0 + c;
            wt[c * TK + k] = (kk < s.M && mm < s.M) ? W[(int64_t)kk * s.M + mm] : 0.0;
        }
        __syncthreads();
        for (int e = tid; e < TT * CK; e += blockDim.x) {
            int t = e % TT, c = e / TT;
            double v = 0.0;
            if (m0 + c < s.M) {
                v = 1.0;
                for (int j = 0; j < s.p; ++j) v *= win[cr[c * s.p + j] * TT + t];
            }
            phis[t * (CK + 1) + c] = v;
        }
        __syncthreads();
        if (m0 >= k0 && tid < TT) {
            for (int c = 0; c < CK && m0 + c < s.M; ++c) macc += phis[tid * (CK + 1) + c] * cvec[m0 + c];
        }
#pragma unroll
        for (int c = 0; c < CK; ++c) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = phis[(ty + 16 * a) * (CK + 1) + c];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = wt[c * TK + tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    if (zout != nullptr) {
        const int64_t zld = (int64_t)nkt * TK;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) zout[(t0 + ty + 16 * a) * zld + k0 + tx + 16 * b] = acc[a][b];
    }
    // partial sums of squares per test point
    double* pvar = part;                               // [nkt][Npad]
    double* pmean = part + (int64_t)nkt * s.Npad;      // [nkt][Npad]
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        double q = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) q += acc[a][b] * acc[a][b];
        for (int o = 8; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (tx == 0) pvar[(int64_t)kt * s.Npad + t0 + ty + 16 * a] = q;
    }
    if (tid < TT) pmean[(int64_t)kt * s.Npad + t0 + tid] = macc;
}

__global__ void predict64_reduce_kernel(const double* __restrict__ part, int nkt, int64_t Npad,
                                        int64_t Ns, double sigma2, double* __restrict__ mean,
                                        double* __restrict__ var) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ns) return;
    double sv = 0.0, sm = 0.0;
    for (int k = 0; k < nkt; ++k) {
        sv += part[(int64_t)k * Npad + t];
        sm += part[(int64_t)(nkt + k) * Npad + t];
    }
    mean[t] = sm;
    if (var) var[t] = sigma2 * sv;
}

}  // namespace

size_t predict64_part_elems(int64_t Npad, int M) {
    const int nkt = (M + TK - 1) / TK;
    return 2 * (size_t)nkt * (size_t)Npad;
}

cudaError_t launch_predict64(const GpShape& s, const double* tab, const double* W, const double* c,
                             double sigma2, double* part, double* mean, double* var,
                             cudaStream_t stream, double* zout) {
    const int maxrows = gp_max_window_rows(s, CK);
    const size_t smem = sizeof(double) * ((size_t)maxrows * TT + TT * (CK + 1) + CK * TK) +
                        sizeof(int) * maxrows + sizeof(unsigned short) * CK * s.p + 16;
    if (smem > 48 * 1024) {
        cudaError_t e = gp_allow_max_smem((const void*)predict64_kernel);
        if (e != cudaSuccess) return e;
    }
    const int nkt = (s.M + TK - 1) / TK;
    dim3 grid((unsigned)(s.Npad / TT), (unsigned)nkt);
    predict64_kernel<<<grid, 256, smem, stream>>>(s, tab, W, c, maxrows, part, zout);
    predict64_reduce_kernel<<<(unsigned)((s.N + 255) / 256), 256, 0, stream>>>(part, nkt, s.Npad, s.N,
                                                                            sigma2, mean, var);
    return cudaGetLastError();
}

size_t predict64_z_elems(int64_t Npad, int M) {
    return (size_t)Npad * (size_t)(((M + TK - 1) / TK) * TK);
}
