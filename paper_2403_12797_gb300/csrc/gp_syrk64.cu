// gp_syrk64.cu -- float64 fused Phi generation + Gram contraction (CUDA cores).
//
// Computes the two products of Sec. 2.2 that touch the N training rows,
// G = Phi^T Phi and b = Phi^T y (Lambda-bar = Lambda^{-1} + Phi^T Phi / sigma^2,
// and the Phi^T y of W in Eq. 11), in float64. Phi (Eq. 19) is generated
// chunk by chunk in shared memory from the per-dimension eigenfunction
// tables and never written to global memory.
//
// Grid: x = lower-triangular 64 x 64 tile pair (I >= J) of G, y = split of
// the N rows. Each CTA writes its own partial tile; gp_assemble.cu sums the
// splits in a fixed order, so the result is deterministic.
#include "gp_kernels.cuh"

namespace {

constexpr int TM = SYRK64_TM;
constexpr int BK = SYRK64_BK;

struct Smem64 {
    double* winI;
    double* winJ;
    double* phiI;
    double* phiJ;
    double* yv;
    int* trI;
    int* trJ;
    unsigned short* crI;
    unsigned short* crJ;
};

__host__ __device__ inline size_t smem64_layout(int maxrows, int p, char* base, Smem64* L) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) & ~size_t(15);
        return o;
    };
    size_t oWI = take(sizeof(double) * maxrows * BK);
    size_t oWJ = take(sizeof(double) * maxrows * BK);
    size_t oPI = take(sizeof(double) * BK * TM);
    size_t oPJ = take(sizeof(double) * BK * TM);
    size_t oY = take(sizeof(double) * BK);
    size_t oTI = take(sizeof(int) * maxrows);
    size_t oTJ = take(sizeof(int) * maxrows);
    size_t oCI = take(sizeof(unsigned short) * TM * p);
    size_t oCJ = take(sizeof(unsigned short) * TM * p);
    if (L) {
        L->winI = (double*)(base + oWI);
        L->winJ = (double*)(base + oWJ);
        L->phiI = (double*)(base + oPI);
        L->phiJ = (double*)(base + oPJ);
        L->yv = (double*)(base + oY);
        L->trI = (int*)(base + oTI);
        L->trJ = (int*)(base + oTJ);
        L->crI = (unsigned short*)(base + oCI);
        L->crJ = (unsigned short*)(base + oCJ);
    }
    return off;
}

__device__ __forceinline__ void setup_tile(const GpShape& s, const TileWindow& w, int m0, int* tr,
                           unsigned short* cr) {
    for (int r = threadIdx.x; r < w.nrows; r += blockDim.x) tr[r] = window_table_row(s, w, r);
    for (int e = threadIdx.x; e < TM * s.p; e += blockDim.x) {
        int c = e / s.p, j = e % s.p;
        int m = m0 + c;
        cr[e] = (unsigned short)(m < s.M ? window_row(s, w, j, m) : 0);
    }
}

__device__ __forceinline__ void load_window(const GpShape& s, const double* __restrict__ tab, const int* tr,
                            int nrows, int64_t i0, double* win) {
    for (int e = threadIdx.x; e < nrows * BK; e += blockDim.x) {
        int r = e / BK, k = e % BK;
        win[e] = __ldg(tab + (int64_t)tr[r] * s.Npad + i0 + k);
    }
}

__device__ __forceinline__ void gen_phi(const GpShape& s, const double* win, const unsigned short* cr, int m0,
                        double* phi) {
    for (int e = threadIdx.x; e < BK * TM; e += blockDim.x) {
        int c = e % TM, k = e / TM;
        double v = 0.0;
        if (m0 + c < s.M) {
            v = 1.0;
            for (int j = 0; j < s.p; ++j) v *= win[cr[c * s.p + j] * BK + k];
        }
        phi[k * TM + c] = v;
    }
}

__global__ void __launch_bounds__(256) syrk64_kernel(GpShape s, const double* __restrict__ tab,
                                                     const double* __restrict__ ypad, int64_t rps,
                                                     int npairs, int maxrows,
                                                     double* __restrict__ Gpart,
                                                     double* __restrict__ bpart) {
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ TileWindow wI, wJ;
    Smem64 sm;
    smem64_layout(maxrows, s.p, smem_raw, &sm);

    const int q = blockIdx.x, split = blockIdx.y;
    int I, J;
    tri_pair(q, &I, &J);
    const int tid = threadIdx.x;
    if (tid == 0) {
        tile_window(s, I * TM, TM, &wI);
        tile_window(s, J * TM, TM, &wJ);
    }
    __syncthreads();
    setup_tile(s, wI, I * TM, sm.trI, sm.crI);
    if (J != I) setup_tile(s, wJ, J * TM, sm.trJ, sm.crJ);
    __syncthreads();

    const int tx = tid % 16, ty = tid / 16;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    double bacc = 0.0;

    const double* phiB = (J == I) ? sm.phiI : sm.phiJ;
    int64_t r0 = (int64_t)split * rps;
    int64_t r1 = r0 + rps;
    if (r1 > s.Npad) r1 = s.Npad;
    for (int64_t i0 = r0; i0 < r1; i0 += BK) {
        load_window(s, tab, sm.trI, wI.nrows, i0, sm.winI);
        if (J != I) load_window(s, tab, sm.trJ, wJ.nrows, i0, sm.winJ);
        if (tid < BK) sm.yv[tid] = ypad[i0 + tid];
        __syncthreads();
        gen_phi(s, sm.winI, sm.crI, I * TM, sm.phiI);
        if (J != I) gen_phi(s, sm.winJ, sm.crJ, J * TM, sm.phiJ);
        __syncthreads();
        if (J == 0 && tid < TM) {
#pragma unroll
            for (int k = 0; k < BK; ++k) bacc += sm.phiI[k * TM + tid] * sm.yv[k];
        }
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sm.phiI[k * TM + ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = phiB[k * TM + tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    double* out = Gpart + ((int64_t)split * npairs + q) * (TM * TM);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) out[(ty + 16 * a) * TM + tx + 16 * b] = acc[a][b];
    if (J == 0 && tid < TM) bpart[(int64_t)split * s.Mpad + I * TM + tid] = bacc;
}

}  // namespace

size_t syrk64_smem_bytes(const GpShape& s) {
    return smem64_layout(gp_max_window_rows(s, TM), s.p, nullptr, nullptr);
}

cudaError_t launch_syrk64(const GpShape& s, const double* tab, const double* ypad, int nsplit,
                          int64_t rows_per_split, double* Gpart, double* bpart,
                          cudaStream_t stream) {
    int maxrows = gp_max_window_rows(s, TM);
    size_t smem = smem64_layout(maxrows, s.p, nullptr, nullptr);
    int T = s.Mpad / TM;
    int npairs = T * (T + 1) / 2;
    if (smem > 48 * 1024) {
        cudaError_t e = gp_allow_max_smem((const void*)syrk64_kernel);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)npairs, (unsigned)nsplit);
    syrk64_kernel<<<grid, 256, smem, stream>>>(s, tab, ypad, rows_per_split, npairs, maxrows, Gpart,
                                               bpart);
    return cudaGetLastError();
}
