// gp_cov.cu -- the full predictive covariance block of Eq. 12.
//
// In the M x M form the posterior covariance of the latent f at the test
// points is Sigma_* = sigma^2 Phi_* A^{-1} Phi_*^T; with A = L L^T and
// W = L^{-1} this is sigma^2 Z Z^T for Z = Phi_* W^T (N_* x M), whose
// squared row norms are the predictive variances. The predict kernels leave
// Z behind (gp_predict_tc.cu as bf16 hi/lo operand blocks, gp_predict64.cu
// in float64); here the Gram of its rows is formed and written as the full
// symmetric N_* x N_* matrix, plus sigma^2 on the diagonal when the
// covariance of the noisy y_* is asked for.
//
// Mixed precision (cov_tc_kernel): one CTA per lower-triangle 128 x 128 tile
// (I, J) of Sigma_*; the tile is a tcgen05 MMA of M = N = 128 over the
// columns of Z, hi*hi + hi*lo + lo*hi as in the variance. Warp 4 streams
// the packed rows of Z of tiles I and J (one bulk copy each per 64-column
// stage; a diagonal tile loads its rows once and uses them as both
// operands), warp 5 issues the MMAs into a 128-column TMEM accumulator, and
// warps 0-3 write the tile (rows of tile J, coalesced along the test points
// of tile I) and, through shared memory, its transpose (a diagonal tile: both
// triangles from the entries on and above its diagonal).
//
// Float64 (cov64_kernel): the same tiling on the CUDA cores, 64 x 64 tiles.
#include "gp_kernels.cuh"
#include "gp_tc.cuh"

namespace {

constexpr int CT = PREDTC_TT;                  // 128 test points per tile
constexpr int ZBK = PREDTC_BK;                 // 32 columns of Z per packed chunk
constexpr int HALF_BYTES = CT * ZBK * 2;       // 8 KB: hi (or lo) block of a chunk
constexpr int CHUNK_BYTES = 2 * HALF_BYTES;    // hi + lo
constexpr int KC = 2;                          // chunks per pipeline stage
constexpr int OPB = KC * CHUNK_BYTES;          // 32 KB per operand per stage
constexpr int STAGES = 3;
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = (ZBK / 8) * 128;
constexpr int EPI_WARPS = 4;
constexpr int LOAD_W = 4, MMA_W = 5;
constexpr int NTHREADS = 192;
constexpr unsigned FULLMASK = 0xffffffffu;
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * 2 * OPB + 8 * (2 * STAGES + 1) + 8;

__global__ void __launch_bounds__(NTHREADS, 1)
    cov_tc_kernel(const uint8_t* __restrict__ zpack, int64_t Ns, int nkc, double sigma2, int noisy,
                  double* __restrict__ cov, GpStatus* st) {
    extern __shared__ __align__(1024) char smem_raw[];
    char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* stage = (uint8_t*)base;  // STAGES x [rows of tile I | rows of tile J]
    uint64_t* full = (uint64_t*)(base + (size_t)STAGES * 2 * OPB);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;
    uint32_t* tmem_base = (uint32_t*)(accf + 1);

    int I, J;
    tri_pair((int)blockIdx.x, &I, &J);
    const bool diag = (I == J);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nit = nkc / KC;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(accf, 1);
        mbar_fence_init();
    }
    if (warp == MMA_W) tmem_alloc(tmem_base, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_base;

    if (warp == LOAD_W) {
        // ------------------------------------------------------------ loader
        if (lane == 0) {
            const uint32_t bytes = diag ? (uint32_t)OPB : 2u * OPB;
            int it = 0;
            for (; it < nit; ++it) {
                const int stg = it % STAGES;
                if (it >= STAGES && !mbar_wait(&empty[stg], ((it / STAGES) - 1) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 40);
                    break;
                }
                uint8_t* sb = stage + (size_t)stg * 2 * OPB;
                mbar_arrive_expect_tx(&full[stg], bytes);
                bulk_g2s(sb, zpack + ((size_t)I * nkc + (size_t)it * KC) * CHUNK_BYTES, OPB, &full[stg]);
                if (!diag)
                    bulk_g2s(sb + OPB, zpack + ((size_t)J * nkc + (size_t)it * KC) * CHUNK_BYTES, OPB,
                             &full[stg]);
            }
            // the copies still in flight land before the CTA can leave
            for (int g = it - STAGES; g < it; ++g)
                if (g >= 0) mbar_wait(&full[g % STAGES], (g / STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == MMA_W) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(CT, CT);
            const uint32_t sbase = smem_u32(stage);
            for (int it = 0; it < nit; ++it) {
                const int stg = it % STAGES;
                if (!mbar_wait(&full[stg], (it / STAGES) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 41);
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = sbase + (uint32_t)stg * 2 * OPB;
                const uint32_t b0 = diag ? a0 : a0 + OPB;
#pragma unroll
                for (int q = 0; q < KC; ++q)
#pragma unroll
                    for (int ks = 0; ks < ZBK / 16; ++ks) {
                        const uint32_t ah = a0 + q * CHUNK_BYTES + ks * 2 * LBO;
                        const uint32_t bh = b0 + q * CHUNK_BYTES + ks * 2 * LBO;
                        const uint64_t dAh = smem_desc(ah, LBO, SBO), dAl = smem_desc(ah + HALF_BYTES, LBO, SBO);
                        const uint64_t dBh = smem_desc(bh, LBO, SBO), dBl = smem_desc(bh + HALF_BYTES, LBO, SBO);
                        mma_bf16(tmem, dAh, dBh, idesc, (it > 0 || q > 0 || ks > 0) ? 1u : 0u);
                        mma_bf16(tmem, dAh, dBl, idesc, 1u);
                        mma_bf16(tmem, dAl, dBh, idesc, 1u);
                    }
                mma_commit(&empty[stg]);
            }
            // also after a timeout: the accumulator's barrier completes once
            // every MMA issued so far has, so TMEM is freed only after them
            mma_commit(accf);
            mbar_wait(accf, 0);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue (warps 0-3)
        const bool got = __all_sync(FULLMASK, mbar_wait(accf, 0));
        if (!got) {
            if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 42);
        } else {
            tc_fence_after();
            // the operand stages are idle once the accumulator is complete:
            // 32 x 33 doubles of each warp's transposes live there
            double* tr = reinterpret_cast<double*>(stage) + (size_t)warp * 32 * 33;
            const int64_t row = (int64_t)I * CT + warp * 32 + lane;  // test point of tile I (TMEM lane)
#pragma unroll 1
            for (int cc = 0; cc < CT / 32; ++cc) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
                const int64_t c0 = (int64_t)J * CT + cc * 32;  // test points of tile J
                // Sigma_*[c0 + j][row]: consecutive lanes, consecutive addresses.
                // A diagonal tile holds D and D^T from separate tensor-core
                // sums, which may round apart: both triangles of it come from
                // its entries with col >= row, so the result is exactly symmetric.
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = c0 + j;
                    if (row < Ns && col < Ns && (!diag || col >= row)) {
                        double x = sigma2 * (double)v[j];
                        if (noisy && col == row) x += sigma2;
                        cov[col * Ns + row] = x;
                    }
                }
                // Sigma_*[row][c0 + j] through a transpose in shared memory
                if (!diag || c0 + 31 > (int64_t)I * CT + warp * 32) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) tr[j * 33 + lane] = sigma2 * (double)v[j];
                    __syncwarp();
                    const int64_t col = c0 + lane;
#pragma unroll 4
                    for (int r = 0; r < 32; ++r) {
                        const int64_t rr = (int64_t)I * CT + warp * 32 + r;
                        if (rr < Ns && col < Ns && (!diag || col > rr)) cov[rr * Ns + col] = tr[lane * 33 + r];
                    }
                    __syncwarp();
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_W) {
        tc_fence_after();
        tmem_dealloc(tmem, 128);
    }
}

// ---------------------------------------------------------------- float64

constexpr int CT64 = 64;  // test points per tile
constexpr int CK64 = 16;  // columns of Z per step

__global__ void __launch_bounds__(256) cov64_kernel(const double* __restrict__ Z, int64_t Ns, int zld,
                                                    double sigma2, int noisy, double* __restrict__ cov) {
    __shared__ double za[CK64][CT64 + 1], zb[CK64][CT64 + 1];
    int I, J;
    tri_pair((int)blockIdx.x, &I, &J);
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t r0 = (int64_t)I * CT64, c0 = (int64_t)J * CT64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < zld; k0 += CK64) {
        for (int e = tid; e < CT64 * CK64; e += 256) {
            const int r = e / CK64, c = e % CK64;
            za[c][r] = Z[(r0 + r) * zld + k0 + c];
            zb[c][r] = Z[(c0 + r) * zld + k0 + c];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CK64; ++c) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = za[c][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = zb[c][tx + 16 * b];
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
            const int64_t row = r0 + ty + 16 * a, col = c0 + tx + 16 * b;
            if (row >= Ns || col >= Ns) continue;
            double x = sigma2 * acc[a][b];
            if (noisy && row == col) x += sigma2;
            cov[row * Ns + col] = x;
            if (I != J) cov[col * Ns + row] = x;
        }
}

}  // namespace

cudaError_t launch_cov_tc(const uint8_t* zpack, int64_t Ns, int64_t Npad, int M, double sigma2, int noisy,
                          double* cov, GpStatus* st, cudaStream_t stream) {
    if (Ns <= 0) return cudaSuccess;
    const int nkc = gp_round_up(M, PREDTC_KB) / ZBK;  // a multiple of KC
    const int nt = (int)(Npad / CT);
    cudaError_t e = cudaFuncSetAttribute(cov_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((int64_t)nt * (nt + 1) / 2);
    cov_tc_kernel<<<grid, NTHREADS, SMEM_BYTES, stream>>>(zpack, Ns, nkc, sigma2, noisy, cov, st);
    return cudaGetLastError();
}

cudaError_t launch_cov64(const double* Z, int64_t Ns, int zld, double sigma2, int noisy, double* cov,
                         cudaStream_t stream) {
    if (Ns <= 0) return cudaSuccess;
    const int nt = (int)((Ns + CT64 - 1) / CT64);
    const unsigned grid = (unsigned)((int64_t)nt * (nt + 1) / 2);
    cov64_kernel<<<grid, 256, 0, stream>>>(Z, Ns, zld, sigma2, noisy, cov);
    return cudaGetLastError();
}
