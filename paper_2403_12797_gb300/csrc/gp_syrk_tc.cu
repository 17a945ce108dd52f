// gp_syrk_tc.cu -- fused Phi generation + bf16x3 tensor-core Gram (tcgen05, TMEM).
//
// Computes G = Phi^T Phi and b = Phi^T y over the N training rows (the
// products of Lambda-bar and of W in Sec. 2.2). Phi (Eq. 19) is generated in
// shared memory, chunk by chunk, from the per-dimension eigenfunction tables
// and never written to global memory.
//
// Precision: each Phi value v (float32) is split into bf16 hi = bf16(v) and
// lo = bf16(v - hi); the MMA accumulates hi*hi + hi*lo + lo*hi (+ lo*lo) in
// float32 TMEM. Without lo*lo every diagonal entry of G would be biased low
// by sum(lo^2) (~2.7e-6 relative): the 3-product mode adds that sum, taken
// on the CUDA cores, instead.
//
// CTA = one 128 x 128 lower-triangular tile pair (I >= J) of G and one split
// of the rows:
//   warps 0-3  producers: copy the tables' window rows for the chunk into
//              shared memory, form the Phi tiles of column tiles I and J in
//              the K-major core-matrix layout (8 columns x 16 bytes), split
//              them into hi/lo and publish the pipeline stage; the CTAs with
//              J == 0 also accumulate b_I = Phi_I^T y and reduce it with warp
//              shuffles. After the last chunk they are the epilogue: TMEM ->
//              registers -> float32 partial tile in global memory.
//   warp 4     allocates TMEM and issues the MMAs (one elected lane):
//              6 x (128 x 128 x 16) per 32-row chunk; tcgen05.commit frees
//              the stage.
// Split partials are summed in float64 by gp_assemble.cu.
#include "gp_kernels.cuh"
#include "gp_tc.cuh"

namespace {

constexpr int TM = SYRKTC_TM;         // 128
constexpr int BK = SYRKTC_BK;         // 32 data rows per chunk
constexpr int STAGES = 4;
constexpr int WSTRIDE = BK + 4;       // floats per window row (bank-conflict padding)
constexpr int TILE_BYTES = TM * BK * 2;  // one bf16 operand tile: 8 KB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A hi, A lo, B hi, B lo
constexpr uint32_t LBO = 128;         // K-adjacent core matrices
constexpr uint32_t SBO = (BK / 8) * 128;  // 8-row groups
constexpr int NPROD = 128;
constexpr int NTHREADS = NPROD + 32;

struct SmemTC {
    uint8_t* stage;      // STAGES x STAGE_BYTES (1024-aligned)
    float* winI;         // maxrows x WSTRIDE
    float* winJ;
    float* yv;           // BK
    int* trI;
    int* trJ;
    unsigned short* crI;  // TM x p
    unsigned short* crJ;
    uint64_t* full;      // STAGES
    uint64_t* empty;     // STAGES
    uint64_t* accf;      // 1
    uint32_t* tmem_base;
};

__host__ __device__ inline size_t smem_tc_layout(int maxrows, int p, char* base, SmemTC* L) {
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = (off + align - 1) / align * align;
        size_t o = off;
        off += bytes;
        return o;
    };
    size_t oS = take((size_t)STAGES * STAGE_BYTES, 1024);
    size_t oWI = take(sizeof(float) * maxrows * WSTRIDE, 16);
    size_t oWJ = take(sizeof(float) * maxrows * WSTRIDE, 16);
    size_t oY = take(sizeof(float) * BK, 16);
    size_t oTI = take(sizeof(int) * maxrows, 16);
    size_t oTJ = take(sizeof(int) * maxrows, 16);
    size_t oCI = take(sizeof(unsigned short) * TM * p, 16);
    size_t oCJ = take(sizeof(unsigned short) * TM * p, 16);
    size_t oF = take(sizeof(uint64_t) * STAGES, 8);
    size_t oE = take(sizeof(uint64_t) * STAGES, 8);
    size_t oA = take(sizeof(uint64_t), 8);
    size_t oT = take(sizeof(uint32_t), 8);
    if (L) {
        L->stage = (uint8_t*)(base + oS);
        L->winI = (float*)(base + oWI);
        L->winJ = (float*)(base + oWJ);
        L->yv = (float*)(base + oY);
        L->trI = (int*)(base + oTI);
        L->trJ = (int*)(base + oTJ);
        L->crI = (unsigned short*)(base + oCI);
        L->crJ = (unsigned short*)(base + oCJ);
        L->full = (uint64_t*)(base + oF);
        L->empty = (uint64_t*)(base + oE);
        L->accf = (uint64_t*)(base + oA);
        L->tmem_base = (uint32_t*)(base + oT);
    }
    return off + 1024;  // slack for aligning the dynamic base
}

__device__ void setup_tile(const GpShape& s, const TileWindow& w, int m0, int* tr,
                           unsigned short* cr, int tid, int nthr) {
    for (int r = tid; r < w.nrows; r += nthr) tr[r] = window_table_row(s, w, r);
    for (int e = tid; e < TM * s.p; e += nthr) {
        int c = e / s.p, j = e % s.p;
        int m = m0 + c;
        cr[e] = (unsigned short)(m < s.M ? window_row(s, w, j, m) : 0xFFFF);
    }
}

// window rows (nrows x BK floats) of the chunk starting at data row i0
__device__ __forceinline__ void load_window(const GpShape& s, const float* __restrict__ tab,
                                            const int* tr, int nrows, int64_t i0, float* win,
                                            int tid) {
    const int nv = nrows * (BK / 4);
    for (int e = tid; e < nv; e += NPROD) {
        const int r = e / (BK / 4), v = e % (BK / 4);
        const float4 x = __ldg(reinterpret_cast<const float4*>(tab + (int64_t)tr[r] * s.Npad + i0) + v);
        *reinterpret_cast<float4*>(win + r * WSTRIDE + 4 * v) = x;
    }
}

// Phi values of column r (window rows cr[r*p..]) for data rows 8g..8g+7 of the chunk.
__device__ __forceinline__ void phi8(const float* win, const unsigned short* crr, int p, int g,
                                     float v[8]) {
    if (crr[0] == 0xFFFF) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.f;
        return;
    }
    {
        const float4* w = reinterpret_cast<const float4*>(win + crr[0] * WSTRIDE + 8 * g);
        float4 a = w[0], b = w[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    for (int j = 1; j < p; ++j) {
        const float4* w = reinterpret_cast<const float4*>(win + crr[j] * WSTRIDE + 8 * g);
        float4 a = w[0], b = w[1];
        v[0] *= a.x; v[1] *= a.y; v[2] *= a.z; v[3] *= a.w;
        v[4] *= b.x; v[5] *= b.y; v[6] *= b.z; v[7] *= b.w;
    }
}

// Split 8 values into bf16 hi/lo, store both core-matrix rows; returns the
// sum of lo^2 (the expected value of the dropped lo*lo product on the diagonal).
__device__ __forceinline__ float store_hilo(uint8_t* hi_tile, uint8_t* lo_tile, int r, int g,
                                            const float v[8]) {
    uint32_t h[4], l[4];
    float lsq = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
        const float2 lf = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&l[q]));
        lsq = fmaf(lf.x, lf.x, fmaf(lf.y, lf.y, lsq));
    }
    const uint32_t off = (uint32_t)(r >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(r & 7) * 16;
    *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
    return lsq;
}

// FOUR = false: hi*hi + hi*lo + lo*hi on the tensor cores, and the diagonal
// CTAs add sum(lo^2) per column (dpart), the only part of the dropped lo*lo
// product whose expectation is not zero. FOUR = true: all four products.
template <bool FOUR>
__global__ void __launch_bounds__(NTHREADS, 1)
    syrk_tc_kernel(GpShape s, const float* __restrict__ tab, const float* __restrict__ ypad,
                   int64_t rps, int npairs, int maxrows, float* __restrict__ Gpart,
                   float* __restrict__ bpart, float* __restrict__ dpart, GpStatus* st) {
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ TileWindow wI, wJ;
    __shared__ int s_ok;
    char* base = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    SmemTC sm;
    smem_tc_layout(maxrows, s.p, base, &sm);

    const int q = blockIdx.x, split = blockIdx.y;
    int I, J;
    tri_pair(q, &I, &J);
    const bool diag = (I == J);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    const int64_t r0 = (int64_t)split * rps;
    int64_t r1 = r0 + rps;
    if (r1 > s.Npad) r1 = s.Npad;
    const int nchunks = r0 < r1 ? (int)((r1 - r0) / BK) : 0;

    if (tid == 0) {
        tile_window(s, I * TM, TM, &wI);
        tile_window(s, J * TM, TM, &wJ);
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&sm.full[i], NPROD);
            mbar_init(&sm.empty[i], 1);
        }
        mbar_init(sm.accf, 1);
        mbar_fence_init();
    }
    if (warp == 4) tmem_alloc(sm.tmem_base, TM);
    __syncthreads();
    if (tid < NPROD) {
        setup_tile(s, wI, I * TM, sm.trI, sm.crI, tid, NPROD);
        if (!diag) setup_tile(s, wJ, J * TM, sm.trJ, sm.crJ, tid, NPROD);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_base;

    if (warp < 4) {
        // ------------------------------------------------------------ producers
        const int g = lane >> 3;       // 8-row group of the chunk
        const int rl = lane & 7;       // column within an 8-column core group
        float bacc[4] = {0.f, 0.f, 0.f, 0.f};
        float dacc[4] = {0.f, 0.f, 0.f, 0.f};
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int stg = c % STAGES;
            const int64_t i0 = r0 + (int64_t)c * BK;
            named_bar_sync(1, NPROD);  // previous chunk's windows are consumed
            load_window(s, tab, sm.trI, wI.nrows, i0, sm.winI, tid);
            if (!diag) load_window(s, tab, sm.trJ, wJ.nrows, i0, sm.winJ, tid);
            if (tid < BK) sm.yv[tid] = ypad[i0 + tid];
            // one thread waits for the stage to be released by the MMAs and
            // broadcasts the outcome, so every producer leaves the loop together
            if (tid == 0) {
                int fine = 1;
                if (c >= STAGES && !mbar_wait(&sm.empty[stg], ((c / STAGES) - 1) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 1);
                    fine = 0;
                }
                s_ok = fine;
            }
            named_bar_sync(1, NPROD);
            if (!s_ok) {
                ok = false;
                break;
            }
            uint8_t* sb = sm.stage + (size_t)stg * STAGE_BYTES;
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int r = 8 * (it * 4 + warp) + rl;
                float v[8];
                phi8(sm.winI, sm.crI + r * s.p, s.p, g, v);
                const float lsq = store_hilo(sb, sb + TILE_BYTES, r, g, v);
                if (!FOUR && diag) dacc[it] += lsq;
                if (J == 0) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) bacc[it] = fmaf(v[k], sm.yv[8 * g + k], bacc[it]);
                }
            }
            if (!diag) {
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int r = 8 * (it * 4 + warp) + rl;
                    float v[8];
                    phi8(sm.winJ, sm.crJ + r * s.p, s.p, g, v);
                    store_hilo(sb + 2 * TILE_BYTES, sb + 3 * TILE_BYTES, r, g, v);
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&sm.full[stg]);
        }
        if (J == 0) {
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                float v = bacc[it];
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                if (lane < 8) {
                    const int r = 8 * (it * 4 + warp) + rl;
                    bpart[(int64_t)split * s.Mpad + I * TM + r] = v;
                }
            }
        }
        if (!FOUR && diag) {
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                float v = dacc[it];
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                if (lane < 8) {
                    const int r = 8 * (it * 4 + warp) + rl;
                    dpart[(int64_t)split * s.Mpad + I * TM + r] = v;
                }
            }
        }
        // ------------------------------------------------------------ epilogue
        bool got = ok && mbar_wait(sm.accf, 0);
        if (!got && ok) gp_set_status(st, GP_ETIMEOUT, 2);
        got = __all_sync(0xffffffffu, got);  // tcgen05.ld is warp-collective
        tc_fence_after();
        if (got) {
            const int row = warp * 32 + lane;
            float* out = Gpart + ((int64_t)split * npairs + q) * (TM * TM) + (int64_t)row * TM;
#pragma unroll 1
            for (int ch = 0; ch < TM / 32; ++ch) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
                float4* o4 = reinterpret_cast<float4*>(out + ch * 32);
#pragma unroll
                for (int k = 0; k < 8; ++k) o4[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            }
        }
    } else {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(TM, TM);
            const uint32_t sbase = smem_u32(sm.stage);
            for (int c = 0; c < nchunks; ++c) {
                const int stg = c % STAGES;
                if (!mbar_wait(&sm.full[stg], (c / STAGES) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 3);
                    break;
                }
                tc_fence_after();
                const uint32_t a_hi = sbase + stg * STAGE_BYTES;
                const uint32_t a_lo = a_hi + TILE_BYTES;
                const uint32_t b_hi = diag ? a_hi : a_hi + 2 * TILE_BYTES;
                const uint32_t b_lo = diag ? a_lo : a_hi + 3 * TILE_BYTES;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t ko = ks * 2 * LBO;
                    const uint64_t dAh = smem_desc(a_hi + ko, LBO, SBO);
                    const uint64_t dAl = smem_desc(a_lo + ko, LBO, SBO);
                    const uint64_t dBh = smem_desc(b_hi + ko, LBO, SBO);
                    const uint64_t dBl = smem_desc(b_lo + ko, LBO, SBO);
                    mma_bf16(tmem, dAh, dBh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                    mma_bf16(tmem, dAh, dBl, idesc, 1u);
                    mma_bf16(tmem, dAl, dBh, idesc, 1u);
                    if (FOUR) mma_bf16(tmem, dAl, dBl, idesc, 1u);
                }
                mma_commit(&sm.empty[stg]);
            }
            mma_commit(sm.accf);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        tmem_dealloc(tmem, TM);
    }
}

}  // namespace

size_t syrktc_smem_bytes(const GpShape& s) {
    return smem_tc_layout(gp_max_window_rows(s, TM), s.p, nullptr, nullptr);
}

cudaError_t launch_syrk_tc(const GpShape& s, const float* tab, const float* ypad, int nsplit,
                           int64_t rows_per_split, bool four, float* Gpart, float* bpart,
                           float* dpart, GpStatus* st, cudaStream_t stream) {
    const int maxrows = gp_max_window_rows(s, TM);
    const size_t smem = smem_tc_layout(maxrows, s.p, nullptr, nullptr);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = four ? syrk_tc_kernel<true> : syrk_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int T = s.Mpad / TM;
    const int npairs = T * (T + 1) / 2;
    dim3 grid((unsigned)npairs, (unsigned)nsplit);
    kern<<<grid, NTHREADS, smem, stream>>>(s, tab, ypad, rows_per_split, npairs, maxrows, Gpart,
                                           bpart, dpart, st);
    return cudaGetLastError();
}
