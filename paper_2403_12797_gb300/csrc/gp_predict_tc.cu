// gp_predict_tc.cu -- fused Phi_* generation + bf16x3 tensor-core predict (tcgen05, TMEM, TMA).
//
//   mean_i = phi(x*_i)^T c                      (Eq. 11 in the M x M form)
//   var_i  = sigma^2 |W phi(x*_i)|^2,  W = L^{-1}  (diagonal of Eq. 12)
//
// CTA = 128 test points. Z = Phi_* W^T (128 x M) is accumulated in TMEM 512
// columns at a time ("super-tile" of four 128-column blocks of W's rows).
// For every 32-column chunk of Phi_*:
//   warps 0-3  producers: load the test points' table window rows, form the
//              Phi_* chunk (float32), add its contribution to the mean
//              (float32 products, float64 running sum), split it into bf16
//              hi/lo in the K-major core-matrix layout and publish it;
//   warp 5     loads the matching packed hi/lo blocks of W with one bulk
//              (TMA) copy per chunk;
//   warp 4     issues hi*hi + hi*lo + lo*hi MMAs (M=128, N=128, K=16) into
//              each block's TMEM accumulator, skipping blocks where W is zero
//              (W is lower triangular).
// After a super-tile, warps 0-3 read their rows of Z from TMEM and add the
// squares into the variance.
#include "gp_kernels.cuh"
#include "gp_tc.cuh"

namespace {

constexpr int TT = PREDTC_TT;       // 128 test points
constexpr int BK = PREDTC_BK;       // 32 columns of Phi_* per chunk
constexpr int KB = PREDTC_KB;       // 128 rows of W per block
constexpr int SUPER = PREDTC_SUPER; // 4 blocks in TMEM
constexpr int STAGES = 2;
constexpr int A_BYTES = TT * BK * 2;         // 8 KB per hi or lo tile
constexpr int WB_BYTES = KB * BK * 2;        // 8 KB per hi or lo block of W
constexpr int STAGE_BYTES = 2 * A_BYTES + SUPER * 2 * WB_BYTES;  // 80 KB
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = (BK / 8) * 128;     // 512
constexpr int NPROD = 128;
constexpr int NTHREADS = NPROD + 64;
constexpr int WBUF = 3;                      // window ring: chunks prefetched two ahead

struct SmemP {
    uint8_t* stage;
    float* win;               // WBUF x maxrows x TT: window rows of the prefetched chunks
    int* cr;                  // WBUF x crp4: column -> window-row map of those chunks
    uint64_t* full;           // producers' Phi_* tile is ready (count NPROD)
    uint64_t* wfull;          // the W bulk copy has landed (count 1 + tx bytes)
    uint64_t* empty;
    uint64_t* accf;
    uint64_t* tfree;
    uint32_t* tmem_base;
};

__host__ __device__ inline size_t smem_p_layout(int maxrows, int crp4, char* base, SmemP* L) {
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = (off + align - 1) / align * align;
        size_t o = off;
        off += bytes;
        return o;
    };
    size_t oS = take((size_t)STAGES * STAGE_BYTES, 1024);
    size_t oW = take(sizeof(float) * WBUF * maxrows * TT, 16);
    size_t oC = take(sizeof(int) * WBUF * crp4, 16);
    size_t oF = take(sizeof(uint64_t) * STAGES, 8);
    size_t oX = take(sizeof(uint64_t) * STAGES, 8);
    size_t oE = take(sizeof(uint64_t) * STAGES, 8);
    size_t oA = take(sizeof(uint64_t), 8);
    size_t oR = take(sizeof(uint64_t), 8);
    size_t oM = take(sizeof(uint32_t), 8);
    if (L) {
        L->stage = (uint8_t*)(base + oS);
        L->win = (float*)(base + oW);
        L->cr = (int*)(base + oC);
        L->full = (uint64_t*)(base + oF);
        L->wfull = (uint64_t*)(base + oX);
        L->empty = (uint64_t*)(base + oE);
        L->accf = (uint64_t*)(base + oA);
        L->tfree = (uint64_t*)(base + oR);
        L->tmem_base = (uint32_t*)(base + oM);
    }
    return off + 1024;
}

// number of 32-column chunks of Phi_* that meet the blocks b0 .. b0+nblk-1
__host__ __device__ inline int super_chunks(int M, int b0, int nblk) {
    int mend = (b0 + nblk) * KB;
    if (mend > M) mend = M;
    return (mend + BK - 1) / BK;
}

__global__ void __launch_bounds__(NTHREADS, 1)
    predict_tc_kernel(GpShape s, const float* __restrict__ tab, const uint8_t* __restrict__ Wpack,
                      const int* __restrict__ cinfo, int maxrows, const double* __restrict__ cvec,
                      double sigma2, double* __restrict__ mean, double* __restrict__ var,
                      GpStatus* st) {
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ int s_ok[2];
    char* base = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int maxrows4 = (maxrows + 3) & ~3;
    const int crp4 = (BK * s.p + 3) & ~3;
    const int cstride = 4 + maxrows4 + crp4;
    SmemP sm;
    smem_p_layout(maxrows, crp4, base, &sm);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t t0 = (int64_t)blockIdx.x * TT;
    const int nblocks = (s.M + KB - 1) / KB;     // blocks of W rows with k < M
    const int nsuper = (nblocks + SUPER - 1) / SUPER;
    const int KBtot = s.Mpad / KB;               // blocks in the packed layout

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&sm.full[i], NPROD);
            mbar_init(&sm.wfull[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        mbar_init(sm.accf, 1);
        mbar_init(sm.tfree, NPROD);
        mbar_fence_init();
    }
    if (warp == 4) tmem_alloc(sm.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_base;

    if (warp < 4) {
        // ------------------------------------------------------------ producers + epilogue
        const int t = tid;
        double macc = 0.0, vacc = 0.0;
        bool ok = true;
        int gc = 0;
        int nbc = 0;
        const int wsz = maxrows * TT;
        // prefetch cursor over the (super-tile, chunk) sequence, WBUF-1 chunks ahead
        int pf_sup = 0, pf_c = 0, pf_q = 0;
        auto prefetch_next = [&]() {
            if (pf_sup < nsuper) {
                const int buf = pf_q % WBUF;
                const int* ci = cinfo + (int64_t)pf_c * cstride;
                const int nrows = __ldg(ci);
                for (int e = tid; e < nrows * (TT / 4); e += NPROD) {
                    const int r = e / (TT / 4), v = e % (TT / 4);
                    const int row = __ldg(ci + 4 + r);
                    cp_async16(sm.win + buf * wsz + r * TT + 4 * v, tab + (int64_t)row * s.Npad + t0 + 4 * v);
                }
                for (int e = tid; e < crp4 / 4; e += NPROD)
                    cp_async16(sm.cr + buf * crp4 + 4 * e, ci + 4 + maxrows4 + 4 * e);
                if (++pf_c >= super_chunks(s.M, pf_sup * SUPER, min(SUPER, nblocks - pf_sup * SUPER))) {
                    ++pf_sup;
                    pf_c = 0;
                }
            }
            cp_async_commit();  // one group per chunk, possibly empty
            ++pf_q;
        };
        prefetch_next();
        prefetch_next();
        for (int sup = 0; sup < nsuper && ok; ++sup) {
            const int b0 = sup * SUPER;
            const int nblk = min(SUPER, nblocks - b0);
            const int nch = super_chunks(s.M, b0, nblk);
            const bool last = (sup == nsuper - 1);
            for (int c = 0; c < nch; ++c, ++gc) {
                const int stg = gc % STAGES;
                const int buf = gc % WBUF;
                cp_async_wait<1>();  // this thread's copies for chunk gc have landed
                // One barrier per chunk (one thread waits for the stage and
                // broadcasts; the two flags alternate so a flag is rewritten
                // only after every reader passed a later barrier): all copies
                // of chunk gc are visible and chunk gc-1 has been consumed.
                const int slot = nbc++ & 1;
                if (tid == 0) {
                    int fine = 1;
                    if (gc >= STAGES && !mbar_wait(&sm.empty[stg], ((gc / STAGES) - 1) & 1)) {
                        gp_set_status(st, GP_ETIMEOUT, 11);
                        fine = 0;
                    }
                    s_ok[slot] = fine;
                }
                named_bar_sync(1, NPROD);
                if (!s_ok[slot]) {
                    ok = false;
                    break;
                }
                prefetch_next();
                const float* win = sm.win + buf * wsz;
                const int* cr = sm.cr + buf * crp4;
                uint8_t* sb = sm.stage + (size_t)stg * STAGE_BYTES;
                float mpart = 0.f;
#pragma unroll
                for (int g = 0; g < BK / 8; ++g) {
                    float v[8];
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const int* crr = cr + (g * 8 + kk) * s.p;
                        float x = 0.f;
                        if (crr[0] >= 0) {
                            x = win[crr[0] * TT + t];
                            for (int j = 1; j < s.p; ++j) x *= win[crr[j] * TT + t];
                        }
                        v[kk] = x;
                    }
                    if (last) {
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const int m = c * BK + g * 8 + kk;
                            if (m < s.M) mpart = fmaf(v[kk], (float)__ldg(cvec + m), mpart);
                        }
                    }
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
                    const uint32_t off = (uint32_t)(t >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(t & 7) * 16;
                    *reinterpret_cast<uint4*>(sb + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(sb + A_BYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
                macc += (double)mpart;
                fence_proxy_async_smem();
                mbar_arrive(&sm.full[stg]);
            }
            if (!ok) break;
            // epilogue of this super-tile: rows of Z from TMEM. One thread
            // waits and broadcasts, so all producers take the same branch.
            const int slot = nbc++ & 1;
            if (tid == 0) {
                int fine = mbar_wait(sm.accf, sup & 1) ? 1 : 0;
                if (!fine) gp_set_status(st, GP_ETIMEOUT, 12);
                s_ok[slot] = fine;
            }
            named_bar_sync(1, NPROD);
            const bool got = s_ok[slot] != 0;
            tc_fence_after();
            if (got) {
                for (int bb = 0; bb < nblk; ++bb) {
#pragma unroll 1
                    for (int ch = 0; ch < KB / 32; ++ch) {
                        float v[32];
                        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + bb * KB + ch * 32, v);
                        float q = 0.f;
#pragma unroll
                        for (int i = 0; i < 32; ++i) q = fmaf(v[i], v[i], q);
                        vacc += (double)q;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(sm.tfree);
            if (!got) {
                ok = false;
                break;
            }
        }
        cp_async_wait<0>();  // no copy of this thread may still be in flight at exit
        if (ok && t0 + t < s.N) {
            mean[t0 + t] = macc;
            if (var) var[t0 + t] = sigma2 * vacc;
        }
    } else if (warp == 4) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(TT, KB);
            const uint32_t sbase = smem_u32(sm.stage);
            int gc = 0;
            bool ok = true;
            for (int sup = 0; sup < nsuper && ok; ++sup) {
                const int b0 = sup * SUPER;
                const int nblk = min(SUPER, nblocks - b0);
                const int nch = super_chunks(s.M, b0, nblk);
                if (sup > 0 && !mbar_wait(sm.tfree, (sup - 1) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 13);
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < nch; ++c, ++gc) {
                    const int stg = gc % STAGES;
                    if (!mbar_wait(&sm.full[stg], (gc / STAGES) & 1) ||
                        !mbar_wait(&sm.wfull[stg], (gc / STAGES) & 1)) {
                        gp_set_status(st, GP_ETIMEOUT, 14);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_hi = sbase + stg * STAGE_BYTES;
                    const uint32_t a_lo = a_hi + A_BYTES;
                    const uint32_t wbase = a_hi + 2 * A_BYTES;
                    for (int bb = 0; bb < nblk; ++bb) {
                        if (c > 4 * (b0 + bb) + 3) continue;  // W[k][m] = 0 for m > k
                        const uint32_t w_hi = wbase + bb * 2 * WB_BYTES;
                        const uint32_t w_lo = w_hi + WB_BYTES;
                        const uint32_t d = tmem + bb * KB;
#pragma unroll
                        for (int ks = 0; ks < BK / 16; ++ks) {
                            const uint32_t ko = ks * 2 * LBO;
                            const uint64_t dAh = smem_desc(a_hi + ko, LBO, SBO);
                            const uint64_t dAl = smem_desc(a_lo + ko, LBO, SBO);
                            const uint64_t dBh = smem_desc(w_hi + ko, LBO, SBO);
                            const uint64_t dBl = smem_desc(w_lo + ko, LBO, SBO);
                            mma_bf16(d, dAh, dBh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                            mma_bf16(d, dAh, dBl, idesc, 1u);
                            mma_bf16(d, dAl, dBh, idesc, 1u);
                        }
                    }
                    mma_commit(&sm.empty[stg]);
                }
                mma_commit(sm.accf);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ W loader (TMA)
        if (lane == 0) {
            int gc = 0;
            bool ok = true;
            for (int sup = 0; sup < nsuper && ok; ++sup) {
                const int b0 = sup * SUPER;
                const int nblk = min(SUPER, nblocks - b0);
                const int nch = super_chunks(s.M, b0, nblk);
                for (int c = 0; c < nch; ++c, ++gc) {
                    const int stg = gc % STAGES;
                    if (gc >= STAGES && !mbar_wait(&sm.empty[stg], ((gc / STAGES) - 1) & 1)) {
                        gp_set_status(st, GP_ETIMEOUT, 15);
                        ok = false;
                        break;
                    }
                    const uint32_t bytes = (uint32_t)nblk * 2 * WB_BYTES;
                    uint8_t* dst = sm.stage + (size_t)stg * STAGE_BYTES + 2 * A_BYTES;
                    const uint8_t* src = Wpack + ((size_t)c * KBtot + b0) * 2 * WB_BYTES;
                    mbar_arrive_expect_tx(&sm.wfull[stg], bytes);
                    bulk_g2s(dst, src, bytes, &sm.wfull[stg]);
                }
            }
            // before leaving, wait (bounded) for the copies this thread issued
            for (int g = gc - STAGES; g < gc; ++g)
                if (g >= 0) mbar_wait(&sm.wfull[g % STAGES], (g / STAGES) & 1);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// W (M x M float64, lower) -> packed bf16 hi/lo blocks: for chunk c (32
// columns m) and block b (128 rows k), hi then lo, each 128 x 32 in the
// K-major core-matrix layout of the MMA's B operand.
__global__ void pack_w_kernel(const double* __restrict__ W, int M, int Mpad, uint8_t* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int KBt = Mpad / KB;
    const int nch = Mpad / BK;
    const int64_t total = (int64_t)nch * KBt * KB * (BK / 8);
    if (idx >= total) return;
    const int g = (int)(idx % (BK / 8));
    const int r = (int)((idx / (BK / 8)) % KB);
    const int b = (int)((idx / ((BK / 8) * KB)) % KBt);
    const int c = (int)(idx / ((int64_t)(BK / 8) * KB * KBt));
    const int k = b * KB + r;
    float v[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const int m = c * BK + g * 8 + kk;
        v[kk] = (k < M && m < M && m <= k) ? (float)W[(int64_t)k * M + m] : 0.f;
    }
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
    uint8_t* blk = out + ((size_t)c * KBt + b) * 2 * WB_BYTES;
    const uint32_t off = (uint32_t)(r >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(r & 7) * 16;
    *reinterpret_cast<uint4*>(blk + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(blk + WB_BYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace

size_t predtc_wpack_bytes(int M) {
    const size_t Mpad = (size_t)gp_round_up(M, KB);
    return 4 * Mpad * Mpad;
}

void launch_pack_w_bf16x3(const double* W, int M, uint16_t* Wpack, cudaStream_t stream) {
    const int Mpad = (int)gp_round_up(M, KB);
    const int64_t total = (int64_t)(Mpad / BK) * (Mpad / KB) * KB * (BK / 8);
    pack_w_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(W, M, Mpad, (uint8_t*)Wpack);
}

namespace {
int predtc_maxrows(const GpShape& s) { return gp_max_window_rows(s, BK); }
int predtc_cstride(const GpShape& s) {
    return 4 + ((predtc_maxrows(s) + 3) & ~3) + ((BK * s.p + 3) & ~3);
}
}  // namespace

size_t predtc_cinfo_ints(const GpShape& s) {
    return (size_t)((s.M + BK - 1) / BK) * predtc_cstride(s);
}

// Per 32-column chunk c of Phi_*: [nrows, 0, 0, 0][table row of each window
// row][window row of (column, dimension), -1 beyond M], padded to 16 bytes.
void predtc_build_cinfo(const GpShape& s, int* out) {
    const int maxrows4 = (predtc_maxrows(s) + 3) & ~3;
    const int cs = predtc_cstride(s);
    const int nch = (s.M + BK - 1) / BK;
    for (int c = 0; c < nch; ++c) {
        int* ci = out + (size_t)c * cs;
        for (int i = 0; i < cs; ++i) ci[i] = 0;
        TileWindow w;
        tile_window(s, c * BK, BK, &w);
        ci[0] = w.nrows;
        for (int r = 0; r < w.nrows; ++r) ci[4 + r] = window_table_row(s, w, r);
        for (int cc = 0; cc < BK; ++cc)
            for (int j = 0; j < s.p; ++j) {
                const int m = c * BK + cc;
                ci[4 + maxrows4 + cc * s.p + j] = m < s.M ? window_row(s, w, j, m) : -1;
            }
    }
}

size_t predtc_smem_bytes(const GpShape& s) {
    return smem_p_layout(predtc_maxrows(s), (BK * s.p + 3) & ~3, nullptr, nullptr);
}

cudaError_t launch_predict_tc(const GpShape& s, const float* tab, const uint16_t* Wpack,
                              const int* cinfo, const double* c, double sigma2, double* mean,
                              double* var, GpStatus* st, cudaStream_t stream) {
    const int maxrows = predtc_maxrows(s);
    const size_t smem = predtc_smem_bytes(s);
    if (smem > (227 - 2) * 1024) return cudaErrorInvalidConfiguration;  // static shared memory beside it
    cudaError_t e = gp_allow_max_smem((const void*)predict_tc_kernel);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(s.Npad / TT);
    predict_tc_kernel<<<grid, NTHREADS, smem, stream>>>(s, tab, (const uint8_t*)Wpack, cinfo, maxrows,
                                                        c, sigma2, mean, var, st);
    return cudaGetLastError();
}
