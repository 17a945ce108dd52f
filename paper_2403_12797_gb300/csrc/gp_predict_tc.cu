// gp_predict_tc.cu -- fused Phi_* generation + bf16x3 tensor-core predict (tcgen05, TMEM, TMA).
//
//   mean_i = phi(x*_i)^T c                      (Eq. 11 in the M x M form)
//   var_i  = sigma^2 |W phi(x*_i)|^2,  W = L^{-1}  (diagonal of Eq. 12)
//
// CTA = 128 test points. Z = Phi_* W^T (128 x M) is accumulated in TMEM 512
// columns at a time ("super-tile" of four 128-column blocks of W's rows).
// For every 32-column chunk of Phi_* a pipeline stage holds the chunk's
// table window (the rows phi_d(x*_{.j}) its columns touch, for the CTA's
// test points), the chunk's column -> window-row map, the packed hi/lo
// blocks of W, and the generated hi/lo tile of Phi_*:
//   warp 9     (all lanes) copies the window rows, the map and the W blocks
//              with 1-D bulk (TMA) copies that complete on one mbarrier;
//   warps 0-7  producers, two threads per test point (warps 0-3 and 4-7
//              each take half of the chunk's columns): form the Phi_* chunk
//              in float32 (p a compile-time constant for p <= 4), add its
//              contribution to the mean (float32 products with a float32
//              copy of c, float64 running sum), split it into bf16 hi/lo in
//              the K-major core-matrix layout and publish it;
//   warp 8     issues hi*hi + hi*lo + lo*hi MMAs (M=128, N=128, K=16) into
//              each block's TMEM accumulator, skipping blocks where W is zero
//              (W is lower triangular).
// After a super-tile, the producers read their rows of Z from TMEM (each
// half every other 32 columns) and add the squares into the variance; the
// two halves' sums meet in shared memory at the end. With zpack given, the
// rows of Z are also stored (bf16 hi/lo, the operand layout of the MMAs
// here: per 128-point tile and 32-column chunk an 8 KB hi and an 8 KB lo
// block) for the covariance block of Eq. 12 (gp_cov.cu).
// Every wait is bounded; a warp decides with a
// vote, so tcgen05 loads stay warp-uniform and no CTA-wide barrier is left
// waiting for a warp that gave up.
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
constexpr int WIN_OFF = 2 * A_BYTES + SUPER * 2 * WB_BYTES;  // 80 KB: window after A and W
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = (BK / 8) * 128;     // 512
constexpr int NPROD = 2 * TT;                // two producer threads per test point (8 warps)
constexpr int NPW = NPROD / 32;
constexpr int MMA_W = NPW;                   // warp 8: MMA issuer
constexpr int NTHREADS = NPROD + 64;         // + warp 9: loader
constexpr unsigned FULLMASK = 0xffffffffu;

// Stage: [A hi | A lo | W blocks (hi, lo) x SUPER | window (maxrows + 1 rows
// of TT floats; the last row is zero) | column map (crp4 ints) | the chunk's
// BK float32 coefficients of c (the last super-tile's chunks, which form the
// mean)], 1 KB aligned.
__host__ __device__ inline uint32_t stage_bytes(int maxrows, int crp4) {
    const uint32_t end = WIN_OFF + (uint32_t)(maxrows + 1) * TT * 4 + (uint32_t)crp4 * 4 + BK * 4;
    return (end + 1023u) & ~1023u;
}
__host__ __device__ inline uint32_t map_off(int maxrows) { return WIN_OFF + (uint32_t)(maxrows + 1) * TT * 4; }

// barriers after the stages: full[S], wfull[S], empty[S], accf, tfree, combf[2], tmem base
__host__ __device__ inline size_t smem_bytes(int maxrows, int crp4) {
    return 1024 + (size_t)STAGES * stage_bytes(maxrows, crp4) + 8 * (3 * STAGES + 4) + 8;
}

// number of 32-column chunks of Phi_* that meet the blocks b0 .. b0+nblk-1
__host__ __device__ inline int super_chunks(int M, int b0, int nblk) {
    int mend = (b0 + nblk) * KB;
    if (mend > M) mend = M;
    return (mend + BK - 1) / BK;
}

// Phi_* of eight columns for test point t: column kk is the product of the
// window entries at the P float offsets map[kk * P + j] (+ t).
template <int P>
__device__ __forceinline__ void gen8(const float* win, const int* map, int p, int t, float* v) {
    if constexpr (P > 0) {
        int o[8 * P];
#pragma unroll
        for (int q = 0; q < 2 * P; ++q) {
            const int4 w = reinterpret_cast<const int4*>(map)[q];
            o[4 * q] = w.x;
            o[4 * q + 1] = w.y;
            o[4 * q + 2] = w.z;
            o[4 * q + 3] = w.w;
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            float x = win[o[kk * P] + t];
#pragma unroll
            for (int j = 1; j < P; ++j) x *= win[o[kk * P + j] + t];
            v[kk] = x;
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            float x = win[map[kk * p] + t];
            for (int j = 1; j < p; ++j) x *= win[map[kk * p + j] + t];
            v[kk] = x;
        }
    }
}

__host__ __device__ inline int nsuper_of(int M) { return ((M + KB - 1) / KB + SUPER - 1) / SUPER; }

// Item w of the launch: (request, 128-point tile, super-tile). A plain
// predict passes its one request by value and no item table: its items are
// the tiles' super-tiles, the costlier (later) super-tiles first, or only
// the last super-tiles when neither the variance nor Z is wanted.
__device__ __forceinline__ const PredReq& item_req(const PredReq& r0, const PredReq* __restrict__ reqs,
                                                   const int2* __restrict__ items, int w, int& tile, int& sup) {
    if (items == nullptr) {
        const int ntiles = (int)(r0.Npad / TT), ns = nsuper_of(r0.M);
        tile = w % ntiles;
        sup = ns - 1 - w / ntiles;
        return r0;
    }
    const int2 it = __ldg(items + w);
    const PredReq& R = reqs[it.x];
    const int ns = nsuper_of(R.M);
    tile = it.y / ns;
    sup = it.y % ns;
    return R;
}

template <int P>
__global__ void __launch_bounds__(NTHREADS, 1)
    predict_tc_kernel(const __grid_constant__ PredReq r0, const PredReq* __restrict__ reqs,
                      const int2* __restrict__ items,
                      int nitems, int maxrows_all, int crp4_all) {
    extern __shared__ __align__(1024) char smem_raw[];
    // 1 KB alignment by offsetting the shared array itself (keeps the
    // shared state space visible to the compiler)
    char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    // the stage layout is sized for the largest window and map of the launch
    const uint32_t SB = stage_bytes(maxrows_all, crp4_all);
    const uint32_t MAPO = map_off(maxrows_all);
    const uint32_t CFO = MAPO + (uint32_t)crp4_all * 4;  // the chunk's coefficients of c (16-byte aligned)
    uint8_t* stage = (uint8_t*)base;
    uint64_t* full = (uint64_t*)(base + (size_t)STAGES * SB);
    uint64_t* wfull = full + STAGES;
    uint64_t* empty = wfull + STAGES;
    uint64_t* accf = empty + STAGES;
    uint64_t* tfree = accf + 1;
    uint64_t* combf = tfree + 1;  // [2]
    uint32_t* tmem_base = (uint32_t*)(combf + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], NPW);
            mbar_init(&wfull[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(accf, 1);
        mbar_init(tfree, NPW);
        mbar_init(&combf[0], NPW / 2);
        mbar_init(&combf[1], NPW / 2);
        mbar_fence_init();
    }
    if (warp == MMA_W) tmem_alloc(tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_base;
    // the second half of a test point's producer threads hands its sums to
    // the first here, double-buffered by item
    __shared__ double comb_m[2][TT], comb_v[2][TT];
    const int t = tid & (TT - 1);     // test point (and TMEM lane) of a producer thread
    const int hf = tid / TT;          // its half of every 32-column chunk

    // Pipeline counters run on across the items of this CTA (chunks gc,
    // super-tiles gs, items li), so every barrier's phase follows from them.
    if (warp < NPW) {
        // ------------------------------------------------------------ producers + epilogue
        bool ok = true;
        int gc = 0, gs = 0, li = 0;
        for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x, ++li) {
            int tile, isup;
            const PredReq& R = item_req(r0, reqs, items, w, tile, isup);
            const int p = P > 0 ? P : R.p;
            const int M = R.M;
            const int64_t t0 = (int64_t)tile * TT;
            const int nblocks = (M + KB - 1) / KB;  // blocks of W rows with k < M
            const int nsuper = (nblocks + SUPER - 1) / SUPER;
            const int KBtot = R.Mpad / KB;           // blocks in the packed layout
            uint8_t* zpack = R.zpack;
            GpStatus* st = R.st;
            double macc = 0.0, vacc = 0.0;
            for (int sup = isup; sup <= isup && ok; ++sup, ++gs) {  // this item's super-tile
                const int b0 = sup * SUPER;
                const int nblk = min(SUPER, nblocks - b0);
                const int nch = super_chunks(M, b0, nblk);
                const bool last = (sup == nsuper - 1);
                for (int c = 0; c < nch; ++c, ++gc) {
                    const int stg = gc % STAGES;
                    // the stage's A tile is free (MMAs of chunk gc - STAGES done)
                    // and its window and map have landed
                    bool wt = gc < STAGES || mbar_wait(&empty[stg], ((gc / STAGES) - 1) & 1);
                    wt = wt && mbar_wait(&wfull[stg], (gc / STAGES) & 1);
                    if (!__all_sync(FULLMASK, wt)) {
                        if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 11);
                        ok = false;
                        break;
                    }
                    uint8_t* sb = stage + (size_t)stg * SB;
                    const float* win = reinterpret_cast<const float*>(sb + WIN_OFF);
                    const int* map = reinterpret_cast<const int*>(sb + MAPO);
                    float mpart = 0.f;
#pragma unroll
                    for (int g = 2 * hf; g < 2 * hf + 2; ++g) {
                        float v[8];
                        gen8<P>(win, map + g * 8 * p, p, t, v);
                        if (last) {
                            const float4* cs = reinterpret_cast<const float4*>(sb + CFO) + 2 * g;
                            const float4 ca = cs[0], cb = cs[1];
                            mpart = fmaf(v[0], ca.x, mpart);
                            mpart = fmaf(v[1], ca.y, mpart);
                            mpart = fmaf(v[2], ca.z, mpart);
                            mpart = fmaf(v[3], ca.w, mpart);
                            mpart = fmaf(v[4], cb.x, mpart);
                            mpart = fmaf(v[5], cb.y, mpart);
                            mpart = fmaf(v[6], cb.z, mpart);
                            mpart = fmaf(v[7], cb.w, mpart);
                        }
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
                        const uint32_t off = (uint32_t)(t >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(t & 7) * 16;
                        *reinterpret_cast<uint4*>(sb + off) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4*>(sb + A_BYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                    if (last) macc += (double)mpart;
                    // every lane's operand writes before the async proxy's reads;
                    // one arrival per warp
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[stg]);
                }
                if (!ok) break;
                // epilogue of this super-tile: rows of Z from TMEM
                const bool got = __all_sync(FULLMASK, mbar_wait(accf, gs & 1));
                if (!got) {
                    if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 12);
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int bb = 0; bb < nblk; ++bb) {
#pragma unroll 1
                    for (int ch = hf; ch < KB / 32; ch += 2) {  // this half's 32-column pieces
                        float v[32];
                        tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + bb * KB + ch * 32, v);
                        float q = 0.f;
#pragma unroll
                        for (int i = 0; i < 32; ++i) q = fmaf(v[i], v[i], q);
                        vacc += (double)q;
                        if (zpack != nullptr) {
                            // chunk (b0 + bb) * 4 + ch of this tile's rows of Z
                            uint8_t* zb = zpack + ((size_t)tile * (KBtot * (KB / BK)) +
                                                   (size_t)(b0 + bb) * (KB / BK) + ch) * (2 * A_BYTES);
#pragma unroll
                            for (int g = 0; g < BK / 8; ++g) {
                                uint32_t h[4], l[4];
#pragma unroll
                                for (int q2 = 0; q2 < 4; ++q2)
                                    split_bf16x2(v[8 * g + 2 * q2], v[8 * g + 2 * q2 + 1], h[q2], l[q2]);
                                const uint32_t off =
                                    (uint32_t)(t >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(t & 7) * 16;
                                *reinterpret_cast<uint4*>(zb + off) = make_uint4(h[0], h[1], h[2], h[3]);
                                *reinterpret_cast<uint4*>(zb + A_BYTES + off) = make_uint4(l[0], l[1], l[2], l[3]);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tfree);
            }
            if (!ok) break;
            // the two halves' sums of each test point meet: the first half
            // writes mean and variance
            const int cbuf = li & 1;
            if (hf == 1) {
                comb_m[cbuf][t] = macc;
                comb_v[cbuf][t] = vacc;
                __syncwarp();
                if (lane == 0) mbar_arrive(&combf[cbuf]);
            } else {
                if (!__all_sync(FULLMASK, mbar_wait(&combf[cbuf], (li >> 1) & 1))) {
                    if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 16);
                    ok = false;
                    break;
                }
                if (t0 + t < R.Ns) {
                    // the last super-tile meets every chunk of Phi_*: it forms the mean
                    if (isup == nsuper - 1) R.mean[t0 + t] = macc + comb_m[cbuf][t];
                    if (R.var) {
                        const double v = vacc + comb_v[cbuf][t];
                        if (nsuper == 1) R.var[t0 + t] = R.sigma2 * v;
                        else R.vpart[(int64_t)isup * R.Npad + t0 + t] = v;
                    }
                }
            }
        }
    } else if (warp == MMA_W) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(TT, KB);
            const uint32_t sbase = smem_u32(stage);
            int gc = 0, gs = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
                int tile, isup;
                const PredReq& R = item_req(r0, reqs, items, w, tile, isup);
                const int M = R.M;
                GpStatus* st = R.st;
                const int nblocks = (M + KB - 1) / KB;
                for (int sup = isup; sup <= isup && ok; ++sup, ++gs) {
                    const int b0 = sup * SUPER;
                    const int nblk = min(SUPER, nblocks - b0);
                    const int nch = super_chunks(M, b0, nblk);
                    if (gs > 0 && !mbar_wait(tfree, (gs - 1) & 1)) {
                        gp_set_status(st, GP_ETIMEOUT, 13);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int c = 0; c < nch; ++c, ++gc) {
                        const int stg = gc % STAGES;
                        if (!mbar_wait(&full[stg], (gc / STAGES) & 1) ||
                            !mbar_wait(&wfull[stg], (gc / STAGES) & 1)) {
                            gp_set_status(st, GP_ETIMEOUT, 14);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_hi = sbase + stg * SB;
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
                        mma_commit(&empty[stg]);
                    }
                    if (!ok) break;
                    mma_commit(accf);
                }
            }
            // the MMAs issued so far complete before TMEM is freed
            if (gc > 0) mbar_wait(&empty[(gc - 1) % STAGES], ((gc - 1) / STAGES) & 1);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ loader (bulk copies, all lanes)
        int gc = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
            int tile, isup;
            const PredReq& R = item_req(r0, reqs, items, w, tile, isup);
            const int p = P > 0 ? P : R.p;
            const int M = R.M;
            GpStatus* st = R.st;
            const int64_t t0 = (int64_t)tile * TT;
            const int nblocks = (M + KB - 1) / KB;
            const int KBtot = R.Mpad / KB;
            const int mrows = R.maxrows;
            const int crp4 = (BK * p + 3) & ~3;
            const int cstride = 4 + ((mrows + 3) & ~3) + crp4;
            const int* cinfo = R.cinfo;
            const uint8_t* Wpack = R.Wpack;
            const float* tab = R.tab;
            const float* cfg = R.cf;
            const int64_t Npad = R.Npad;
            const int nsuper = (nblocks + SUPER - 1) / SUPER;
            for (int sup = isup; sup <= isup && ok; ++sup) {
                const int b0 = sup * SUPER;
                const int nblk = min(SUPER, nblocks - b0);
                const int nch = super_chunks(M, b0, nblk);
                const bool last = (sup == nsuper - 1);  // its chunks also form the mean
                for (int c = 0; c < nch; ++c, ++gc) {
                    const int stg = gc % STAGES;
                    const int* ci = cinfo + (int64_t)c * cstride;
                    const int nrows = __ldg(ci);
                    // table rows of this lane's window rows (read before the wait)
                    const int row0 = lane < nrows ? __ldg(ci + 4 + lane) : 0;
                    const bool e = gc < STAGES || mbar_wait(&empty[stg], ((gc / STAGES) - 1) & 1);
                    if (!__all_sync(FULLMASK, e)) {
                        if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 15);
                        ok = false;
                        break;
                    }
                    uint8_t* sb = stage + (size_t)stg * SB;
                    // the model's zero window row (columns beyond M map to
                    // it): 128 floats, one float4 a lane, before the arrival
                    reinterpret_cast<float4*>(sb + WIN_OFF + (size_t)mrows * TT * 4)[lane] =
                        make_float4(0.f, 0.f, 0.f, 0.f);
                    __syncwarp();
                    const uint32_t wbytes = (uint32_t)nblk * 2 * WB_BYTES;
                    if (lane == 0)
                        mbar_arrive_expect_tx(&wfull[stg], wbytes + (uint32_t)nrows * TT * 4 + (uint32_t)crp4 * 4 +
                                                               (last ? (uint32_t)BK * 4 : 0u));
                    __syncwarp();
                    if (last && lane == 2) bulk_g2s(sb + CFO, cfg + (size_t)c * BK, (uint32_t)BK * 4, &wfull[stg]);
                    if (lane == 0)
                        bulk_g2s(sb + 2 * A_BYTES, Wpack + ((size_t)c * KBtot + b0) * 2 * WB_BYTES, wbytes,
                                 &wfull[stg]);
                    if (lane == 1)
                        bulk_g2s(sb + MAPO, ci + 4 + ((mrows + 3) & ~3), (uint32_t)crp4 * 4, &wfull[stg]);
                    for (int r = lane; r < nrows; r += 32) {
                        const int row = r < 32 ? row0 : __ldg(ci + 4 + r);
                        bulk_g2s(sb + WIN_OFF + (size_t)r * TT * 4, tab + (int64_t)row * Npad + t0, TT * 4,
                                 &wfull[stg]);
                    }
                }
            }
        }
        // before leaving, wait (bounded) for the copies this warp issued
        for (int g = gc - STAGES; g < gc; ++g)
            if (g >= 0) mbar_wait(&wfull[g % STAGES], (g / STAGES) & 1);
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_W) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// var = sigma2 * sum over the super-tiles (in their order) of the partial
// variances; blockIdx.y = request (the one by value when reqs is NULL)
__global__ void __launch_bounds__(256) predict_reduce_kernel(const __grid_constant__ PredReq r0,
                                                             const PredReq* __restrict__ reqs) {
    const PredReq& R = reqs ? reqs[blockIdx.y] : r0;
    const int ns = nsuper_of(R.M);
    if (ns == 1 || R.var == nullptr) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R.Ns) return;
    double v = 0.0;
    for (int k = 0; k < ns; ++k) v += R.vpart[(int64_t)k * R.Npad + t];
    R.var[t] = R.sigma2 * v;
}

}  // namespace

// packed hi/lo blocks of W (4 Mpad^2 bytes), then c in float32 (Mpad floats)
size_t predtc_wpack_bytes(int M) {
    const size_t Mpad = (size_t)gp_round_up(M, KB);
    return 4 * Mpad * Mpad + 4 * Mpad;
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
// row][float offset (window row x TT) of each (column, dimension); columns
// beyond M point at the zero row maxrows], padded to 16 bytes.
void predtc_build_cinfo(const GpShape& s, int* out) {
    const int maxrows = predtc_maxrows(s);
    const int maxrows4 = (maxrows + 3) & ~3;
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
                ci[4 + maxrows4 + cc * s.p + j] = (m < s.M ? window_row(s, w, j, m) : maxrows) * TT;
            }
    }
}

size_t predtc_smem_bytes(const GpShape& s) {
    return smem_bytes(predtc_maxrows(s), (BK * s.p + 3) & ~3);
}

int predtc_window_rows(const GpShape& s) { return predtc_maxrows(s); }

int predtc_nsuper(int M) { return nsuper_of(M); }

size_t predtc_vpart_elems(int64_t Npad, int M) {
    const int ns = nsuper_of(M);
    return ns > 1 ? (size_t)ns * (size_t)Npad : 0;
}

size_t predtc_batch_smem_bytes(int maxrows_all, int p) { return smem_bytes(maxrows_all, (BK * p + 3) & ~3); }

namespace {
int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

template <int P>
cudaError_t predict_tc_launch_t(const PredReq& r0, const PredReq* reqs, const int2* items, int nitems,
                                int maxrows_all, int p, cudaStream_t stream) {
    if (nitems <= 0) return cudaSuccess;
    const int crp4 = (BK * p + 3) & ~3;
    const size_t smem = smem_bytes(maxrows_all, crp4);
    if (smem > (227 - 5) * 1024) return cudaErrorInvalidConfiguration;  // static shared memory beside it
    cudaError_t e = gp_allow_max_smem((const void*)predict_tc_kernel<P>);
    if (e != cudaSuccess) return e;
    // persistent: one CTA per SM (the stages take most of its shared memory)
    const int grid = nitems < sm_count() ? nitems : sm_count();
    predict_tc_kernel<P><<<(unsigned)grid, NTHREADS, smem, stream>>>(r0, reqs, items, nitems, maxrows_all, crp4);
    return cudaGetLastError();
}

cudaError_t predict_tc_dispatch(const PredReq& r0, const PredReq* reqs, const int2* items, int nitems,
                                int maxrows_all, int p, cudaStream_t stream) {
    switch (p) {
        case 1: return predict_tc_launch_t<1>(r0, reqs, items, nitems, maxrows_all, p, stream);
        case 2: return predict_tc_launch_t<2>(r0, reqs, items, nitems, maxrows_all, p, stream);
        case 3: return predict_tc_launch_t<3>(r0, reqs, items, nitems, maxrows_all, p, stream);
        case 4: return predict_tc_launch_t<4>(r0, reqs, items, nitems, maxrows_all, p, stream);
        default: return predict_tc_launch_t<0>(r0, reqs, items, nitems, maxrows_all, p, stream);
    }
}
}  // namespace

cudaError_t launch_predict_tc(const GpShape& s, const float* tab, const uint16_t* Wpack, const int* cinfo,
                              double sigma2, double* mean, double* var, GpStatus* st, cudaStream_t stream,
                              uint8_t* zpack, double* vpart) {
    PredReq r{};
    r.Ns = s.N;
    r.Npad = s.Npad;
    r.p = s.p;
    r.n = s.n;
    r.M = s.M;
    r.Mpad = (int)gp_round_up(s.M, KB);
    r.maxrows = predtc_maxrows(s);
    r.tab = const_cast<float*>(tab);
    r.Wpack = (const uint8_t*)Wpack;
    r.cf = reinterpret_cast<const float*>((const uint8_t*)Wpack + 4 * (size_t)r.Mpad * r.Mpad);
    r.cinfo = cinfo;
    r.sigma2 = sigma2;
    r.mean = mean;
    r.var = var;
    r.zpack = zpack;
    r.vpart = vpart;
    r.st = st;
    const int ns = nsuper_of(s.M);
    if (var != nullptr && ns > 1 && vpart == nullptr) return cudaErrorInvalidValue;
    const int ntiles = (int)(s.Npad / TT);
    const int nitems = ntiles * ((var != nullptr || zpack != nullptr) ? ns : 1);
    cudaError_t e = predict_tc_dispatch(r, nullptr, nullptr, nitems, r.maxrows, s.p, stream);
    if (e != cudaSuccess || var == nullptr || ns == 1 || s.N == 0) return e;
    predict_reduce_kernel<<<dim3((unsigned)((s.N + 255) / 256), 1), 256, 0, stream>>>(r, nullptr);
    return cudaGetLastError();
}

void launch_predict_reduce_batch(const PredReq* reqs, int nreq, int64_t max_npad, cudaStream_t stream) {
    if (nreq <= 0 || max_npad <= 0) return;
    PredReq none{};
    predict_reduce_kernel<<<dim3((unsigned)((max_npad + 255) / 256), (unsigned)nreq), 256, 0, stream>>>(none, reqs);
}

cudaError_t launch_predict_tc_batch(const PredReq* reqs, const int2* items, int nitems, int p, int maxrows_all,
                                    cudaStream_t stream) {
    PredReq none{};
    return predict_tc_dispatch(none, reqs, items, nitems, maxrows_all, p, stream);
}

size_t predtc_zpack_bytes(int64_t Npad, int M) {
    return (size_t)Npad * (size_t)gp_round_up(M, KB) * 4;
}
