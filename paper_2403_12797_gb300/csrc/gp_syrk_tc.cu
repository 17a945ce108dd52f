// gp_syrk_tc.cu -- fused Phi generation + bf16 tensor-core Gram with exact block sums (tcgen05, TMEM).
//
// Computes G = Phi^T Phi and b = Phi^T y over the N training rows (the
// products of Lambda-bar and of W in Sec. 2.2). Phi (Eq. 19) is generated in
// shared memory, chunk by chunk, from the per-dimension eigenfunction tables
// and never written to global memory.
//
// Precision. The tensor cores' float32 accumulation truncates, so a long
// sum in TMEM drifts low by ~2e-8 per accumulate step; over the thousands of
// steps of a large N that bias (~1e-4 relative on G) is amplified by the
// conditioning of A into percent-level errors of the posterior. The kernel
// therefore keeps the dominant part of every tensor-core sum exact:
//   * for every 512-row block, each column m is scaled by 2^(7 - E_m), where
//     2^(E_m) bounds |Phi[:, m]| inside the block (the product of the block's
//     per-dimension table maxima), so |w| <= 128 for w = Phi * 2^(7 - E_m);
//   * w = s1 + lo with the integer s1 = rint(w) (exact in fp16) and the
//     remainder lo = fp16(w - s1), |w - s1| <= 1/2 (2^-12 absolute error);
//   * acc1 += s1 s1' is an integer sum below 2^24 for blocks of 512 rows,
//     hence exact in float32; acc2 += s1 lo' + lo s1' + lo lo' is a few
//     percent of G, so its truncation over one block (~2e-6 of itself) is
//     negligible;
//   * after each block the producers multiply acc1 + acc2 by the exact power
//     of two that maps the block's column scaling to the global one and add
//     it into float32 registers; every FLUSH_BLOCKS blocks those are folded
//     into the split's partial tile of float pairs (hi + lo, an exact
//     two-sum, ~46 bits), while the MMAs fill the other
//     TMEM buffer (two buffers x 256 columns = all 512); summing the blocks
//     in float32 instead would lose ~1e-6 of G over a million rows, enough
//     to make a strongly conditioned A indefinite.
// Representation error: |w - s1 - lo| <= 2^-12 (2^-19 of the block bound).
//
// CTA = one 128 x 128 lower-triangular tile pair (I >= J) of G and one split
// of the rows:
//   warps 0-15 producers (one 8-column core group each): copy the tables'
//              window rows for the chunk into shared memory, form Phi for
//              column tiles I and J in the K-major core-matrix layout
//              (8 columns x 16 bytes), split, publish the stage; J == 0 CTAs
//              also accumulate b_I = Phi_I^T y (float32, warp-shuffle
//              reduction). They drain TMEM and write the (scaled) partial
//              tile at the end.
//   warp 16    allocates TMEM and issues the MMAs (one elected lane):
//              4 x (128 x 128 x 16) per 16 rows; tcgen05.commit frees stages
//              and signals finished blocks.
// Split partials are summed and unscaled in float64 by gp_assemble.cu.
#include "gp_kernels.cuh"
#include "gp_tc.cuh"

namespace {

constexpr int TM = SYRKTC_TM;              // 128
constexpr int BK = SYRKTC_BK;              // 32 data rows per chunk
constexpr int STAGES = 4;                  // largest pipeline depth (nst <= STAGES at run time)
constexpr int WBUF = 3;                    // table-window ring (chunks prefetched ahead)
constexpr int BLOCK_CHUNKS = 16;           // 512 rows per exact TMEM block
constexpr int FLUSH_BLOCKS = 4;            // blocks summed in float32 registers between flushes
constexpr int WSTRIDE = BK + 4;            // floats per window row (bank-conflict padding)
constexpr int TILE_BYTES = TM * BK * 2;    // one bf16 operand tile: 8 KB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A s1, A s2, B s1, B s2
constexpr uint32_t LBO = 128;              // K-adjacent core matrices
constexpr uint32_t SBO = (BK / 8) * 128;   // 8-row groups
constexpr int NPROD = 512;                 // 16 producer warps: one 8-column core group each
constexpr int NPW = NPROD / 32;
constexpr int CPT = TM / (NPW / 4);        // tile columns per thread in the TMEM drain (32)
constexpr int MMA_WARP = NPW;
constexpr int NTHREADS = NPROD + 32;
constexpr uint32_t TMEM_COLS = 512;        // 2 buffers x (acc1 | acc2)

struct SmemTC {
    uint8_t* stage;       // STAGES x STAGE_BYTES (1024-aligned)
    float* winI;          // WBUF x maxrows x WSTRIDE
    float* winJ;
    float* yv;            // WBUF x BK
    float* scI;           // 2 x TM: block column scales 2^(7 - E_blk), by block parity
    float* scJ;
    float* muI;           // 2 x TM: drain multipliers 2^(E_blk - E_glob)
    float* muJ;
    int* egI;             // TM: global column exponents E_glob
    int* egJ;
    int* trI;
    int* trJ;
    unsigned short* crI;  // TM x p
    unsigned short* crJ;
    uint64_t* full;       // STAGES
    uint64_t* empty;      // STAGES
    uint64_t* accf;       // 2: block finished in TMEM buffer u
    uint64_t* drained;    // 2: TMEM buffer u has been read back
    uint32_t* tmem_base;
};

__host__ __device__ inline size_t smem_tc_layout(int maxrows, int p, int nst, char* base, SmemTC* L) {
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = (off + align - 1) / align * align;
        size_t o = off;
        off += bytes;
        return o;
    };
    size_t oS = take((size_t)nst * STAGE_BYTES, 1024);
    size_t oWI = take(sizeof(float) * WBUF * maxrows * WSTRIDE, 16);
    size_t oWJ = take(sizeof(float) * WBUF * maxrows * WSTRIDE, 16);
    size_t oY = take(sizeof(float) * WBUF * BK, 16);
    size_t oSI = take(sizeof(float) * 2 * TM, 16);
    size_t oSJ = take(sizeof(float) * 2 * TM, 16);
    size_t oMI = take(sizeof(float) * 2 * TM, 16);
    size_t oMJ = take(sizeof(float) * 2 * TM, 16);
    size_t oEI = take(sizeof(int) * TM, 16);
    size_t oEJ = take(sizeof(int) * TM, 16);
    size_t oTI = take(sizeof(int) * maxrows, 16);
    size_t oTJ = take(sizeof(int) * maxrows, 16);
    size_t oCI = take(sizeof(unsigned short) * TM * p, 16);
    size_t oCJ = take(sizeof(unsigned short) * TM * p, 16);
    size_t oF = take(sizeof(uint64_t) * STAGES, 8);
    size_t oE = take(sizeof(uint64_t) * STAGES, 8);
    size_t oA = take(sizeof(uint64_t) * 2, 8);
    size_t oD = take(sizeof(uint64_t) * 2, 8);
    size_t oT = take(sizeof(uint32_t), 8);
    if (L) {
        L->stage = (uint8_t*)(base + oS);
        L->winI = (float*)(base + oWI);
        L->winJ = (float*)(base + oWJ);
        L->yv = (float*)(base + oY);
        L->scI = (float*)(base + oSI);
        L->scJ = (float*)(base + oSJ);
        L->muI = (float*)(base + oMI);
        L->muJ = (float*)(base + oMJ);
        L->egI = (int*)(base + oEI);
        L->egJ = (int*)(base + oEJ);
        L->trI = (int*)(base + oTI);
        L->trJ = (int*)(base + oTJ);
        L->crI = (unsigned short*)(base + oCI);
        L->crJ = (unsigned short*)(base + oCJ);
        L->full = (uint64_t*)(base + oF);
        L->empty = (uint64_t*)(base + oE);
        L->accf = (uint64_t*)(base + oA);
        L->drained = (uint64_t*)(base + oD);
        L->tmem_base = (uint32_t*)(base + oT);
    }
    return off + 1024;  // slack for aligning the dynamic base
}

// exponent e with |x| < 2^e (0 for x == 0)
__device__ __forceinline__ int bound_exp(unsigned int bits) {
    int e = 0;
    frexpf(__uint_as_float(bits), &e);
    return e;
}

// sum over dimensions of the table-maximum exponents of column m
__device__ __forceinline__ int column_exp(const GpShape& s, const unsigned int* __restrict__ tm, int m) {
    int E = 0;
    for (int j = 0; j < s.p; ++j) E += bound_exp(tm[j * s.n + (m / s.stride[j]) % s.n]);
    return E < -100 ? -100 : E;
}

// Window rows, column -> window-row map and global column exponents of one tile.
__device__ void setup_tile(const GpShape& s, const TileWindow& w, int m0,
                           const unsigned int* __restrict__ tmax, int* tr, unsigned short* cr,
                           int* eg, int* colexp_out, int tid, int nthr) {
    for (int r = tid; r < w.nrows; r += nthr) tr[r] = window_table_row(s, w, r);
    for (int e = tid; e < TM * s.p; e += nthr) {
        int c = e / s.p, j = e % s.p;
        int m = m0 + c;
        cr[e] = (unsigned short)(m < s.M ? window_row(s, w, j, m) : 0xFFFF);
    }
    for (int c = tid; c < TM; c += nthr) {
        const int m = m0 + c;
        const int E = m < s.M ? column_exp(s, tmax, m) : 0;
        eg[c] = E;
        if (colexp_out && m < s.M) colexp_out[m] = E;
    }
}

// Column scales of one tile for the 512-row block whose table maxima are tmb:
// quantisation scale 2^(7 - E_blk) (|Phi * scale| <= 128 inside the block) and
// the drain multiplier 2^(E_blk - E_glob) <= 1 back to the global scaling.
__device__ __forceinline__ void block_scales(const GpShape& s, int m0, const unsigned int* __restrict__ tmb,
                                             const int* eg, float* sc, float* mu, int c) {
    const int m = m0 + c;
    if (m >= s.M) {
        sc[c] = 0.f;
        mu[c] = 0.f;
        return;
    }
    const int E = column_exp(s, tmb, m);
    sc[c] = ldexpf(1.f, 7 - E);
    mu[c] = ldexpf(1.f, E - eg[c]);
}

// Start the asynchronous copy of the window rows (nrows x BK floats) of the
// chunk starting at data row i0 into win (16-byte cp.async per thread).
__device__ __forceinline__ void load_window_async(const GpShape& s, const float* __restrict__ tab,
                                                  const int* tr, int nrows, int64_t i0, float* win,
                                                  int tid) {
    const int nv = nrows * (BK / 4);
    for (int e = tid; e < nv; e += NPROD) {
        const int r = e / (BK / 4), v = e % (BK / 4);
        cp_async16(win + r * WSTRIDE + 4 * v, tab + (int64_t)tr[r] * s.Npad + i0 + 4 * v);
    }
}

// Phi values of one column for data rows 8g..8g+7 of the chunk: the product
// over dimensions of the column's window rows, whose float offsets woff[j]
// (window row x WSTRIDE) are held in registers; woff[0] < 0 marks a padding
// column (m >= M). P = 0 takes p at run time and the offsets from the
// column's window-row map crr in shared memory.
template <int P>
__device__ __forceinline__ void phi8(const float* win, const int* woff, const unsigned short* crr, int p,
                                     int g, float v[8]) {
    const int o0 = (P > 0) ? woff[0] : (crr[0] == 0xFFFF ? -1 : crr[0] * WSTRIDE);
    if (o0 < 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.f;
        return;
    }
    {
        const float4* w = reinterpret_cast<const float4*>(win + o0 + 8 * g);
        float4 a = w[0], b = w[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    auto mul_row = [&](int oj) {
        const float4* w = reinterpret_cast<const float4*>(win + oj + 8 * g);
        float4 a = w[0], b = w[1];
        v[0] *= a.x; v[1] *= a.y; v[2] *= a.z; v[3] *= a.w;
        v[4] *= b.x; v[5] *= b.y; v[6] *= b.z; v[7] *= b.w;
    };
    if constexpr (P > 0) {
#pragma unroll
        for (int j = 1; j < P; ++j) mul_row(woff[j]);
    } else {
        for (int j = 1; j < p; ++j) mul_row(crr[j] * WSTRIDE);
    }
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Scale 8 values by sc and split each into the integer s1 = rint(w)
// (|s1| <= 128, exact in fp16) and the remainder lo = fp16(w - s1)
// (|lo| <= 1/2, 11-bit precision, subnormals below 2^-14); store both
// core-matrix rows. The float-to-integer rounding and float16 packing
// instructions run at a fraction of the FMA rate, so s1 avoids both: adding
// 1.5 * 2^23 rounds w to the nearest integer k (ties to even) in the low
// mantissa bits of t, the integer k + 1152 has the float16 bit pattern
// 0x6480 + k (exponent 2^10), and one exact half2 subtraction of 1152 leaves
// k. Only the remainder takes a float16 conversion.
__device__ __forceinline__ void store_slices(uint8_t* s1_tile, uint8_t* lo_tile, int r, int g,
                                             const float v[8], float sc) {
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // v * sc is exact (sc is a power of two), so one rounding each: t rounds
        // v sc + 1.5 2^23 to an integer, a = rint(v sc), lo = v sc - a exactly
        const float t0 = __fmaf_rn(v[2 * q], sc, kMagic), t1 = __fmaf_rn(v[2 * q + 1], sc, kMagic);
        const float a0 = __fsub_rn(t0, kMagic), a1 = __fsub_rn(t1, kMagic);
        const uint32_t b0 = (uint32_t)__float_as_int(t0) - 0x4B400000u + 0x6480u;
        const uint32_t b1 = (uint32_t)__float_as_int(t1) - 0x4B400000u + 0x6480u;
        const uint32_t raw = __byte_perm(b0, b1, 0x5410);
        uint32_t k2;
        asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(k2) : "r"(raw), "r"(0x64806480u));  // - (1152, 1152)
        h[q] = k2;
        l[q] = pack_half2(__fmaf_rn(v[2 * q], sc, -a0), __fmaf_rn(v[2 * q + 1], sc, -a1));
    }
    const uint32_t off = (uint32_t)(r >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(r & 7) * 16;
    *reinterpret_cast<uint4*>(s1_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// P = p for p <= 4 (offsets in registers, products unrolled), 0 otherwise.
template <int P>
__global__ void __launch_bounds__(NTHREADS, 1)
    syrk_tc_kernel(GpShape s, const float* __restrict__ tab, const unsigned int* __restrict__ tmaxb,
                   const unsigned int* __restrict__ tmax,
                   const float* __restrict__ ypad, int64_t rps, int npairs, int maxrows, int nst,
                   float2* __restrict__ Gpart, double* __restrict__ bpart,
                   int* __restrict__ colexp, GpStatus* st) {
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ TileWindow wI, wJ;
    __shared__ int s_ok[2];
    char* base = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    SmemTC sm;
    smem_tc_layout(maxrows, s.p, nst, base, &sm);

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
    const int nblocks = (nchunks + BLOCK_CHUNKS - 1) / BLOCK_CHUNKS;

    if (tid == 0) {
        tile_window(s, I * TM, TM, &wI);
        tile_window(s, J * TM, TM, &wJ);
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&sm.full[i], NPROD);
            mbar_init(&sm.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.accf[i], 1);
            mbar_init(&sm.drained[i], NPROD);
        }
        mbar_fence_init();
    }
    if (warp == MMA_WARP) tmem_alloc(sm.tmem_base, TMEM_COLS);
    __syncthreads();
    if (tid < NPROD) {
        setup_tile(s, wI, I * TM, tmax, sm.trI, sm.crI, sm.egI, (J == 0 && split == 0) ? colexp : nullptr,
                   tid, NPROD);
        if (!diag) setup_tile(s, wJ, J * TM, tmax, sm.trJ, sm.crJ, sm.egJ, nullptr, tid, NPROD);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_base;

    if (warp < NPW) {
        // ------------------------------------------------------------ producers
        // generation: this thread's tile column r (core group = warp), data rows 8g..8g+7
        const int g = lane >> 3;
        const int rl = lane & 7;
        const int r = 8 * warp + rl;
        // drain: TMEM lanes 32*quarter.. (tile rows), tile columns CPT*cgrp ..
        const int quarter = warp & 3;
        const int cgrp = warp >> 2;
        int woffI[P > 0 ? P : 1], woffJ[P > 0 ? P : 1];
        if constexpr (P > 0) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const unsigned short ci = sm.crI[r * s.p + j];
                woffI[j] = (j == 0 && ci == 0xFFFF) ? -1 : ci * WSTRIDE;
                const unsigned short cj = diag ? ci : sm.crJ[r * s.p + j];
                woffJ[j] = (j == 0 && cj == 0xFFFF) ? -1 : cj * WSTRIDE;
            }
        }
        // b: float32 within a block, float64 across blocks
        float bacc = 0.f;
        double bsum = 0.0;
        // This thread's part of its tile row: blocks are summed in float32
        // registers (gacc) for FLUSH_BLOCKS blocks, then folded into the
        // split's partial tile, kept as unevaluated float pairs hi + lo
        // (~46-bit sums), by an exact two-sum in float32 arithmetic
        // (read-modify-write of memory only this thread touches, resident in
        // L2). The long sums over blocks thus lose nothing that matters, while
        // staying off the slow float64 pipe and off the drain's critical path
        // most of the time.
        float2* grow = Gpart + ((int64_t)split * npairs + q) * (TM * TM) +
                       (int64_t)(quarter * 32 + lane) * TM + cgrp * CPT;
        float gacc[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) gacc[i] = 0.f;
        bool flushed = false;
        auto flush = [&]() {
            // hi + v = s + e exactly (Knuth's two-sum); lo collects e
            auto add2 = [](float& hi, float& lo, float v) {
                const float s = __fadd_rn(hi, v);
                const float t = __fsub_rn(s, hi);
                const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, t)), __fsub_rn(v, t));
                hi = s;
                lo = __fadd_rn(lo, e);
            };
            float4* g4 = reinterpret_cast<float4*>(grow);  // (hi, lo) of two elements
#pragma unroll
            for (int k = 0; k < CPT / 2; ++k) {
                float4 o = flushed ? g4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                add2(o.x, o.y, gacc[2 * k]);
                add2(o.z, o.w, gacc[2 * k + 1]);
                g4[k] = o;
                gacc[2 * k] = 0.f;
                gacc[2 * k + 1] = 0.f;
            }
            flushed = true;
        };
        bool ok = true;

        // One thread waits and broadcasts, so every producer takes the same
        // path. Successive calls alternate between two flags: a flag is
        // rewritten only after the barrier of the following call, which every
        // reader of its previous value has passed.
        int nbc = 0;
        auto bcast_wait = [&](uint64_t* bar, uint32_t parity, int site) -> bool {
            const int slot = nbc++ & 1;
            if (tid == 0) {
                int fine = (bar == nullptr || mbar_wait(bar, parity)) ? 1 : 0;
                if (!fine) gp_set_status(st, GP_ETIMEOUT, site);
                s_ok[slot] = fine;
            }
            named_bar_sync(1, NPROD);
            return s_ok[slot] != 0;
        };
        auto drain = [&](int d) -> bool {
            const int u = d & 1;
            if (!bcast_wait(&sm.accf[u], (d >> 1) & 1, 4)) return false;
            tc_fence_after();
            const uint32_t lrow = ((uint32_t)(quarter * 32) << 16) + (uint32_t)u * 256 + cgrp * CPT;
            // back to the global column scaling (exact powers of two)
            const float mrow = sm.muI[u * TM + quarter * 32 + lane];
            const float* mcol = (diag ? sm.muI : sm.muJ) + u * TM + cgrp * CPT;
#pragma unroll
            for (int ch = 0; ch < CPT / 16; ++ch) {
                float a1[16], a2[16];
                tmem_ld16(tmem + lrow + ch * 16, a1);
                tmem_ld16(tmem + lrow + 128 + ch * 16, a2);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    gacc[ch * 16 + i] = fmaf(a1[i] + a2[i], mrow * mcol[ch * 16 + i], gacc[ch * 16 + i]);
            }
            tc_fence_before();
            mbar_arrive(&sm.drained[u]);
            if ((d + 1) % FLUSH_BLOCKS == 0 || d + 1 == nblocks) flush();
            return true;
        };

        // table windows are prefetched WBUF-1 chunks ahead into a ring
        const int wsz = maxrows * WSTRIDE;
        auto prefetch = [&](int cc) {
            if (cc < nchunks) {
                const int buf = cc % WBUF;
                const int64_t i0 = r0 + (int64_t)cc * BK;
                load_window_async(s, tab, sm.trI, wI.nrows, i0, sm.winI + buf * wsz, tid);
                if (!diag) load_window_async(s, tab, sm.trJ, wJ.nrows, i0, sm.winJ + buf * wsz, tid);
                if (tid < BK / 4) cp_async16(sm.yv + buf * BK + 4 * tid, ypad + i0 + 4 * tid);
            }
            cp_async_commit();  // one group per chunk, possibly empty
        };
        prefetch(0);
        prefetch(1);

        int next_drain = 0;
        float scI = 0.f, scJ = 0.f;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int stg = c % nst;
            const int buf = c % WBUF;
            cp_async_wait<1>();        // this thread's copies for chunk c have landed
            const float* winI = sm.winI + buf * wsz;
            const float* winJ = sm.winJ + buf * wsz;
            const float* yv = sm.yv + buf * BK;
            const int slot = (c / BLOCK_CHUNKS) & 1;
            const bool newblk = (c % BLOCK_CHUNKS == 0);
            if (newblk) {
                bsum += (double)bacc;
                bacc = 0.f;
                // a new 512-row block: its column scales (the drain of the
                // block two back, which used this slot, is complete)
                const unsigned int* tmb = tmaxb + ((r0 + (int64_t)c * BK) / GP_TAB_BLOCK) * (s.p * s.n);
                if (tid < TM)
                    block_scales(s, I * TM, tmb, sm.egI, sm.scI + slot * TM, sm.muI + slot * TM, tid);
                else if (!diag && tid < 2 * TM)
                    block_scales(s, J * TM, tmb, sm.egJ, sm.scJ + slot * TM, sm.muJ + slot * TM, tid - TM);
            }
            // One barrier per chunk: every thread's copies of chunk c are
            // visible, chunk c-1 is consumed (its window buffer may be
            // refilled), and the pipeline stage has been released by the MMAs.
            if (!bcast_wait(c >= nst ? &sm.empty[stg] : nullptr, ((c / nst) - 1) & 1, 1)) {
                ok = false;
                break;
            }
            if (newblk) {
                scI = sm.scI[slot * TM + r];
                scJ = diag ? scI : sm.scJ[slot * TM + r];
            }
            prefetch(c + 2);
            uint8_t* sb = sm.stage + (size_t)stg * STAGE_BYTES;
            {
                float v[8];
                phi8<P>(winI, woffI, sm.crI + r * s.p, s.p, g, v);
                store_slices(sb, sb + TILE_BYTES, r, g, v, scI);
                if (J == 0) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) bacc = fmaf(v[k], yv[8 * g + k], bacc);
                }
            }
            if (!diag) {
                float v[8];
                phi8<P>(winJ, woffJ, sm.crJ + r * s.p, s.p, g, v);
                store_slices(sb + 2 * TILE_BYTES, sb + 3 * TILE_BYTES, r, g, v, scJ);
            }
            fence_proxy_async_smem();
            mbar_arrive(&sm.full[stg]);
            // drain a finished block once nst chunks of the next one are queued
            while (next_drain < nblocks && min((next_drain + 1) * BLOCK_CHUNKS, nchunks) - 1 + nst <= c) {
                if (!drain(next_drain)) {
                    ok = false;
                    break;
                }
                ++next_drain;
            }
        }
        while (ok && next_drain < nblocks) {
            if (!drain(next_drain)) ok = false;
            ++next_drain;
        }
        cp_async_wait<0>();  // no copy of this thread may still be in flight at exit
        if (J == 0) {
            double v = bsum + (double)bacc;
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (lane < 8) bpart[(int64_t)split * s.Mpad + I * TM + r] = v;
        }
        if (nblocks == 0) {  // a split without rows: its partial tile is zero
#pragma unroll
            for (int k = 0; k < CPT; ++k) grow[k] = make_float2(0.f, 0.f);
        }
    } else {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16_f32(TM, TM);
            const uint32_t sbase = smem_u32(sm.stage);
            for (int c = 0; c < nchunks; ++c) {
                const int stg = c % nst;
                const int d = c / BLOCK_CHUNKS, cb = c % BLOCK_CHUNKS, u = d & 1;
                if (cb == 0 && d >= 2 && !mbar_wait(&sm.drained[u], ((d >> 1) - 1) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 5);
                    break;
                }
                if (!mbar_wait(&sm.full[stg], (c / nst) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 3);
                    break;
                }
                tc_fence_after();
                const uint32_t acc1 = tmem + (uint32_t)u * 256;
                const uint32_t acc2 = acc1 + 128;
                const uint32_t a1 = sbase + stg * STAGE_BYTES;
                const uint32_t a2 = a1 + TILE_BYTES;
                const uint32_t b1 = diag ? a1 : a1 + 2 * TILE_BYTES;
                const uint32_t b2 = diag ? a2 : a1 + 3 * TILE_BYTES;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t ko = ks * 2 * LBO;
                    const uint64_t dA1 = smem_desc(a1 + ko, LBO, SBO);
                    const uint64_t dA2 = smem_desc(a2 + ko, LBO, SBO);
                    const uint64_t dB1 = smem_desc(b1 + ko, LBO, SBO);
                    const uint64_t dB2 = smem_desc(b2 + ko, LBO, SBO);
                    const uint32_t acc = (cb > 0 || ks > 0) ? 1u : 0u;
                    mma_bf16(acc1, dA1, dB1, idesc, acc);   // s1 s1'  (exact)
                    mma_bf16(acc2, dA1, dB2, idesc, acc);   // s1 lo'
                    mma_bf16(acc2, dA2, dB1, idesc, 1u);    // lo s1'
                    mma_bf16(acc2, dA2, dB2, idesc, 1u);    // lo lo'
                }
                mma_commit(&sm.empty[stg]);
                if (cb == BLOCK_CHUNKS - 1 || c == nchunks - 1) mma_commit(&sm.accf[u]);
            }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// deepest pipeline (<= STAGES) whose dynamic shared memory fits one CTA next
// to the kernel's static shared memory (tile windows and flags, under 2 KB);
// 0 if none
int syrk_tc_stages(const GpShape& s, int maxrows, size_t* smem) {
    constexpr size_t kDynamicBudget = (227 - 2) * 1024;
    for (int nst = STAGES; nst >= 2; --nst) {
        *smem = smem_tc_layout(maxrows, s.p, nst, nullptr, nullptr);
        if (*smem <= kDynamicBudget) return nst;
    }
    return 0;
}

}  // namespace

size_t syrktc_smem_bytes(const GpShape& s) {
    size_t smem = 0;
    syrk_tc_stages(s, gp_max_window_rows(s, TM), &smem);
    return smem;
}

cudaError_t launch_syrk_tc(const GpShape& s, const float* tab, const unsigned int* tmaxb,
                           const unsigned int* tmax, const float* ypad, int nsplit,
                           int64_t rows_per_split, float2* Gpart, double* bpart, int* colexp,
                           GpStatus* st, cudaStream_t stream) {
    if (rows_per_split % GP_TAB_BLOCK != 0) return cudaErrorInvalidValue;
    const int maxrows = gp_max_window_rows(s, TM);
    size_t smem = 0;
    const int nst = syrk_tc_stages(s, maxrows, &smem);
    if (nst == 0) return cudaErrorInvalidConfiguration;
    const int T = s.Mpad / TM;
    const int npairs = T * (T + 1) / 2;
    dim3 grid((unsigned)npairs, (unsigned)nsplit);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = gp_allow_max_smem((const void*)kern);
        if (e != cudaSuccess) return e;
        kern<<<grid, NTHREADS, smem, stream>>>(s, tab, tmaxb, tmax, ypad, rows_per_split, npairs, maxrows,
                                               nst, Gpart, bpart, colexp, st);
        return cudaGetLastError();
    };
    switch (s.p) {
        case 1: return go(syrk_tc_kernel<1>);
        case 2: return go(syrk_tc_kernel<2>);
        case 3: return go(syrk_tc_kernel<3>);
        case 4: return go(syrk_tc_kernel<4>);
        default: return go(syrk_tc_kernel<0>);
    }
}
