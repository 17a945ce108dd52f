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
//   * for every GP_TAB_BLOCK (1024) row block, each column m is scaled by
//     2^(6 - E_m), where 2^(E_m) bounds the exact maximum of |Phi[:, m]|
//     inside the block (launch_colexp), so |w| < 64 for w = Phi * 2^(6 - E_m);
//     a looser bound (the product of per-dimension table maxima is ~13x the
//     true maximum on Gaussian inputs) would leave s1 a few bits and put most
//     of each value in the truncating remainder sums;
//   * w = s1 + lo with the integer s1 = rint(w) (exact in fp16) and the
//     remainder lo = fp16(w - s1), |w - s1| <= 1/2 (2^-12 absolute error);
//   * acc1 += s1 s1' is an integer sum of magnitude at most 1024 * 64^2 =
//     2^22 over a block, hence exact in float32; acc2 += s1 lo' + lo s1' + lo lo'
//     is small beside it, so its truncation over one block is negligible
//     (the CTA-pair kernel sums 4096 rows, 2^24, under the largest exponent
//     of four blocks);
//   * after each block the producers multiply acc1 + acc2 by the exact power
//     of two that maps the block's column scaling to the global one and add
//     it into a float32 sum held in TMEM (columns 256-383, beside acc1 and
//     acc2); every FLUSH_BLOCKS blocks that sum is folded into the split's
//     partial tile, kept as unevaluated float pairs hi + lo (an exact
//     two-sum, ~46 bits) in L2-resident memory that only the folding thread
//     touches. Summing the blocks in float32 instead would lose ~1e-6 of G
//     over a million rows, enough to make a strongly conditioned A
//     indefinite. With 1024-row blocks a drain is rare, so the accumulators
//     are single-buffered: the MMAs of the next block wait for it.
// Representation error: |w - s1 - lo| <= 2^-12 (2^-18 of the block bound).
//
// CTA = one 128 x 128 lower-triangular tile pair (I >= J) of G and one split
// of the rows, pipelined over chunks of 32 rows through nst stages:
//   warp 17    (all lanes) copies the chunk's table window -- the tile's
//              rows of the chunk-major table, at most two contiguous ranges
//              per dimension and tile, plus y -- with 1-D bulk (TMA) copies
//              into a ring of up to 8 window slots, each released by the
//              producer warps once they have read it;
//   warps 0-15 producers (one 8-column core group each): form Phi for
//              column tiles I and J in the K-major core-matrix layout
//              (8 columns x 16 bytes) from the window, split, publish the
//              stage; J == 0 CTAs also accumulate b_I = Phi_I^T y (float32,
//              warp-shuffle reduction). They drain TMEM after each block
//              and write the (scaled) partial tile at the end.
//   warp 16    allocates TMEM and issues the MMAs (one elected lane):
//              4 x (128 x 128 x 16) per 16 rows; tcgen05.commit frees stages
//              (A tiles and windows) and signals finished blocks.
// Every warp waits on mbarriers by itself (bounded, decided by a warp vote):
// there is no CTA-wide barrier inside the pipeline. The block exponents E_m
// per block and the global ones come from launch_colexp, run first.
// The grid is one CTA per (pair, split) work item, the rows split per class
// of pair (SyrkSplit: diagonal pairs generate one operand tile and take
// longer splits; the pairs (I, 0) also form b), so the classes end together.
// Split partials are summed and unscaled in float64 by gp_assemble.cu.
#include "gp_syrk_tc.cuh"

namespace {

using namespace gpsyrk;

constexpr int TM = SYRKTC_TM;              // 128
constexpr int CW = SYRKTC_BK;              // 32 rows per table chunk
constexpr int STAGES = 4;                  // largest pipeline depth (nst <= STAGES at run time)
constexpr int WRMAX = 8;                   // deepest table-window ring (nwr <= WRMAX at run time)
constexpr int FLUSH_BLOCKS = 4;            // blocks summed in the TMEM float32 sum between flushes
// A pipeline stage holds H table chunks (KS = 32 H rows; H = 2 unless the
// windows of two chunks do not fit): per-stage costs -- waits, arrivals, the
// MMA issue -- are paid once per KS rows.
template <int H> struct StageGeom {
    static constexpr int KS = CW * H;                     // rows per stage
    static constexpr int TILE = TM * KS * 2;              // one 16-bit operand tile
    static constexpr int BYTES = 4 * TILE;                // A s1, A lo, B s1, B lo
    static constexpr uint32_t SBO = (KS / 8) * 128;       // 8-row groups
    static constexpr int BLOCK = GP_TAB_BLOCK / KS;       // stages per exact GP_TAB_BLOCK-row TMEM block
    static constexpr int BFOLD = 512 / KS;                // stages between float64 folds of b
};
constexpr int NPROD = 512;                 // 16 producer warps: one 8-column core group each
constexpr int NPW = NPROD / 32;
constexpr int CPT = TM / (NPW / 4);        // tile columns per thread in the TMEM drain (32)
constexpr int MMA_WARP = NPW;
constexpr int NTHREADS = NPROD + 64;
constexpr uint32_t TMEM_COLS = 512;        // acc1 | acc2 | float32 block sum | unused
constexpr unsigned FULLMASK = 0xffffffffu;

struct SmemTC {
    uint8_t* stage;       // nst x StageGeom<H>::BYTES (1024-aligned)
    float* win;           // nwr x H x (2 maxrows + 1) x WS: windows of tiles I, J and y, per chunk
    int* egI;             // TM: global column exponents E_glob
    int* egJ;
    unsigned short* crI;  // TM x p: window row of (column, dimension)
    unsigned short* crJ;
    int* rng;             // copy ranges (table row, rows, window row), 3 ints each
    uint64_t* full;       // STAGES: producers' tiles published (one arrival per producer warp)
    uint64_t* empty;      // STAGES: MMAs of the stage done
    uint64_t* tfull;      // WRMAX: window landed (count 1 + tx bytes)
    uint64_t* wempty;     // WRMAX: every producer warp has read the window (count NPW)
    uint64_t* accf;       // the block's MMAs are done (acc1, acc2 final)
    uint64_t* drained;    // acc1 and acc2 have been read back (one arrival per producer warp)
    uint32_t* tmem_base;
};

__host__ __device__ inline size_t smem_tc_layout(int maxrows, int p, int nst, int nwr, int H, char* base,
                                                  SmemTC* L) {
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = (off + align - 1) / align * align;
        size_t o = off;
        off += bytes;
        return o;
    };
    size_t oS = take((size_t)nst * 4 * TM * (CW * H) * 2, 1024);
    size_t oW = take(sizeof(float) * nwr * H * win_floats(maxrows), 16);
    size_t oEI = take(sizeof(int) * TM, 16);
    size_t oEJ = take(sizeof(int) * TM, 16);
    size_t oCI = take(sizeof(unsigned short) * TM * p, 16);
    size_t oCJ = take(sizeof(unsigned short) * TM * p, 16);
    size_t oR = take(sizeof(int) * 3 * max_ranges(p), 16);
    size_t oF = take(sizeof(uint64_t) * STAGES, 8);
    size_t oE = take(sizeof(uint64_t) * STAGES, 8);
    size_t oX = take(sizeof(uint64_t) * WRMAX, 8);
    size_t oY = take(sizeof(uint64_t) * WRMAX, 8);
    size_t oA = take(sizeof(uint64_t) * 2, 8);
    size_t oD = take(sizeof(uint64_t) * 2, 8);
    size_t oT = take(sizeof(uint32_t), 8);
    if (L) {
        L->stage = (uint8_t*)(base + oS);
        L->win = (float*)(base + oW);
        L->egI = (int*)(base + oEI);
        L->egJ = (int*)(base + oEJ);
        L->crI = (unsigned short*)(base + oCI);
        L->crJ = (unsigned short*)(base + oCJ);
        L->rng = (int*)(base + oR);
        L->full = (uint64_t*)(base + oF);
        L->empty = (uint64_t*)(base + oE);
        L->tfull = (uint64_t*)(base + oX);
        L->wempty = (uint64_t*)(base + oY);
        L->accf = (uint64_t*)(base + oA);
        L->drained = (uint64_t*)(base + oD);
        L->tmem_base = (uint32_t*)(base + oT);
    }
    return off + 1024;  // slack for aligning the dynamic base
}

// 8 consecutive floats of the table in global memory (read-only path)
__device__ __forceinline__ void ld_row8g(const float* p, float v[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// the same from shared memory (generic pointer), and the product with one
__device__ __forceinline__ void ld_row8s(const float* p, float v[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void mul_row8s(const float* p, float v[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] *= a.x; v[1] *= a.y; v[2] *= a.z; v[3] *= a.w;
    v[4] *= b.x; v[5] *= b.y; v[6] *= b.z; v[7] *= b.w;
}

// Column exponents from exact block maxima. For block b (GP_TAB_BLOCK rows)
// and column m, bmax[b * Mpad + m] = max over the block's rows i of
// |Phi[i, m]| (float bits; non-negative floats order as their bits), with
// Phi formed from the chunk-major float32 table exactly as the Gram kernels
// form it: the left-to-right product over the dimensions (Eq. 19). Then
// ebx[b * Mpad + m] = E with that maximum times (1 + 2^-20) below 2^E (so
// any other rounding order of the products also stays below 2^E), -100 for
// a column that is zero in the block, and colexp[m] = the largest E over the
// blocks: the Gram kernels' scaled values w = Phi 2^(6 - E) have |w| < 64.
// Columns are m = u n + k: u the digits of the upper p - 1 dimensions, k the
// last dimension's digit (stride 1).

// One thread: one u, 8 consecutive k, rows 8g .. 8g + 7 of every 32-row
// chunk of block b (g = lane & 3), table read through the read-only cache.
// The general form (any p, any table size), one CTA column per block. WB:
// also the block's partials of b = Phi^T y (one row range: bblk[b * Mpad + m]).
template <int P, bool WB>  // p (1..4), or 0: p at run time
__global__ void __launch_bounds__(256) colmax_ldg_kernel(GpShape s, const float* __restrict__ tabc, int U, int K8,
                                                         unsigned int* __restrict__ bmax, float* __restrict__ bblk) {
    const int b = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t & 3, item = t >> 2;
    const int k8 = item % K8, u = item / K8;
    const bool active = u < U;
    const int n = s.n, p = P > 0 ? P : s.p;
    const int64_t RC = (int64_t)(p * n + 1) * WS;
    const int64_t q0 = (int64_t)b * (GP_TAB_BLOCK / CW);
    const int64_t q1 = min(q0 + GP_TAB_BLOCK / CW, s.Npad / CW);
    int uoff[GP_PMAX];
    {
        int rest = u;
#pragma unroll
        for (int j = GP_PMAX - 2; j >= 0; --j) {  // digit of dimension j
            if (j < p - 1) {
                uoff[j] = (j * n + rest % n) * WS + 8 * g;
                rest /= n;
            }
        }
    }
    const int kbase = k8 * 8;
    const int nk = min(8, n - kbase);
    const int koff = ((p - 1) * n + kbase) * WS + 8 * g;
    const int yoff = p * n * WS + 8 * g;  // the chunk's y row
    float mx[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float bs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (active) {
        for (int64_t q = q0; q < q1; ++q) {
            const float* c = tabc + q * RC;
            float yr[8];
            if constexpr (WB) ld_row8g(c + yoff, yr);
            float pre[8];
            if (p > 1) {
                ld_row8g(c + uoff[0], pre);
                for (int j = 1; j + 1 < p; ++j) {
                    float r[8];
                    ld_row8g(c + uoff[j], r);
#pragma unroll
                    for (int i = 0; i < 8; ++i) pre[i] *= r[i];
                }
            }
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                if (kk < nk) {
                    float v[8];
                    ld_row8g(c + koff + kk * WS, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float x = p > 1 ? pre[i] * v[i] : v[i];
                        mx[kk] = fmaxf(mx[kk], fabsf(x));
                        if constexpr (WB) bs[kk] = fmaf(x, yr[i], bs[kk]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        mx[kk] = fmaxf(mx[kk], __shfl_xor_sync(0xffffffffu, mx[kk], 1));
        mx[kk] = fmaxf(mx[kk], __shfl_xor_sync(0xffffffffu, mx[kk], 2));
        if constexpr (WB) {
            bs[kk] += __shfl_xor_sync(0xffffffffu, bs[kk], 1);
            bs[kk] += __shfl_xor_sync(0xffffffffu, bs[kk], 2);
        }
    }
    if (!active || g != 0) return;
    for (int kk = 0; kk < nk; ++kk) {
        bmax[(int64_t)b * s.Mpad + u * n + kbase + kk] = __float_as_uint(mx[kk]);
        if constexpr (WB) bblk[(int64_t)b * s.Mpad + u * n + kbase + kk] = bs[kk];
    }
}

constexpr int CM_ITEMS = 64;   // (UT products x 8 digits) items per CTA: 4 threads each
constexpr int CM_STAGES = 4;   // deepest chunk ring

// The staged form for p <= 4: the chunks of a range of block b's rows pass
// through a shared-memory ring (cp.async, CM_STAGES deep, so the copies run
// several chunks ahead of the arithmetic). A thread forms its UT upper-digit
// products for its 8 rows once per chunk, then takes the last dimension's 8
// digits one row at a time (UT = 4, 2 with b, or 1 when there are too few
// products to fill a CTA that way); item i of the CTA's tile takes
// u = (i / K8) UT .. and k = (i % K8) 8 ... blockIdx = (item tile, row range,
// block). Each CTA folds its maxima into bmax with one atomicMax per column.
// WB: also b = Phi^T y, one FMA a value with the chunk's y row, summed in
// float32 over the CTA's rows and written per (block, row range) to bblk.
template <int P, int UT, bool WB>
__global__ void __launch_bounds__(256, 2) colmax_ring_kernel(GpShape s, const float* __restrict__ tabc, int U, int K8,
                                                          int nitems, int rr, unsigned int* __restrict__ bmax,
                                                          float* __restrict__ bblk) {
    extern __shared__ __align__(16) float ring[];
    const int n = s.n;
    const int rows = P * n + 1;
    const int cf = rows * WS;  // floats of one chunk
    const int b = blockIdx.z;
    const int64_t qb0 = (int64_t)b * (GP_TAB_BLOCK / CW);
    const int64_t qb1 = min(qb0 + GP_TAB_BLOCK / CW, s.Npad / CW);
    const int64_t per = (qb1 - qb0 + rr - 1) / rr;
    const int64_t q0 = qb0 + (int64_t)blockIdx.y * per;
    const int nq = (int)max((int64_t)0, min(qb1, q0 + per) - q0);
    const int g = threadIdx.x & 3;
    const int item = blockIdx.x * CM_ITEMS + (threadIdx.x >> 2);
    const bool active = item < nitems;
    const int k8 = item % K8, uq = item / K8;
    const int kbase = k8 * 8;
    const int nk = active ? min(8, n - kbase) : 0;
    const int koff = ((P - 1) * n + kbase) * WS + 8 * g;
    const int yoff = P * n * WS + 8 * g;  // the chunk's y row
    int uoff[UT][P > 1 ? P - 1 : 1];
    int nu = 0;  // valid upper-digit products of this thread
#pragma unroll
    for (int uu = 0; uu < UT; ++uu) {
        const int u = uq * UT + uu;
        if (active && u < U) nu = uu + 1;
        int rest = u < U ? u : 0;
#pragma unroll
        for (int j = P - 2; j >= 0; --j) {
            uoff[uu][j] = (j * n + rest % n) * WS + 8 * g;
            rest /= n;
        }
    }
    float mx[UT][8], bs[UT][8];
#pragma unroll
    for (int uu = 0; uu < UT; ++uu)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mx[uu][kk] = bs[uu][kk] = 0.f;
    const uint32_t ring_s = smem_u32(ring);
    auto load = [&](int slot, int64_t q) {
        const float* src = tabc + q * (int64_t)cf;
        for (int f = threadIdx.x * 4; f < cf; f += blockDim.x * 4)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(ring_s + 4u * (uint32_t)(slot * cf + f)),
                         "l"(src + f)
                         : "memory");
    };
#pragma unroll
    for (int st = 0; st < CM_STAGES - 1; ++st) {
        if (st < nq) load(st, q0 + st);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = 0; i < nq; ++i) {
        asm volatile("cp.async.wait_group %0;" ::"n"(CM_STAGES - 2) : "memory");
        __syncthreads();  // chunk i is in; every thread is done with chunk i - 1's slot
        if (i + CM_STAGES - 1 < nq) load((i + CM_STAGES - 1) % CM_STAGES, q0 + i + CM_STAGES - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const float* c = ring + (i % CM_STAGES) * cf;
        float pre[UT][8];
        if constexpr (P > 1) {
#pragma unroll
            for (int uu = 0; uu < UT; ++uu) {
                if (uu < nu) {
                    ld_row8s(c + uoff[uu][0], pre[uu]);
#pragma unroll
                    for (int j = 1; j < P - 1; ++j) mul_row8s(c + uoff[uu][j], pre[uu]);
                }
            }
        }
        float yr[8];
        if constexpr (WB) ld_row8s(c + yoff, yr);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            if (kk < nk) {
                float lr[8];
                ld_row8s(c + koff + kk * WS, lr);
#pragma unroll
                for (int uu = 0; uu < UT; ++uu) {
                    if (uu < nu) {
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const float x = P > 1 ? pre[uu][r] * lr[r] : lr[r];
                            mx[uu][kk] = fmaxf(mx[uu][kk], fabsf(x));
                            if constexpr (WB) bs[uu][kk] = fmaf(x, yr[r], bs[uu][kk]);
                        }
                    }
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int uu = 0; uu < UT; ++uu)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            mx[uu][kk] = fmaxf(mx[uu][kk], __shfl_xor_sync(0xffffffffu, mx[uu][kk], 1));
            mx[uu][kk] = fmaxf(mx[uu][kk], __shfl_xor_sync(0xffffffffu, mx[uu][kk], 2));
            if constexpr (WB) {
                bs[uu][kk] += __shfl_xor_sync(0xffffffffu, bs[uu][kk], 1);
                bs[uu][kk] += __shfl_xor_sync(0xffffffffu, bs[uu][kk], 2);
            }
        }
    if (g != 0) return;
#pragma unroll
    for (int uu = 0; uu < UT; ++uu)
        if (uu < nu)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
                if (kk < nk) {
                    const int m = (uq * UT + uu) * n + kbase + kk;
                    if (nq > 0) atomicMax(bmax + (int64_t)b * s.Mpad + m, __float_as_uint(mx[uu][kk]));
                    // every (block, row range) writes its partial, zero for an empty range
                    if constexpr (WB) bblk[((int64_t)b * rr + blockIdx.y) * s.Mpad + m] = bs[uu][kk];
                }
}

// b = Phi^T y from the partials: one warp per column, lanes over the
// (block, row range) partials in a fixed order, a fixed shuffle tree.
__global__ void __launch_bounds__(256) colb_kernel(GpShape s, int nparts, const float* __restrict__ bblk,
                                                   double* __restrict__ b) {
    const int m = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= s.M) return;  // whole warps
    double v = 0.0;
    for (int q = lane; q < nparts; q += 32) v += (double)bblk[(int64_t)q * s.Mpad + m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) b[m] = v;
}

// ebx, the pair blocks' exponents ebx4 and colexp from bmax: one warp per
// column, lanes over the pair blocks (each the GP_PAIR_BLOCK / GP_TAB_BLOCK
// scale blocks under it).
__global__ void __launch_bounds__(256) colexp_kernel(GpShape s, int nblk, int nblk4,
                                                     const unsigned int* __restrict__ bmax,
                                                     signed char* __restrict__ ebx, signed char* __restrict__ ebx4,
                                                     int* __restrict__ colexp) {
    constexpr int SUB = GP_PAIR_BLOCK / GP_TAB_BLOCK;
    const int m = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= s.Mpad) return;  // whole warps
    int emax = -100;
    for (int b4 = lane; b4 < nblk4; b4 += 32) {
        int e4 = m < s.M ? -100 : 0;
        for (int b = b4 * SUB; b < min(nblk, (b4 + 1) * SUB); ++b) {
            int E = 0;
            if (m < s.M) {
                const float x = __uint_as_float(bmax[(int64_t)b * s.Mpad + m]);
                E = -100;
                if (x > 0.f) {
                    frexpf(x * 1.00000095367431640625f, &E);  // (1 + 2^-20) max < 2^E
                    E = E < -100 ? -100 : (E > 127 ? 127 : E);
                }
                e4 = max(e4, E);
            }
            ebx[(int64_t)b * s.Mpad + m] = (signed char)E;
        }
        ebx4[(int64_t)b4 * s.Mpad + m] = (signed char)e4;
        emax = max(emax, e4);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if (lane == 0) colexp[m] = m < s.M ? emax : 0;
}

// Phi values of one column for data rows 8g..8g+7 of the chunk: the product
// over dimensions of the column's window rows, whose float offsets woff[j]
// (window row x WS) are held in registers; woff[0] < 0 marks a padding
// column (m >= M). P = 0 takes p at run time and the offsets from the
// column's window-row map crr in shared memory.
template <int P>
__device__ __forceinline__ void phi8(const float* win, const int* woff, const unsigned short* crr, int p,
                                     int g, float v[8]) {
    const int o0 = (P > 0) ? woff[0] : (crr[0] == 0xFFFF ? -1 : crr[0] * WS);
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
        for (int j = 1; j < p; ++j) mul_row(crr[j] * WS);
    }
}

// P = p for p <= 4 (offsets in registers, products unrolled), 0 otherwise;
// H = table chunks per pipeline stage. BATCH: the launch covers several
// problems (SyrkBatchProb table, all with this p): a CTA finds its problem
// by its item number, copies the problem's shape to the head of its dynamic
// shared memory (the layout follows it) and runs the problem's item as a
// launch of that problem alone would.
template <int P, int H, bool BATCH>
__global__ void __launch_bounds__(NTHREADS, 1)
    syrk_tc_kernel(const __grid_constant__ GpShape s_arg, const float* __restrict__ tabc_arg,
                   const signed char* __restrict__ ebx_arg, const int* __restrict__ colexp_arg,
                   const __grid_constant__ SyrkSplit sp_arg, int T_arg, int maxrows, int nst, int nwr,
                   float2* __restrict__ Gpart_arg, double* __restrict__ bpart_arg, GpStatus* st_arg,
                   const SyrkBatchProb* __restrict__ probs, int nprob) {
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ TileWindow wI, wJ;
    __shared__ int s_nrng;
    char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    int item0 = blockIdx.x;
    const SyrkBatchProb* pb = nullptr;
    if constexpr (BATCH) {
        int lo = 0, hi = nprob - 1;  // the last problem whose first item is <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].item0 <= (int64_t)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        pb = probs + lo;
        item0 = (int)(blockIdx.x - pb->item0);
        const int* src = reinterpret_cast<const int*>(&pb->s);
        int* dst = reinterpret_cast<int*>(base);
        for (int i = threadIdx.x; i < (int)(sizeof(GpShape) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        base += SYRK_BATCH_SHAPE_BYTES;
    }
    const GpShape& s = BATCH ? *reinterpret_cast<const GpShape*>(base - SYRK_BATCH_SHAPE_BYTES) : s_arg;
    const float* __restrict__ tabc = BATCH ? pb->tabc : tabc_arg;
    const signed char* __restrict__ ebx = BATCH ? pb->ebx : ebx_arg;
    const int* __restrict__ colexp = BATCH ? pb->colexp : colexp_arg;
    const SyrkSplit& sp = BATCH ? pb->sp : sp_arg;
    const int T = BATCH ? pb->T : T_arg;
    float2* __restrict__ Gpart = BATCH ? pb->Gpart : Gpart_arg;
    double* __restrict__ bpart = BATCH ? pb->bpart : bpart_arg;
    GpStatus* st = BATCH ? pb->st : st_arg;
    SmemTC sm;
    smem_tc_layout(maxrows, s.p, nst, nwr, H, base, &sm);
    using GM = StageGeom<H>;

    // work item -> (pair class, pair, split): the class-0 items (diagonal
    // pairs (k, k)) first, then class 1 ((k + 1, 0)), then class 2 (the
    // strictly lower pairs below row 0 and right of column 0); within a class
    // the pair index runs fastest
    int I, J, split, cls;
    {
        int item = item0;
        const int n0 = T, n1 = T - 1, n2 = (T - 1) * (T - 2) / 2;
        if (item < n0 * sp.n[0]) {
            cls = 0;
            I = J = item % n0;
            split = item / n0;
        } else if ((item -= n0 * sp.n[0]) < n1 * sp.n[1]) {
            cls = 1;
            I = item % n1 + 1;
            J = 0;
            split = item / n1;
        } else {
            item -= n1 * sp.n[1];
            cls = 2;
            int a, b;
            tri_pair(item % n2, &a, &b);
            I = a + 2;
            J = b + 1;
            split = item / n2;
        }
    }
    const int npairs = T * (T + 1) / 2;
    const int q = I * (I + 1) / 2 + J;
    const bool diag = (I == J);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    const int64_t rows_c = cls == 0 ? sp.rows[0] : (cls == 1 ? sp.rows[1] : sp.rows[2]);  // no local copy
    const int64_t r0 = (int64_t)split * rows_c;
    int64_t r1 = r0 + rows_c;
    if (r1 > s.Npad) r1 = s.Npad;
    // pipeline stages of KS rows (split boundaries are multiples of GP_TAB_BLOCK
    // rows and Npad of 128, so KS divides every split)
    const int nchunks = r0 < r1 ? (int)((r1 - r0) / GM::KS) : 0;
    const int nblocks = (nchunks + GM::BLOCK - 1) / GM::BLOCK;
    const int64_t RC = (int64_t)(s.p * s.n + 1) * WS;  // floats per table chunk
    const int wsz1 = win_floats(maxrows);                // one chunk's window
    const int wsz = H * wsz1;                            // one window slot

    if (tid == 0) {
        tile_window(s, I * TM, TM, &wI);
        tile_window(s, J * TM, TM, &wJ);
        int nr = tile_ranges(s, wI, 0, sm.rng, 0);
        const int nwin0 = diag ? wI.nrows : wI.nrows + wJ.nrows;
        if (!diag) nr = tile_ranges(s, wJ, wI.nrows, sm.rng, nr);
        sm.rng[3 * nr] = s.p * s.n;  // y
        sm.rng[3 * nr + 1] = 1;
        sm.rng[3 * nr + 2] = nwin0;
        s_nrng = nr + 1;
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&sm.full[i], NPW);
            mbar_init(&sm.empty[i], 1);
        }
        for (int i = 0; i < WRMAX; ++i) {
            mbar_init(&sm.tfull[i], 1);
            mbar_init(&sm.wempty[i], NPW);
        }
        mbar_init(sm.accf, 1);
        mbar_init(sm.drained, NPW);
        mbar_fence_init();
    }
    if (warp == MMA_WARP) tmem_alloc(sm.tmem_base, TMEM_COLS);
    __syncthreads();
    for (int e = tid; e < TM * s.p; e += NTHREADS) {
        const int c = e / s.p, j = e % s.p;
        const int mi = I * TM + c, mj = J * TM + c;
        sm.crI[e] = (unsigned short)(mi < s.M ? window_row(s, wI, j, mi) : 0xFFFF);
        sm.crJ[e] = (unsigned short)(mj < s.M ? window_row(s, wJ, j, mj) : 0xFFFF);
    }
    for (int c = tid; c < TM; c += NTHREADS) {
        sm.egI[c] = colexp[I * TM + c];
        sm.egJ[c] = colexp[J * TM + c];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_base;
    const int nrowsI = wI.nrows;
    const int nwin = (diag ? nrowsI : nrowsI + wJ.nrows) + 1;

    if (warp < NPW) {
        // ------------------------------------------------------------ producers
        // generation: this thread's tile column r (core group = warp), data rows 8g..8g+7
        const int g = lane >> 3;
        const int rl = lane & 7;
        const int r = 8 * warp + rl;
        // drain: TMEM lanes 32*quarter.. (tile rows), tile columns CPT*cgrp ..
        const int quarter = warp & 3;
        const int cgrp = warp >> 2;
        const unsigned short* crrI = sm.crI + r * s.p;
        const unsigned short* crrJ = (diag ? sm.crI : sm.crJ) + r * s.p;
        int woffI[P > 0 ? P : 1], woffJ[P > 0 ? P : 1];
        if constexpr (P > 0) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const unsigned short ci = crrI[j], cj = crrJ[j];
                woffI[j] = (j == 0 && ci == 0xFFFF) ? -1 : ci * WS;
                woffJ[j] = (j == 0 && cj == 0xFFFF) ? -1 : cj * WS;
            }
        }
        const int jwin = diag ? 0 : nrowsI * WS;  // tile J's window inside the stage window
        const int ywin = (nwin - 1) * WS;
        // b: float32 within a block, float64 across blocks
        float bacc = 0.f;
        double bsum = 0.0;
        // This thread's part of its tile row in the split's partial tile:
        // (hi, lo) float pairs of CPT columns.
        float2* grow = Gpart + ((int64_t)split * npairs + q) * (TM * TM) +
                       (int64_t)(quarter * 32 + lane) * TM + cgrp * CPT;
        bool flushed = false;  // the partial tile holds a first fold
        bool ok = true;
        const int blk0 = (int)(r0 / GP_TAB_BLOCK);
        const uint32_t lrow = ((uint32_t)(quarter * 32) << 16) + cgrp * CPT;  // lanes, first column
        auto drain = [&](int d) -> bool {
            if (!__all_sync(FULLMASK, mbar_wait(sm.accf, d & 1))) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 4);
                return false;
            }
            tc_fence_after();
            // back to the global column scaling: 2^(E_blk - E_glob) (exact powers of two)
            const signed char* eb = ebx + (int64_t)(blk0 + d) * s.Mpad;
            const int row = quarter * 32 + lane;
            const float mrow = pow2_down((int)eb[I * TM + row] - sm.egI[row]);
            const signed char* ebc = eb + J * TM + cgrp * CPT;
            const int* egc = (diag ? sm.egI : sm.egJ) + cgrp * CPT;
            const bool fresh = (d % FLUSH_BLOCKS == 0);                  // the TMEM sum is empty
            const bool fold = ((d + 1) % FLUSH_BLOCKS == 0 || d + 1 == nblocks);
            float4* g4 = reinterpret_cast<float4*>(grow);  // (hi, lo) of two columns
            // hi + v = s + e exactly (Knuth's two-sum); lo collects e
            auto add2 = [](float& hi, float& lo, float v) {
                const float sum = __fadd_rn(hi, v);
                const float t = __fsub_rn(sum, hi);
                const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, t)), __fsub_rn(v, t));
                hi = sum;
                lo = __fadd_rn(lo, e);
            };
#pragma unroll 1
            for (int ch = 0; ch < CPT / 8; ++ch) {
                const int2 e2 = *reinterpret_cast<const int2*>(ebc + ch * 8);
                float a1[8], a2[8], g[8];
                tmem_ld8(tmem + lrow + ch * 8, a1);
                tmem_ld8(tmem + lrow + 128 + ch * 8, a2);
                if (!fresh) tmem_ld8(tmem + lrow + 256 + ch * 8, g);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int eblk = (int)(signed char)((i < 4 ? e2.x : e2.y) >> (8 * (i & 3)));
                    const float mc = pow2_down(eblk - egc[ch * 8 + i]);
                    g[i] = fmaf(a1[i] + a2[i], mrow * mc, fresh ? 0.f : g[i]);
                }
                if (fold) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float4 o = flushed ? g4[ch * 4 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
                        add2(o.x, o.y, g[2 * k]);
                        add2(o.z, o.w, g[2 * k + 1]);
                        g4[ch * 4 + k] = o;
                    }
                } else {
                    tmem_st8(tmem + lrow + 256 + ch * 8, g);
                }
            }
            if (fold) flushed = true;
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(sm.drained);
            return true;
        };

        const int mI = I * TM + r, mJ = J * TM + r;
        // block exponents of this thread's columns, loaded one block ahead
        int eI = 0, eJ = 0;
        if (nblocks > 0) {
            eI = ebx[(int64_t)blk0 * s.Mpad + mI];
            eJ = ebx[(int64_t)blk0 * s.Mpad + mJ];
        }
        int next_drain = 0;
        float scI = 0.f, scJ = 0.f;
        // ring positions of chunk c: stage stg (phase sph = (c / nst) & 1) and
        // window slot wsl (phase wph = (c / nwr) & 1), advanced without division
        int stg = 0, sph = 0, wsl = 0, wph = 0;
        for (int c = 0; c < nchunks && ok; ++c) {
            // the stage's A tiles are free (MMAs of chunk c - nst done) and
            // the chunk's window has landed
            bool w = c < nst || mbar_wait(&sm.empty[stg], sph ^ 1);
            w = w && mbar_wait(&sm.tfull[wsl], wph);
            if (!__all_sync(FULLMASK, w)) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 1);
                ok = false;
                break;
            }
            if (c % GM::BFOLD == 0) {
                bsum += (double)bacc;
                bacc = 0.f;
            }
            if (c % GM::BLOCK == 0) {
                // a new block: quantisation scales 2^(6 - E_blk)
                scI = pow2i(6 - eI);
                scJ = pow2i(6 - eJ);
                const int nb = c / GM::BLOCK + 1;
                if (nb < nblocks) {
                    eI = ebx[(int64_t)(blk0 + nb) * s.Mpad + mI];
                    eJ = ebx[(int64_t)(blk0 + nb) * s.Mpad + mJ];
                }
            }
            uint8_t* sb = sm.stage + (size_t)stg * GM::BYTES;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float* win = sm.win + wsl * wsz + h * wsz1;  // chunk h of the stage
                const int kg = 4 * h + g;                          // K group of these 8 rows
                {
                    float v[8];
                    phi8<P>(win, woffI, crrI, s.p, g, v);
                    store_slices<GM::SBO>(sb, sb + GM::TILE, r, kg, v, scI);
                    if (J == 0) {
                        const float4* y4 = reinterpret_cast<const float4*>(win + ywin + 8 * g);
                        const float4 ya = y4[0], yb = y4[1];
                        bacc = fmaf(v[0], ya.x, bacc);
                        bacc = fmaf(v[1], ya.y, bacc);
                        bacc = fmaf(v[2], ya.z, bacc);
                        bacc = fmaf(v[3], ya.w, bacc);
                        bacc = fmaf(v[4], yb.x, bacc);
                        bacc = fmaf(v[5], yb.y, bacc);
                        bacc = fmaf(v[6], yb.z, bacc);
                        bacc = fmaf(v[7], yb.w, bacc);
                    }
                }
                if (!diag) {
                    float v[8];
                    phi8<P>(win + jwin, woffJ, crrJ, s.p, g, v);
                    store_slices<GM::SBO>(sb + 2 * GM::TILE, sb + 3 * GM::TILE, r, kg, v, scJ);
                }
            }
            // every lane's operand writes are ordered before the async proxy's
            // reads; one arrival per warp after the warp barrier
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.wempty[wsl]);  // this warp is done with the window
                mbar_arrive(&sm.full[stg]);
            }
            if (++stg == nst) {
                stg = 0;
                sph ^= 1;
            }
            if (++wsl == nwr) {
                wsl = 0;
                wph ^= 1;
            }
            // drain a finished block once one chunk of the next one is queued
            // (its MMAs are normally done by then; the next block's wait for it)
            while (next_drain < nblocks && min((next_drain + 1) * GM::BLOCK, nchunks) <= c) {
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
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16_f32(TM, TM);
            const uint32_t sbase = smem_u32(sm.stage);
            int stg = 0, sph = 0;
            for (int c = 0; c < nchunks; ++c) {
                const int d = c / GM::BLOCK, cb = c % GM::BLOCK;
                // the accumulators of block d - 1 have been read back
                if (cb == 0 && d >= 1 && !mbar_wait(sm.drained, (d - 1) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 5);
                    break;
                }
                if (!mbar_wait(&sm.full[stg], sph)) {
                    gp_set_status(st, GP_ETIMEOUT, 3);
                    break;
                }
                tc_fence_after();
                const uint32_t acc1 = tmem;
                const uint32_t acc2 = tmem + 128;
                const uint32_t a1 = sbase + stg * GM::BYTES;
                const uint32_t a2 = a1 + GM::TILE;
                const uint32_t b1 = diag ? a1 : a1 + 2 * GM::TILE;
                const uint32_t b2 = diag ? a2 : a1 + 3 * GM::TILE;
#pragma unroll
                for (int ks = 0; ks < GM::KS / 16; ++ks) {
                    const uint32_t ko = ks * 2 * LBO;
                    const uint64_t dA1 = smem_desc(a1 + ko, LBO, GM::SBO);
                    const uint64_t dA2 = smem_desc(a2 + ko, LBO, GM::SBO);
                    const uint64_t dB1 = smem_desc(b1 + ko, LBO, GM::SBO);
                    const uint64_t dB2 = smem_desc(b2 + ko, LBO, GM::SBO);
                    const uint32_t acc = (cb > 0 || ks > 0) ? 1u : 0u;
                    mma_bf16(acc1, dA1, dB1, idesc, acc);   // s1 s1'  (exact)
                    mma_bf16(acc2, dA1, dB2, idesc, acc);   // s1 lo'
                    mma_bf16(acc2, dA2, dB1, idesc, 1u);    // lo s1'
                    mma_bf16(acc2, dA2, dB2, idesc, 1u);    // lo lo'
                }
                mma_commit(&sm.empty[stg]);
                if (cb == GM::BLOCK - 1 || c == nchunks - 1) mma_commit(sm.accf);
                if (++stg == nst) {
                    stg = 0;
                    sph ^= 1;
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ window loader (bulk copies)
        const int nr = s_nrng;
        const uint32_t wbytes = (uint32_t)(H * nwin * WS * 4);
        // this lane's copy range (at most one per lane: 4p + 1 <= 32 ranges for p <= 7)
        int rdst = 0, rsrc = 0, rlen = 0;
        for (int k = lane; k < nr; k += 32) {
            rdst = sm.rng[3 * k + 2] * WS;
            rsrc = sm.rng[3 * k] * WS;
            rlen = sm.rng[3 * k + 1] * WS * 4;
        }
        const bool multi = nr > 32;
        int c = 0, wsl = 0, wph = 0;
        for (; c < nchunks; ++c) {
            // the window slot is free: every producer warp has read chunk c - nwr
            const bool e = c < nwr || mbar_wait(&sm.wempty[wsl], wph ^ 1);
            if (!__all_sync(FULLMASK, e)) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 6);
                break;
            }
            if (lane == 0) mbar_arrive_expect_tx(&sm.tfull[wsl], wbytes);
            __syncwarp();
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float* src = tabc + ((r0 + (int64_t)c * GM::KS) / CW + h) * RC;
                float* dst = sm.win + wsl * wsz + h * wsz1;
                if (!multi) {
                    if (lane < nr) bulk_g2s(dst + rdst, src + rsrc, (uint32_t)rlen, &sm.tfull[wsl]);
                } else {
                    for (int k = lane; k < nr; k += 32)
                        bulk_g2s(dst + sm.rng[3 * k + 2] * WS, src + (int64_t)sm.rng[3 * k] * WS,
                                 (uint32_t)sm.rng[3 * k + 1] * WS * 4, &sm.tfull[wsl]);
                }
            }
            if (++wsl == nwr) {
                wsl = 0;
                wph ^= 1;
            }
        }
        // before leaving, wait (bounded) for the copies this warp issued
        for (int k = c - nwr; k < c; ++k)
            if (k >= 0) mbar_wait(&sm.tfull[k % nwr], (k / nwr) & 1);
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Pipeline shape: two table chunks per stage when two operand stages and two
// window slots of two chunks fit, else one; then the deepest pipeline (<=
// STAGES operand stages, then <= WRMAX window slots) whose dynamic shared
// memory fits one CTA next to the kernel's static shared memory (tile
// windows and flags, under 2 KB). Returns the operand stages (0 if nothing
// fits).
int syrk_tc_stages(const GpShape& s, int maxrows, int* H, int* nwr, size_t* smem, size_t reserve = 0) {
    const size_t kDynamicBudget = (227 - 2) * 1024 - reserve;
    for (int h = 2; h >= 1; --h)
        for (int nst = STAGES; nst >= 2; --nst)
            for (int w = WRMAX; w >= 2; --w) {
                *smem = smem_tc_layout(maxrows, s.p, nst, w, h, nullptr, nullptr);
                if (*smem <= kDynamicBudget) {
                    *H = h;
                    *nwr = w;
                    return nst;
                }
            }
    return 0;
}

}  // namespace

namespace {
int colexp_sms() {
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
size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }
// bytes of the scale blocks' exponents, and of the pair blocks' after them
size_t ebx_exp_bytes(const GpShape& s) {
    return round16((size_t)((s.Npad + GP_TAB_BLOCK - 1) / GP_TAB_BLOCK) * (size_t)s.Mpad);
}
size_t ebx4_exp_bytes(const GpShape& s) {
    return round16((size_t)((s.Npad + GP_PAIR_BLOCK - 1) / GP_PAIR_BLOCK) * (size_t)s.Mpad);
}
}  // namespace

const signed char* syrktc_pair_exponents(const GpShape& s, const signed char* ebx) { return ebx + ebx_exp_bytes(s); }

namespace {
// The exponent pass's launch: staged (ring) or general, products per thread,
// items, item tiles and row ranges per block. wb: b is formed too.
struct ColPlan {
    bool ring;
    int U, K8, ut, nitems, tiles, rr;
};
ColPlan colexp_plan(const GpShape& s, bool wb) {
    ColPlan c{};
    c.U = 1;
    for (int j = 0; j + 1 < s.p; ++j) c.U *= s.n;
    c.K8 = (s.n + 7) / 8;
    const int nblk = (int)((s.Npad + GP_TAB_BLOCK - 1) / GP_TAB_BLOCK);
    const size_t chunk_bytes = (size_t)(s.p * s.n + 1) * WS * sizeof(float);
    c.ring = s.p <= 4 && CM_STAGES * chunk_bytes <= 96 * 1024;
    c.rr = 1;
    if (!c.ring || nblk == 0) return c;
    // four products a thread (two with b, for its accumulators' registers),
    // or one when that would leave most of a CTA idle; p = 1 has U = 1
    c.ut = (s.p > 1 && (c.U + 3) / 4 * c.K8 >= CM_ITEMS) ? (wb ? 2 : 4) : 1;
    c.nitems = (c.U + c.ut - 1) / c.ut * c.K8;
    c.tiles = (c.nitems + CM_ITEMS - 1) / CM_ITEMS;
    // row ranges per block: about two CTAs per SM in all
    const int64_t want = 2 * (int64_t)colexp_sms();
    c.rr = (int)std::min<int64_t>(GP_TAB_BLOCK / CW,
                                  std::max<int64_t>(1, (want + (int64_t)c.tiles * nblk - 1) / ((int64_t)c.tiles * nblk)));
    return c;
}
}  // namespace

size_t colexp_b_floats(const GpShape& s) {
    const int64_t nblk = (s.Npad + GP_TAB_BLOCK - 1) / GP_TAB_BLOCK;
    return (size_t)nblk * (size_t)colexp_plan(s, true).rr * (size_t)s.Mpad;
}

// the block maxima (float bits) follow both exponent arrays in the ebx buffer
void launch_colexp(const GpShape& s, const float* tabc, int* colexp, signed char* ebx, cudaStream_t stream,
                   float* bblk, double* b) {
    const bool wb = bblk != nullptr && b != nullptr;
    const int nblk = (int)((s.Npad + GP_TAB_BLOCK - 1) / GP_TAB_BLOCK);
    const int nblk4 = (int)((s.Npad + GP_PAIR_BLOCK - 1) / GP_PAIR_BLOCK);
    signed char* ebx4 = ebx + ebx_exp_bytes(s);
    unsigned int* bmax = reinterpret_cast<unsigned int*>(ebx4 + ebx4_exp_bytes(s));
    const ColPlan c = colexp_plan(s, wb);
    if (nblk > 0) {
        cudaMemsetAsync(bmax, 0, sizeof(unsigned int) * (size_t)nblk * s.Mpad, stream);
        if (c.ring) {
            const size_t ring = CM_STAGES * (size_t)(s.p * s.n + 1) * WS * sizeof(float);
            const dim3 grid((unsigned)c.tiles, (unsigned)c.rr, (unsigned)nblk);
            auto go = [&](auto kern) {
                if (ring > 48 * 1024) gp_allow_max_smem((const void*)kern);
                kern<<<grid, CM_ITEMS * 4, ring, stream>>>(s, tabc, c.U, c.K8, c.nitems, c.rr, bmax, bblk);
            };
            switch ((s.p * 8 + c.ut) * 2 + (wb ? 1 : 0)) {
                case (1 * 8 + 1) * 2: go(colmax_ring_kernel<1, 1, false>); break;
                case (1 * 8 + 1) * 2 + 1: go(colmax_ring_kernel<1, 1, true>); break;
                case (2 * 8 + 1) * 2: go(colmax_ring_kernel<2, 1, false>); break;
                case (2 * 8 + 1) * 2 + 1: go(colmax_ring_kernel<2, 1, true>); break;
                case (2 * 8 + 2) * 2 + 1: go(colmax_ring_kernel<2, 2, true>); break;
                case (2 * 8 + 4) * 2: go(colmax_ring_kernel<2, 4, false>); break;
                case (3 * 8 + 1) * 2: go(colmax_ring_kernel<3, 1, false>); break;
                case (3 * 8 + 1) * 2 + 1: go(colmax_ring_kernel<3, 1, true>); break;
                case (3 * 8 + 2) * 2 + 1: go(colmax_ring_kernel<3, 2, true>); break;
                case (3 * 8 + 4) * 2: go(colmax_ring_kernel<3, 4, false>); break;
                case (4 * 8 + 1) * 2: go(colmax_ring_kernel<4, 1, false>); break;
                case (4 * 8 + 1) * 2 + 1: go(colmax_ring_kernel<4, 1, true>); break;
                case (4 * 8 + 2) * 2 + 1: go(colmax_ring_kernel<4, 2, true>); break;
                default: go(colmax_ring_kernel<4, 4, false>); break;
            }
        } else {
            const int64_t threads = (int64_t)c.U * c.K8 * 4;
            const dim3 g2((unsigned)((threads + 255) / 256), (unsigned)nblk);
            auto go = [&](auto kern) { kern<<<g2, 256, 0, stream>>>(s, tabc, c.U, c.K8, bmax, bblk); };
            switch (s.p * 2 + (wb ? 1 : 0)) {
                case 1 * 2: go(colmax_ldg_kernel<1, false>); break;
                case 1 * 2 + 1: go(colmax_ldg_kernel<1, true>); break;
                case 2 * 2: go(colmax_ldg_kernel<2, false>); break;
                case 2 * 2 + 1: go(colmax_ldg_kernel<2, true>); break;
                case 3 * 2: go(colmax_ldg_kernel<3, false>); break;
                case 3 * 2 + 1: go(colmax_ldg_kernel<3, true>); break;
                case 4 * 2: go(colmax_ldg_kernel<4, false>); break;
                case 4 * 2 + 1: go(colmax_ldg_kernel<4, true>); break;
                default:
                    if (wb) go(colmax_ldg_kernel<0, true>);
                    else go(colmax_ldg_kernel<0, false>);
                    break;
            }
        }
    }
    const int64_t warps = s.Mpad;
    colexp_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, stream>>>(s, nblk, nblk4, bmax, ebx, ebx4, colexp);
    if (wb) {
        if (nblk > 0) {
            colb_kernel<<<(unsigned)(((int64_t)s.M * 32 + 255) / 256), 256, 0, stream>>>(s, nblk * c.rr, bblk, b);
        } else {
            cudaMemsetAsync(b, 0, sizeof(double) * s.M, stream);
        }
    }
}

size_t syrktc_smem_bytes(const GpShape& s) {
    size_t smem = 0;
    int nwr = 0, H = 0;
    syrk_tc_stages(s, gp_max_window_rows(s, TM), &H, &nwr, &smem);
    return smem;
}

size_t syrktc_ebx_bytes(const GpShape& s) {
    return ebx_exp_bytes(s) + ebx4_exp_bytes(s) +
           sizeof(unsigned int) * (size_t)((s.Npad + GP_TAB_BLOCK - 1) / GP_TAB_BLOCK) * s.Mpad;
}

cudaError_t launch_syrk_tc(const GpShape& s, const float* tabc, const SyrkSplit& sp, float2* Gpart, double* bpart,
                           int* colexp, signed char* ebx, GpStatus* st, cudaStream_t stream) {
    if (s.Npad % (2 * CW) != 0) return cudaErrorInvalidValue;
    for (int c = 0; c < 3; ++c)
        if (sp.n[c] < 1 || sp.rows[c] < GP_TAB_BLOCK || sp.rows[c] % GP_TAB_BLOCK != 0) return cudaErrorInvalidValue;
    const int maxrows = gp_max_window_rows(s, TM);
    size_t smem = 0;
    int nwr = 0, H = 1;
    const int nst = syrk_tc_stages(s, maxrows, &H, &nwr, &smem);
    if (nst == 0) return cudaErrorInvalidConfiguration;
    const int T = s.Mpad / TM;
    const int64_t items = (int64_t)T * sp.n[0] + (int64_t)(T - 1) * sp.n[1] + (int64_t)(T - 1) * (T - 2) / 2 * sp.n[2];
    dim3 grid((unsigned)items);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = gp_allow_max_smem((const void*)kern);
        if (e != cudaSuccess) return e;
        kern<<<grid, NTHREADS, smem, stream>>>(s, tabc, ebx, colexp, sp, T, maxrows, nst, nwr, Gpart, bpart, st,
                                               nullptr, 0);
        return cudaGetLastError();
    };
    if (H == 2) {
        switch (s.p) {
            case 1: return go(syrk_tc_kernel<1, 2, false>);
            case 2: return go(syrk_tc_kernel<2, 2, false>);
            case 3: return go(syrk_tc_kernel<3, 2, false>);
            case 4: return go(syrk_tc_kernel<4, 2, false>);
            default: return go(syrk_tc_kernel<0, 2, false>);
        }
    }
    switch (s.p) {
        case 1: return go(syrk_tc_kernel<1, 1, false>);
        case 2: return go(syrk_tc_kernel<2, 1, false>);
        case 3: return go(syrk_tc_kernel<3, 1, false>);
        case 4: return go(syrk_tc_kernel<4, 1, false>);
        default: return go(syrk_tc_kernel<0, 1, false>);
    }
}

int64_t syrktc_items(const GpShape& s, const SyrkSplit& sp) {
    const int T = s.Mpad / TM;
    return (int64_t)T * sp.n[0] + (int64_t)(T - 1) * sp.n[1] + (int64_t)(T - 1) * (T - 2) / 2 * sp.n[2];
}

cudaError_t launch_syrk_tc_batch(const SyrkBatchProb* probs, int nprob, int64_t items, int p, int maxrows,
                                 cudaStream_t stream) {
    if (items <= 0) return cudaSuccess;
    GpShape sh{};
    sh.p = p;
    size_t smem = 0;
    int nwr = 0, H = 1;
    const int nst = syrk_tc_stages(sh, maxrows, &H, &nwr, &smem, SYRK_BATCH_SHAPE_BYTES);
    if (nst == 0) return cudaErrorInvalidConfiguration;
    smem += SYRK_BATCH_SHAPE_BYTES;
    const GpShape none{};
    const SyrkSplit nosp{};
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = gp_allow_max_smem((const void*)kern);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)items, NTHREADS, smem, stream>>>(none, nullptr, nullptr, nullptr, nosp, 0, maxrows, nst, nwr,
                                                          nullptr, nullptr, nullptr, probs, nprob);
        return cudaGetLastError();
    };
    if (H == 2) {
        switch (p) {
            case 1: return go(syrk_tc_kernel<1, 2, true>);
            case 2: return go(syrk_tc_kernel<2, 2, true>);
            case 3: return go(syrk_tc_kernel<3, 2, true>);
            case 4: return go(syrk_tc_kernel<4, 2, true>);
            default: return go(syrk_tc_kernel<0, 2, true>);
        }
    }
    switch (p) {
        case 1: return go(syrk_tc_kernel<1, 1, true>);
        case 2: return go(syrk_tc_kernel<2, 1, true>);
        case 3: return go(syrk_tc_kernel<3, 1, true>);
        case 4: return go(syrk_tc_kernel<4, 1, true>);
        default: return go(syrk_tc_kernel<0, 1, true>);
    }
}
