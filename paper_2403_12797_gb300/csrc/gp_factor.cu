// gp_factor.cu -- factorisation of A = L L^T and the inverse W = L^{-1}.
//
// Sec. 3 of the paper inverts Lambda-bar with an LU factorisation; A =
// sigma^2 Lambda-bar is symmetric positive definite, so it is factored by
// Cholesky. On GB300 the float64 pipe retires about 2 FMAs per clock per SM,
// so an M x M factorisation only runs at speed when every SM works on it and
// no time is lost between launches. The three kernels here (Cholesky,
// inverse, solve) are therefore single persistent cooperative launches (at
// most one CTA per SM) that walk their block algorithms step by step,
// separated by grid barriers whose waits are bounded (GP_ETIMEOUT after
// GP_WAIT_NS; nothing can hang):
//
//   Cholesky (right-looking, 32-column panels, look-ahead; float64, or for a
//   mixed fit float32 pivots and panel solves on power-of-two equilibrated
//   blocks and rows, and float32 trailing-update products subtracted from the
//   float64 trailing matrix), per step k:
//     B  one warp per row below the factored diagonal block solves
//        x L_kk^T = a (lane j owns x_j);
//     C  16 helper CTAs update the next diagonal block and count themselves
//        done; CTA 0 waits for them and factors that block (32 x 32, in
//        shared memory) while the other CTAs update the rest of the trailing
//        lower triangle in tiles (16 x 16, or 64 x 64 with float32 products),
//        subtracting L_ik L_jk^T.
//   A non-positive or NaN pivot sets GP_ENOTPD (detail = column); every CTA
//   sees it after the next barrier and returns.
//
//   W = L^{-1} by recursive doubling over diagonal blocks (below), in float32
//   or float64 arithmetic. The mixed-precision fit uses float32 here: W
//   feeds the bf16 hi/lo variance contraction, and as the preconditioner of
//   c = A^{-1} b its error is removed by the float64 iterative refinement.
//
//   c = A^{-1} b through W (below); the mixed fit's solve also packs the
//   predict kernel's operand from W and the final c.
#include "gp_kernels.cuh"
#include "gp_tc.cuh"

#include <math.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <map>
#include <mutex>
#include <utility>

namespace {

constexpr int CB = 32;  // Cholesky panel width
constexpr int UT = 16;  // Cholesky trailing-update tile
constexpr int IB = 32;  // inverse block size
constexpr int NT = 256; // threads per CTA
constexpr int NHELP = 16; // CTAs sharing the next diagonal block's update

struct GridBar {
    unsigned int count;
    unsigned int gen;
};

// Bounded grid-wide barrier for a cooperative launch. Returns false (and
// sets GP_ETIMEOUT, detail 100) if the other CTAs do not arrive within
// wait_ns nanoseconds (GP_WAIT_NS unless a test shortened it).
// `count` only grows (zeroed before the launch): the arrivals at the k-th
// barrier are numbers k G .. k G + G - 1, so a CTA learns from its own
// arrival number which total ends the barrier. The arrival is a release
// and the wait an acquire at GPU scope; together with the CTA barriers on
// both sides they order every thread's writes before the barrier with every
// thread's reads after it.
__device__ bool grid_sync(GridBar* gb, GpStatus* st, uint64_t wait_ns = GP_WAIT_NS) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_fail = 0;
        unsigned int old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gb->count) : "memory");
        const unsigned int target = (old / gridDim.x + 1u) * gridDim.x;
        uint64_t t0 = 0;
        uint32_t it = 0;
        while (true) {
            unsigned int cur;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&gb->count) : "memory");
            if ((int)(cur - target) >= 0) break;
            if ((++it & 255u) == 0) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > wait_ns) {
                    gp_set_status(st, GP_ETIMEOUT, 100);
                    s_fail = 1;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return s_fail == 0;
}

// 1 / x in float64 with three dependent FMAs instead of a division, for
// 2^-1022 <= x < 2^1021 (biased exponent 1..2044; callers check the range):
// the seed is the single-precision reciprocal (rcp.approx.f32) of x's leading
// 23 mantissa bits, rescaled by x's exponent, and one step of Halley's
// third-order iteration r <- r (1 + e + e^2), e = 1 - x r, takes its relative
// error from about 2^-22 to below the float64 rounding level (within one ulp
// of the rounded quotient). There is no division fallback on purpose: the
// compiler would evaluate it on every call.
__device__ __forceinline__ double fast_rcp(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int E = (hi >> 20) & 0x7ff;
    const float m = __int_as_float(0x3F800000 | ((hi & 0xFFFFF) << 3) | ((unsigned)lo >> 29));
    float rm;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rm) : "f"(m));
    const int rb = __float_as_int(rm);
    const int shi = ((((rb >> 23) & 0xff) - 127 + 1023) << 20) | ((rb & 0x7FFFFF) >> 3);
    const int slo = rb << 29;
    double r = __hiloint2double(shi - ((E - 1023) << 20), slo);
    const double e = fma(-x, r, 1.0);
    r = fma(r, fma(e, e, e), r);
    return r;
}

__device__ __forceinline__ int status_code(const GpStatus* st) { return *(volatile const int*)&st->code; }

// ---------------------------------------------------------------- Cholesky

// Workspace header (256 bytes, zeroed by launch_cholesky with one memset):
// the Cholesky's grid barrier and its counter of finished next-diagonal-block
// updates, then the grid barriers of the inverse (byte 64) and of the solve
// (byte 128), which run after it on the same workspace; from byte 256 on,
// 1 / L_jj for every j, then the inverse's buffers.
struct CholWork {
    GridBar bar;
    unsigned int helped;
};
constexpr int TRINV_BAR_OFFSET = 64;
constexpr int SOLVE_BAR_OFFSET = 128;
constexpr int CHOL_RSD_OFFSET = 256;

// T = double: the block as it is. T = float (the mixed fit): the block
// equilibrated by powers of two, C = S A_kk S with S = diag(2^-h_i) and h_i =
// floor(log2(a_ii) / 2), so that 1 <= c_ii < 4 and |c_im| < 4 (A_kk is
// positive definite), which float32 holds whatever the range of A (the noise
// diagonal reaches 1e200). Then L_kk = S^-1 L_C.
template <typename T>
struct PotrfSmem {
    T a[CB][CB + 1];                       // the block: lower part updated in place
    T l[2][CB];                            // multipliers a_ij / d_j of the last two pivots
    T pu[2][CB];                           // a_ij a_{j+1,j} of the last two pivots
    T r[2];                                // 1 / d_j of the last two pivots
    T d[CB];                               // pivots d_j
    double s[CB];                          // sqrt(d_j)
    double rs[CB];                         // 1 / sqrt(d_j)
    int h[CB];                             // T = float: the row scales' exponents h_i
    unsigned short tri[CB * (CB + 1) / 2]; // lower entries (i << 8 | m), columns in decreasing order
    int bad;
};

// 2^k as a double, for -1022 <= k <= 1023 (built from its bits).
__device__ __forceinline__ double pow2d(int k) { return __hiloint2double((k + 1023) << 20, 0); }

// Conversions between float64 and float32 with a power-of-two scale, in
// integer operations on the IEEE-754 fields (a float64 conversion or
// multiply holds its scheduler's float64 pipe for 64 clocks on GB300).
// f32_of_f64_pow2: v * 2^k rounded to nearest, ties to even, for |k| <= 1022;
// results below 2^-126 become a signed zero, above the float range or from
// an infinity or NaN an infinity (the pivot check rejects it). These sit on
// the pivot chain and the panel rows, so they are kept branch-light rather
// than built on gp_d2f_rn (which also forms float32 subnormals): that
// version measured 198 against 184 us for the M = 400 factorisation.
__device__ __forceinline__ float f32_of_f64_pow2(double v, int k) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned sign = hi & 0x80000000u;
    const int ed = (int)((hi >> 20) & 0x7ffu);
    int e = ed - 1023 + 127 + k;                                // biased float32 exponent
    unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);         // the leading 23 fraction bits
    const unsigned rest = lo & 0x1FFFFFFFu;                    // the 29 bits below them
    const bool up = rest > 0x10000000u || (rest == 0x10000000u && (m & 1u));
    m += up ? 1u : 0u;
    if (m == 0x800000u) {                                      // rounding carried into the exponent
        m = 0u;
        ++e;
    }
    if (ed == 0 || e <= 0) return __uint_as_float(sign);
    if (ed == 0x7ff || e >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | m);
}

// f64_of_f32_pow2: f * 2^k exactly, for |k| <= 511 (zero and float32
// subnormals give a signed zero; an infinity or NaN stays one).
__device__ __forceinline__ double f64_of_f32_pow2(float f, int k) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const int ef = (int)((b >> 23) & 0xffu);
    if (ef == 0) return __hiloint2double((int)sign, 0);
    const unsigned ex = ef == 0xff ? 0x7ffu : (unsigned)(ef - 127 + 1023 + k);
    const unsigned hi = sign | (ex << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// 1 / x in float32 for a positive normal x below 2^126: the rcp.approx.f32
// estimate (relative error below 2^-22) refined by one Newton-Raphson step,
// r <- r + r (1 - x r), to within about an ulp.
__device__ __forceinline__ float rcp_newton_f32(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// The pivot check on the bits of a float64 or float32 pivot: a positive
// normal number whose reciprocal is normal too ([2^-1022, 2^1021) or
// [2^-126, 2^126)); zero, negative, NaN and infinity fail.
__device__ __forceinline__ bool pivot_ok(double v) {
    const int hi = __double2hiint(v);
    return hi >= 0x00100000 && hi < 0x7FD00000;
}
__device__ __forceinline__ bool pivot_ok(float v) {
    const int b = __float_as_int(v);
    return b >= 0x00800000 && b < 0x7E800000;
}
__device__ __forceinline__ double pivot_rcp(double v) { return fast_rcp(v); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float pivot_rcp(float v) { return rcp_newton_f32(v); }
__device__ __forceinline__ double quiet_nan(double*) { return __longlong_as_double(0x7FF8000000000000ll); }
__device__ __forceinline__ float quiet_nan(float*) { return __int_as_float(0x7FC00000); }

// Named barriers of the pivot loop, each a pair used alternately (pivot j
// takes id + (j & 1)), so an arrival for pivot j + 1 never lands on a barrier
// that pivot j still occupies:
//   COL   chain -> helper     column j is final (in shared memory)
//   PU    helper -> chain     a_ij a_{j+1,j} is ready
//   R     chain -> helper     1 / d_j is ready
//   PUB   helper -> followers the multipliers of pivot j are ready
//   DONE  followers -> chain  pivot j has been applied to the columns >= j + 2
constexpr int POTRF_BAR_COL = 1;
constexpr int POTRF_BAR_PU = 3;
constexpr int POTRF_BAR_R = 5;
constexpr int POTRF_BAR_PUB = 7;
constexpr int POTRF_BAR_DONE = 9;
constexpr int POTRF_FOLLOW = 160;  // follower threads: warps 2, 3, 5, 6, 7
constexpr int POTRF_PAIR_N = 64;                 // chain + helper
constexpr int POTRF_FOLLOW_N = 32 + POTRF_FOLLOW; // (helper or chain) + followers

// Factor the w x w diagonal block at (kb, kb) in place (one CTA, w <= 32),
// right-looking L D L^T in shared memory, in float64 (T = double) or, for
// the mixed fit, in float32 on the equilibrated block (T = float): a float64
// pivot chain costs ~735 clocks a pivot, and the mixed fit already rounds
// its trailing-update products to float32 (errors of the same order) and
// refines c in float64. Every float64 warp instruction
// holds its scheduler's float64 pipe for 64 cycles, so the pivot chain gets a
// scheduler to itself and as few of them as possible: warp 0 (lane i = row i,
// the current pivot column in a register) broadcasts d_j, forms 1 / d_j
// (fast_rcp, three FMAs) and applies pivot j to column j + 1 with one FMA,
// using a_ij a_{j+1,j} that warp 1 (the helper, another scheduler) formed
// meanwhile; the helper then forms the multipliers l_ij = a_ij / d_j for the
// followers. Warps 2, 3 and 5-7 (the other schedulers; warp 4 shares warp
// 0's float64 pipe and stays idle) apply pivot j to the columns m >= j + 2,
// one lower-triangle entry per thread from a packed table, so no float64 lane
// is spent on rows above the diagonal; the chain waits for them only before
// it reads the next column. Control flow does not depend on the data: a
// pivot outside [2^-1022, 2^1021) (zero, negative, NaN, beyond any value a
// Gram matrix plus the clamped noise diagonal reaches) is checked on its
// high word, recorded as GP_ENOTPD and replaced by NaN (a mixed fit then
// redoes its Gram and factorisation in float64). At the end L_jj =
// 2^h_j sqrt(d_j), L_ij = 2^h_i a_ij / sqrt(d_j) and rsd[kb + j] = 1 / L_jj
// (h = 0 for T = double).
template <typename T>
__device__ __forceinline__ bool chol_potrf(double* __restrict__ L, int M, int kb, int w, GpStatus* st,
                                           double* __restrict__ rsd, PotrfSmem<T>& sm) {
    constexpr bool EQ = sizeof(T) == 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NQ = CB * CB / NT;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {  // every load in flight before the first use
        const int e = tid + q * NT, i = e / CB, m = e % CB;
        v[q] = (i < w && m <= i) ? L[(int64_t)(kb + i) * M + kb + m] : 0.0;
    }
    if (EQ) {
        if (tid < CB) {  // h_i = floor(E_i / 2), a_ii in [2^E_i, 2^(E_i + 1)); 0 if a_ii is not positive normal
            const double dii = tid < w ? L[(int64_t)(kb + tid) * M + kb + tid] : 1.0;
            const int hi = __double2hiint(dii);
            const bool pn = hi >= 0x00100000 && hi < 0x7FF00000;
            sm.h[tid] = pn ? ((((hi >> 20) & 0x7ff) - 1023) >> 1) : 0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int e = tid + q * NT, i = e / CB, m = e % CB;
        if (EQ)
            sm.a[i][m] = (T)f32_of_f64_pow2(v[q], -(sm.h[i] + sm.h[m]));  // |h_i + h_m| <= 1022
        else
            sm.a[i][m] = (T)v[q];
    }
    if (tid < w) {  // column m's entries start after those of the columns > m
        const int m = tid;
        const int st0 = (w - m - 1) * (w - m) / 2;
        for (int i = m; i < w; ++i) sm.tri[st0 + i - m] = (unsigned short)((i << 8) | m);
    }
    if (tid == 0) sm.bad = 0;
    __syncthreads();
    if (EQ) {
        // float32: the chain forms the multipliers itself (a float multiply
        // costs it a few clocks, not a float64 pipe slot), so there is no
        // helper; warps 1-7 apply pivot j to the columns >= j + 2, every
        // thread its fixed entries of the packed table (indexes in registers)
        constexpr int NF = NT - 32;
        static_assert(3 * NF >= (CB - 2) * (CB - 1) / 2, "three table entries per follower thread");
        if (warp == 0) {
            T col = sm.a[lane][0];
            for (int j = 0; j < w; ++j) {
                sm.a[lane][j] = col;  // column j is final (every pivot < j applied)
                const T piv = __shfl_sync(0xffffffffu, col, j);
                const T a1 = __shfl_sync(0xffffffffu, col, (j + 1) & 31);  // a_{j+1,j}
                const bool ok = pivot_ok(piv);
                const T r = ok ? pivot_rcp(piv) : quiet_nan((T*)nullptr);
                const T l = (lane > j && lane < w) ? col * r : (T)0;
                sm.l[j & 1][lane] = l;
                if (lane == 0) {
                    sm.d[j] = piv;
                    if (!ok) {
                        sm.bad = 1;
                        gp_set_status(st, GP_ENOTPD, kb + j);
                    }
                }
                __syncwarp();
                named_bar_arrive(POTRF_BAR_PUB + (j & 1), NT);
                if (j + 1 < w) {
                    // the followers have applied pivot j - 1 to the columns >= j + 1
                    if (j >= 1) named_bar_sync(POTRF_BAR_DONE + ((j - 1) & 1), NT);
                    col = fmaT(-l, a1, sm.a[lane][j + 1]);
                }
            }
            for (int q = (w > 2 ? w - 2 : 0); q < w; ++q) named_bar_sync(POTRF_BAR_DONE + (q & 1), NT);
        } else {
            const int ft = tid - 32;
            const int ntri = w * (w + 1) / 2;
            int ei[3], em[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int e = ft + k * NF;
                const unsigned v = e < ntri ? sm.tri[e] : 0u;
                ei[k] = (int)(v >> 8);
                em[k] = (int)(v & 255u);
            }
            for (int j = 0; j < w; ++j) {
                named_bar_sync(POTRF_BAR_PUB + (j & 1), NT);
                const int nc = w - j - 2;
                const int cnt = nc > 0 ? nc * (nc + 1) / 2 : 0;  // entries of the columns m >= j + 2
                const T* lj = sm.l[j & 1];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (ft + k * NF < cnt) sm.a[ei[k]][em[k]] = fmaT(-lj[ei[k]], sm.a[em[k]][j], sm.a[ei[k]][em[k]]);
                named_bar_arrive(POTRF_BAR_DONE + (j & 1), NT);
            }
        }
    } else if (warp == 0) {
        // ---- the pivot chain
        T col = sm.a[lane][0];
        for (int j = 0; j < w; ++j) {
            sm.a[lane][j] = col;  // column j is final (every pivot < j applied)
            __syncwarp();
            named_bar_arrive(POTRF_BAR_COL + (j & 1), POTRF_PAIR_N);
            const T piv = __shfl_sync(0xffffffffu, col, j);
            const bool ok = pivot_ok(piv);
            const T r = ok ? pivot_rcp(piv) : quiet_nan((T*)nullptr);
            if (lane == 0) {
                sm.r[j & 1] = r;
                sm.d[j] = piv;
                if (!ok) {
                    sm.bad = 1;
                    gp_set_status(st, GP_ENOTPD, kb + j);
                }
            }
            __syncwarp();
            named_bar_arrive(POTRF_BAR_R + (j & 1), POTRF_PAIR_N);
            if (j + 1 < w) {
                named_bar_sync(POTRF_BAR_PU + (j & 1), POTRF_PAIR_N);
                // the followers have applied pivot j - 1 to the columns >= j + 1
                if (j >= 1) named_bar_sync(POTRF_BAR_DONE + ((j - 1) & 1), POTRF_FOLLOW_N);
                col = fmaT(-sm.pu[j & 1][lane], r, sm.a[lane][j + 1]);
            }
        }
        for (int q = (w > 2 ? w - 2 : 0); q < w; ++q) named_bar_sync(POTRF_BAR_DONE + (q & 1), POTRF_FOLLOW_N);
    } else if (warp == 1) {
        // ---- the helper: a_ij a_{j+1,j} for the chain, then the multipliers
        for (int j = 0; j < w; ++j) {
            named_bar_sync(POTRF_BAR_COL + (j & 1), POTRF_PAIR_N);
            const T cj = sm.a[lane][j];
            const bool below = lane > j && lane < w;
            if (j + 1 < w) {
                sm.pu[j & 1][lane] = below ? cj * sm.a[j + 1][j] : (T)0;
                __syncwarp();
                named_bar_arrive(POTRF_BAR_PU + (j & 1), POTRF_PAIR_N);
            }
            named_bar_sync(POTRF_BAR_R + (j & 1), POTRF_PAIR_N);
            sm.l[j & 1][lane] = below ? cj * sm.r[j & 1] : (T)0;
            __syncwarp();
            named_bar_arrive(POTRF_BAR_PUB + (j & 1), POTRF_FOLLOW_N);
        }
    } else if (warp != 4) {
        const int ft = (warp < 4 ? warp - 2 : warp - 3) * 32 + lane;
        for (int j = 0; j < w; ++j) {
            named_bar_sync(POTRF_BAR_PUB + (j & 1), POTRF_FOLLOW_N);
            const int nc = w - j - 2;
            const int cnt = nc > 0 ? nc * (nc + 1) / 2 : 0;  // entries of the columns m >= j + 2
            const T* lj = sm.l[j & 1];
            for (int e = ft; e < cnt; e += POTRF_FOLLOW) {
                const unsigned v = sm.tri[e];
                const int i = (int)(v >> 8), m = (int)(v & 255u);
                sm.a[i][m] = fmaT(-lj[i], sm.a[m][j], sm.a[i][m]);
            }
            named_bar_arrive(POTRF_BAR_DONE + (j & 1), POTRF_FOLLOW_N);
        }
    }
    __syncthreads();
    if (sm.bad) return false;  // uniform: read after the barrier
    if (tid < w) {
        if (EQ) {  // float32 square root and reciprocal; d_j is a positive normal float here
            const float sq = sqrtf((float)sm.d[tid]);
            const float rs = rcp_newton_f32(sq);
            sm.s[tid] = f64_of_f32_pow2(sq, sm.h[tid]);
            sm.d[tid] = (T)rs;  // d_j is not needed any more: 1 / sqrt(d_j) for the products below
            rsd[kb + tid] = f64_of_f32_pow2(rs, -sm.h[tid]);
        } else {
            const double sq = sqrt((double)sm.d[tid]);
            const double rs = 1.0 / sq;
            sm.s[tid] = sq;
            sm.rs[tid] = rs;
            rsd[kb + tid] = rs;
        }
    }
    __syncthreads();
    for (int e = tid; e < CB * CB; e += NT) {
        const int i = e / CB, m = e % CB;
        if (i < w && m <= i) {
            double o;
            if (EQ)
                o = (i == m) ? sm.s[m] : f64_of_f32_pow2((float)(sm.a[i][m] * sm.d[m]), sm.h[i]);
            else
                o = (i == m) ? sm.s[m] : (double)sm.a[i][m] * sm.rs[m];
            L[(int64_t)(kb + i) * M + kb + m] = o;
        }
    }
    __syncthreads();
    return true;
}

// L[r0.., c0..] -= L[r0.., kb..kb+w) L[c0.., kb..kb+w)^T on one 16 x 16 lower tile.
__device__ __forceinline__ void chol_update_tile(double* __restrict__ L, int M, int kb, int w, int r0, int c0,
                                 double (*ti)[CB + 1], double (*tj)[CB + 1]) {
    const int tid = threadIdx.x;
    double vi[UT * CB / NT], vj[UT * CB / NT];
#pragma unroll
    for (int q = 0; q < UT * CB / NT; ++q) {  // all loads in flight before the stores
        const int e = tid + q * NT, r = e / CB, l = e % CB;
        vi[q] = (l < w && r0 + r < M) ? L[(int64_t)(r0 + r) * M + kb + l] : 0.0;
        vj[q] = (l < w && c0 + r < M) ? L[(int64_t)(c0 + r) * M + kb + l] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < UT * CB / NT; ++q) {
        const int e = tid + q * NT;
        ti[e / CB][e % CB] = vi[q];
        tj[e / CB][e % CB] = vj[q];
    }
    __syncthreads();
    const int ty = tid / UT, tx = tid % UT;
    double s = 0.0;
    for (int l = 0; l < w; ++l) s = fma(ti[ty][l], tj[tx][l], s);
    const int i = r0 + ty, j = c0 + tx;
    if (i < M && j <= i) L[(int64_t)i * M + j] -= s;
    __syncthreads();
}

// The mixed-precision fit's trailing update (F32): products in float32 on
// 64 x 64 tiles. The panel is rounded to float, each panel's <= 32-term inner
// products are formed in float (about 3e-7 of the products' magnitude, the
// order of the mixed Gram's own error) and subtracted from the float64
// trailing matrix, so rounding does not compound from panel to panel; the
// diagonal blocks and panel solves stay float64. On GB300 a float FMA issues
// 64 times as fast as a float64 one, and these updates are nearly all of the
// M^3 / 3 flops. Each thread owns a 4 x 4 block (rows ty + 16a, columns
// tx + 16b); the tile's old values are loaded with the panel, so a tile
// makes one round trip to L2. Entries above the diagonal and inside the next
// diagonal block (rows and columns base .. base + wn - 1, the helpers' share)
// are left alone.
constexpr int UF = 64;
__device__ __forceinline__ void chol_update_tile_f32(double* __restrict__ L, int M, int kb, int w, int wn,
                                                     int r0, int c0, float (*ti)[CB + 1], float (*tj)[CB + 1]) {
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;
    const int base = kb + w;
    double vi[UF * CB / NT], vj[UF * CB / NT], old[4][4];
#pragma unroll
    for (int q = 0; q < UF * CB / NT; ++q) {
        const int e = tid + q * NT, r = e / CB, l = e % CB;
        vi[q] = (l < w && r0 + r < M) ? L[(int64_t)(r0 + r) * M + kb + l] : 0.0;
        vj[q] = (l < w && c0 + r < M) ? L[(int64_t)(c0 + r) * M + kb + l] : 0.0;
    }
    bool own[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = r0 + ty + 16 * a, j = c0 + tx + 16 * b;
            own[a][b] = i < M && j <= i && !(i - base < wn && j - base < wn);
            old[a][b] = own[a][b] ? L[(int64_t)i * M + j] : 0.0;
        }
#pragma unroll
    for (int q = 0; q < UF * CB / NT; ++q) {
        const int e = tid + q * NT;
        ti[e / CB][e % CB] = gp_d2f_rn(vi[q]);
        tj[e / CB][e % CB] = gp_d2f_rn(vj[q]);
    }
    __syncthreads();
    float acc[4][4] = {};
    for (int l = 0; l < w; ++l) {
        float av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = ti[ty + 16 * a][l];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = tj[tx + 16 * b][l];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (own[a][b])
                L[(int64_t)(r0 + ty + 16 * a) * M + c0 + tx + 16 * b] = old[a][b] - gp_f2d_exact(acc[a][b]);
    __syncthreads();
}

// Share `part` of `nparts` of the next diagonal block's update
// L[r0 + I][r0 + J] -= sum_l L[r0 + I][kb + l] L[r0 + J][kb + l] (J <= I < wn,
// r0 = kb + w): four threads per entry, each summing every fourth l.
__device__ __forceinline__ void chol_next_diag(double* __restrict__ L, int M, int kb, int w, int wn, int part,
                               int nparts, double (*P)[CB + 1]) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int r0 = kb + w;
    double v[CB * CB / NT];
#pragma unroll
    for (int q = 0; q < CB * CB / NT; ++q) {
        const int e = tid + q * NT, r = e / CB, l = e % CB;
        v[q] = (r < wn && l < w) ? L[(int64_t)(r0 + r) * M + kb + l] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < CB * CB / NT; ++q) {
        const int e = tid + q * NT;
        P[e / CB][e % CB] = v[q];
    }
    __syncthreads();
    const int npairs = wn * (wn + 1) / 2;
    const int quarter = tid & 3;
    const unsigned gmask = 0xFu << (lane & ~3);
    for (int p = part + nparts * (tid >> 2); p < npairs; p += nparts * (NT / 4)) {
        int I, J;
        tri_pair(p, &I, &J);
        double s = 0.0;
        for (int l = quarter; l < w; l += 4) s = fma(P[I][l], P[J][l], s);
        s += __shfl_xor_sync(gmask, s, 1);
        s += __shfl_xor_sync(gmask, s, 2);
        if (quarter == 0) L[(int64_t)(r0 + I) * M + r0 + J] -= s;
    }
    __syncthreads();
}

// Right-looking blocked Cholesky with look-ahead. Step k:
//   B  every CTA solves its panel rows (row rr on CTA rr mod G), one warp a row;
//   -- grid barrier --
//   C  CTAs 1..NHELP update the next diagonal block (a share each) and count
//      themselves done; CTA 0 waits for the count and factors that block while
//      CTAs 1..G-1 apply the rest of the trailing update;
//   -- grid barrier --
// wait_ns bounds every wait (GP_WAIT_NS normally). skip_cta >= 0 is a test of
// failure detection only: that CTA leaves before its first barrier arrival,
// so the others' bounded waits run out and report GP_ETIMEOUT.
template <bool F32>
__global__ void __launch_bounds__(NT, 1) chol_coop_kernel(double* __restrict__ L, int M, GpStatus* st,
                                                       CholWork* cw, uint64_t wait_ns, int skip_cta) {
    __shared__ double a[CB][CB + 1];
    // the update tiles' panel rows: 16-row float64 tiles, or 64-row float32 (F32)
    constexpr int TBYTES = F32 ? 2 * UF * (CB + 1) * 4 : 2 * UT * (CB + 1) * 8;
    __shared__ __align__(16) unsigned char tbuf[TBYTES];
    __shared__ double rdiag[CB];
    __shared__ PotrfSmem<typename std::conditional<F32, float, double>::type> sm;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = (M + CB - 1) / CB;
    const int G = gridDim.x;
    const int nh = (G > 1) ? min(NHELP, G - 1) : 1;
    double* rsd = (double*)((char*)cw + CHOL_RSD_OFFSET);
    GridBar* gb = &cw->bar;
    if ((int)blockIdx.x == skip_cta) return;
    if (blockIdx.x == 0) chol_potrf(L, M, 0, min(CB, M), st, rsd, sm);
    if (!grid_sync(gb, st, wait_ns)) return;
    if (status_code(st) != 0) return;
    for (int k = 0; k < nb; ++k) {
        const int kb = k * CB, w = min(CB, M - kb);
        const int rest = M - kb - w;
        if (rest == 0) break;
        // ---- B: panel rows, x L_kk^T = a (lane j owns x_j). With s_j = 1 / L_jj,
        // x_j = a_j s_j - sum_{l<j} x_l (L_jl s_j): lane j holds the scaled row of
        // L_kk in registers, and each step is one shuffle and one FMA. The rows
        // L_jl s_j are scaled once per CTA as they are loaded (a float64
        // instruction holds its scheduler's float64 pipe for 64 cycles, so
        // forming them in every warp cost more than the solves). A mixed fit
        // (F32) solves in float32, each row scaled by 2^-h_i with h_i =
        // floor(log2(a_ii) / 2) of its current diagonal: the row's squared
        // entries sum to less than a_ii, so the scaled x lie below 2 and the
        // scaled L_kk rows are those of the equilibrated block, which
        // float32 holds whatever the noise diagonal's range.
        if ((int)blockIdx.x < rest) {
            double v[CB * CB / NT], sv[CB * CB / NT];
#pragma unroll
            for (int q = 0; q < CB * CB / NT; ++q) {
                const int e = tid + q * NT, i = e / CB, j = e % CB;
                v[q] = (i < w && j <= i) ? L[(int64_t)(kb + i) * M + kb + j] : 0.0;
                sv[q] = i < w ? rsd[kb + i] : 0.0;
            }
            // F32: the scaled rows in float32, converted once per CTA (in the
            // first half of a's storage)
            float(*af)[CB + 1] = reinterpret_cast<float(*)[CB + 1]>(a);
#pragma unroll
            for (int q = 0; q < CB * CB / NT; ++q) {
                const int e = tid + q * NT;
                if (F32)
                    af[e / CB][e % CB] = f32_of_f64_pow2(v[q] * sv[q], 0);
                else
                    a[e / CB][e % CB] = v[q] * sv[q];
            }
            if (tid < CB) rdiag[tid] = tid < w ? rsd[kb + tid] : 0.0;
            __syncthreads();
            const double rd = rdiag[lane];
            using TS = typename std::conditional<F32, float, double>::type;
            TS ls[CB];
            if ((int)blockIdx.x + G * warp < rest) {
#pragma unroll
                for (int l = 0; l < CB; ++l) ls[l] = F32 ? (TS)af[lane][l] : (TS)a[lane][l];
            }
            for (int rr = blockIdx.x + G * warp; rr < rest; rr += G * (NT / 32)) {
                const int gi = kb + w + rr;
                double* row = L + (int64_t)gi * M + kb;
                int h = 0;
                if (F32) {
                    const int dhi = __double2hiint(L[(int64_t)gi * M + gi]);
                    if (dhi >= 0x00100000 && dhi < 0x7FF00000) h = (((dhi >> 20) & 0x7ff) - 1023) >> 1;
                }
                TS acc = (TS)0;
                if (lane < w) acc = F32 ? (TS)f32_of_f64_pow2(row[lane] * rd, -h) : (TS)(row[lane] * rd);
#pragma unroll
                for (int l = 0; l < CB; ++l) {
                    if (l < w) {
                        const TS xl = __shfl_sync(0xffffffffu, acc, l);
                        if (lane > l) acc = fmaT(-xl, ls[l], acc);
                    }
                }
                if (lane < w) row[lane] = F32 ? f64_of_f32_pow2((float)acc, h) : (double)acc;
            }
            __syncthreads();
        }
        if (!grid_sync(gb, st, wait_ns)) return;
        // ---- C
        const int wn = min(CB, rest);              // width of the next diagonal block
        const int ntr = (rest + UT - 1) / UT;
        const int ntiles = ntr * (ntr + 1) / 2;
        const int nd = (wn + UT - 1) / UT;
        const int ndiag = nd * (nd + 1) / 2;       // tiles of the next diagonal block come first
        const bool helper = (G == 1) || ((int)blockIdx.x >= 1 && (int)blockIdx.x <= nh);
        if (helper) {
            chol_next_diag(L, M, kb, w, wn, G == 1 ? 0 : (int)blockIdx.x - 1, nh, a);
            if (G > 1 && tid == 0) {
                __threadfence();
                asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&cw->helped) : "memory");
            }
        }
        if (blockIdx.x == 0) {
            if (G > 1) {
                if (tid == 0) {
                    s_fail = 0;
                    const unsigned int target = (unsigned)nh * (unsigned)(k + 1);
                    const uint64_t t0 = globaltimer_ns();
                    uint32_t it = 0;
                    while (true) {
                        unsigned int cur;
                        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&cw->helped) : "memory");
                        if (cur >= target) break;
                        if ((++it & 1023u) == 0 && globaltimer_ns() - t0 > wait_ns) {
                            gp_set_status(st, GP_ETIMEOUT, 101);
                            s_fail = 1;
                            break;
                        }
                    }
                }
                __syncthreads();
                if (s_fail) return;
            }
            chol_potrf(L, M, kb + w, wn, st, rsd, sm);
        }
        const int first = (G > 1) ? (int)blockIdx.x - 1 : 0;
        const int stride = (G > 1) ? G - 1 : 1;
        if (G == 1 || blockIdx.x > 0) {
            if constexpr (F32) {
                float(*fi)[CB + 1] = reinterpret_cast<float(*)[CB + 1]>(tbuf);
                float(*fj)[CB + 1] = fi + UF;
                const int nfr = (rest + UF - 1) / UF;
                for (int t = first; t < nfr * (nfr + 1) / 2; t += stride) {
                    int I, J;
                    tri_pair(t, &I, &J);
                    chol_update_tile_f32(L, M, kb, w, wn, kb + w + I * UF, kb + w + J * UF, fi, fj);
                }
            } else {
                double(*ti)[CB + 1] = reinterpret_cast<double(*)[CB + 1]>(tbuf);
                double(*tj)[CB + 1] = ti + UT;
                for (int t = ndiag + first; t < ntiles; t += stride) {
                    int I, J;
                    tri_pair(t, &I, &J);
                    chol_update_tile(L, M, kb, w, kb + w + I * UT, kb + w + J * UT, ti, tj);
                }
            }
        }
        if (!grid_sync(gb, st, wait_ns)) return;
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

// W = L^{-1} by recursive doubling, in float32 (mixed precision) or float64
// arithmetic. With L = [L11 0; L21 L22] the inverse is [W11 0; W21 W22],
// W21 = -W22 (L21 W11). Level 0 inverts the LB-row diagonal blocks of L, one
// per CTA and entirely in shared memory (its own doubling over 32-row
// blocks, separated by CTA barriers only); each level h = LB, 2 LB, ... then
// joins every aligned pair of h-row blocks with two tiled GEMM phases over
// all CTAs,
//   A:  X[S][F]  = L[S][F] W[F][F]     (W[F][F] lower triangular)
//   B:  W[S][F]  = -W[S][S] X[S][F]    (W[S][S] lower triangular),
// F = the first h rows of the pair, S the rest. A grid barrier separates the
// phases, so an M x M inverse takes 2 ceil(log2(M / LB)) + 1 phases whose
// tiles run side by side. Every phase also stores the transposes of the
// blocks it completes, so W^T is ready when the last phase ends.
__device__ __forceinline__ float to_t(double x, float*) { return gp_d2f_rn(x); }
__device__ __forceinline__ double to_t(double x, double*) { return x; }

template <typename T>
struct InvGeom;
// A level-0 CTA moves its whole block through one SM, whose own share of
// the L2 bandwidth is small (tens of bytes per clock), so the blocks are kept
// at 64 rows: more CTAs, each with less to move, and one more grid-wide level.
template <>
struct InvGeom<float> {
    static constexpr int LB = 64;   // rows of a level-0 block
    static constexpr int LD = 68;   // row stride of its shared-memory copies
    static constexpr int XD = 36;   // row stride of its X scratch
};
template <>
struct InvGeom<double> {
    static constexpr int LB = 64;
    static constexpr int LD = 66;
    static constexpr int XD = 34;
};
// level 0's buffers, or the 8192-element staging of tile_mm4 if larger
template <typename T>
constexpr size_t trinv_smem_bytes() {
    using G = InvGeom<T>;
    const size_t l0 = 2 * (size_t)G::LB * G::LD + (size_t)(G::LB / 2) * G::XD + G::LB;
    return sizeof(T) * (l0 > 8192 ? l0 : 8192);
}

// four consecutive elements, 16-byte aligned, in shared memory
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Warp-task k of round m for warp w when 8 warps deal the tasks, sorted by
// decreasing cost, in alternating directions (0..7, 7..0, ...), so that
// every warp's total is about the same.
__device__ __forceinline__ int snake_task(int w, int m) { return 8 * m + ((m & 1) ? 7 - w : w); }

// One level h = H of the doubling inside a level-0 block (shared memory):
//   A  X[S][F] = L[S][F] W[F][F]: a warp-task is 32 rows of sX (lane = row)
//      and one column quad j4, so its trip count k = j4 .. H - 1 (W[F][F] is
//      zero above the diagonal) is the same on every lane;
//   B  W[S][F] = -W[S][S] X[S][F]: a warp-task is 32 / (H / 4) adjacent rows
//      (lanes across the rows' column quads), k = 0 .. the last row's index
//      (W[S][S] is zero above the diagonal).
// Both take k in steps of four with 16-byte loads.
template <typename T, int H>
__device__ __forceinline__ void trinv_level0_pairs(const T* sL, T* sW, T* sX) {
    constexpr int LB = InvGeom<T>::LB, LD = InvGeom<T>::LD, XD = InvGeom<T>::XD;
    constexpr int Q = H / 4;                  // column quads of a pair
    constexpr int NP = LB / (2 * H);          // pairs
    constexpr int NRG = LB / 64;              // 32-row groups of sX
    constexpr int NA = NRG * Q;               // A warp-tasks
    constexpr int R = 32 / Q;                 // rows of a B warp-task
    constexpr int NRB = H / R;                // B warp-tasks per pair
    constexpr int NB = NP * NRB;
    static_assert(NA % 8 == 0 || NA < 8, "A tasks");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
    for (int m = 0; m * 8 < NA; ++m) {
        const int k = snake_task(warp, m);
        if (k >= NA) continue;
        const int jq = k / NRG, rg = k % NRG;  // cost H - 4 jq, decreasing in k
        const int gi = rg * 32 + lane, g = gi / H, i = gi % H, j4 = jq * 4;
        const int F0 = 2 * g * H, S0 = F0 + H;
        const T* lrow = sL + (S0 + i) * LD + F0;
        const T* wcol = sW + F0 * LD + F0 + j4;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int k0 = j4; k0 < H; k0 += 4) {
            T l4[4];
            ld4(lrow + k0, l4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                T w4[4];
                ld4(wcol + (k0 + kk) * LD, w4);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] = fma(l4[kk], w4[c], acc[c]);
            }
        }
        st4(sX + gi * XD + j4, acc);
    }
    __syncthreads();
#pragma unroll 1
    for (int m = 0; m * 8 < NB; ++m) {
        const int k = snake_task(warp, m);
        if (k >= NB) continue;
        const int g = k % NP, rb = NRB - 1 - k / NP;  // cost ~ rb, decreasing in k
        const int i = rb * R + lane / Q, j4 = (lane % Q) * 4, imax = rb * R + R - 1;
        const int F0 = 2 * g * H, S0 = F0 + H;
        const T* wrow = sW + (S0 + i) * LD + S0;
        const T* xcol = sX + g * H * XD + j4;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int k0 = 0; k0 <= imax; k0 += 4) {
            T w4[4];
            ld4(wrow + k0, w4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                T x4[4];
                ld4(xcol + (k0 + kk) * XD, x4);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] = fma(w4[kk], x4[c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = -acc[c];
        st4(sW + (S0 + i) * LD + F0 + j4, acc);
    }
    __syncthreads();
}

// Level 0 for the diagonal block of rows R0 .. R0 + wB - 1 (wB <= LB): its
// inverse in sW (LB x LB, stride LD, zero above the diagonal and beyond wB)
// from the block of L, read into sL in T. Diagonal 32-row blocks by forward
// substitution (one warp per block, lane j forms column j in registers),
// then the pairs of h-row blocks, h = 32, 64, .. LB / 2.
template <typename T>
__device__ __forceinline__ void trinv_level0(const double* __restrict__ L, int M, int R0, int wB, T* sL, T* sW, T* sX,
                             T* srd) {
    constexpr int LB = InvGeom<T>::LB, LD = InvGeom<T>::LD;
    constexpr int RPW = LB / 8, SLOTS = LB / 64, RB = 8;  // rows per warp, double2 per lane and row
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the lower triangle of the block of L in T, rows warp + 8 t, 16-byte
    // loads, RB rows' loads in flight; sW = 0
#pragma unroll 1
    for (int t0 = 0; t0 < RPW; t0 += RB) {
        double2 v[RB][SLOTS];
#pragma unroll
        for (int t = 0; t < RB; ++t) {
            const int i = warp + 8 * (t0 + t);
#pragma unroll
            for (int sl = 0; sl < SLOTS; ++sl) {
                const int j = 64 * sl + 2 * lane;
                const double* src = L + (int64_t)(R0 + i) * M + R0 + j;
                // rows of L are 16-byte aligned only when M and R0 are even:
                // take the pair as two loads otherwise
                if (i < wB && j <= i) {
                    if (((M | R0) & 1) == 0) {
                        v[t][sl] = *reinterpret_cast<const double2*>(src);
                        if (j + 1 > i) v[t][sl].y = 0.0;
                    } else {
                        v[t][sl].x = src[0];
                        v[t][sl].y = j + 1 <= i ? src[1] : 0.0;
                    }
                } else {
                    v[t][sl] = make_double2(0.0, 0.0);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < RB; ++t) {
            const int i = warp + 8 * (t0 + t);
#pragma unroll
            for (int sl = 0; sl < SLOTS; ++sl) {
                const int j = 64 * sl + 2 * lane;
                sL[i * LD + j] = to_t(v[t][sl].x, (T*)nullptr);
                sL[i * LD + j + 1] = to_t(v[t][sl].y, (T*)nullptr);
                sW[i * LD + j] = T(0);
                sW[i * LD + j + 1] = T(0);
            }
        }
    }
    __syncthreads();
    if (tid < LB) srd[tid] = tid < wB ? T(1) / sL[tid * LD + tid] : T(0);
    __syncthreads();
    if (warp < LB / IB) {
        // x[k] = 0 above the diagonal, so every row sums over all k < i; rows
        // and columns from wB on come out zero through srd = 0
        const int D0 = warp * IB;
        const T* a = sL + D0 * LD + D0;
        T x[IB];
#pragma unroll
        for (int i = 0; i < IB; ++i) {
            T sum = T(0);
#pragma unroll
            for (int k = 0; k < i; ++k) sum = fma(a[i * LD + k], x[k], sum);
            const T r = srd[D0 + i];
            x[i] = i < lane ? T(0) : (i == lane ? r : -sum * r);
        }
#pragma unroll
        for (int i = 0; i < IB; ++i) sW[(D0 + i) * LD + D0 + lane] = x[i];
    }
    __syncthreads();
    trinv_level0_pairs<T, 32>(sL, sW, sX);
    if constexpr (LB > 64) trinv_level0_pairs<T, 64>(sL, sW, sX);
}

// 32 x 32 tile acc = sum over the 32-wide K chunks kc = k0, k0 + 32, .. < k1
// of A[r0 + i][kc + j] B[kc + j][c0 + l] (rows, columns and k from M on read
// as zero), returned as in a 256-thread layout: thread t holds row t / 8,
// columns 4 (t % 8) .. + 3. Four groups of 64 threads take every fourth
// chunk; each thread forms a 4 x 4 block of its group's partial tile from
// two 16-byte shared-memory reads per k (a column of A, staged transposed,
// and a row of B), and the partial tiles are summed through shared memory.
// The transposed A chunk keeps 4-element groups contiguous and XOR-swizzles
// them by k / 4 (group (i / 4) ^ (k / 4 % 8)), so that the staging stores
// and the reads are free of bank conflicts. Float operands with M % 4 == 0
// are fetched 16 bytes a lane (an SM sustains several times more bytes per
// clock from 16-byte loads than from 4-byte ones); otherwise element-wise.
// Up to KB2 chunks per group are in registers before the first is used.
// sm: 8192 elements of T.
constexpr int KB2 = 2;
__device__ __forceinline__ void group_bar(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }
__device__ __forceinline__ int at_idx(int k, int i) {
    return k * IB + ((((i >> 2) ^ ((k >> 2) & 7)) << 2) | (i & 3));
}
template <typename T, bool VEC>
__device__ __forceinline__ void tile_mm4_run(const T* __restrict__ A, const T* __restrict__ B, int M, int r0,
                                             int c0, int k0, int k1, T (&acc)[4][4], T* At, T* Bs) {
    const int tid = threadIdx.x, grp = tid >> 6, t = tid & 63, w = t >> 5, l = t & 31;
    const int ty4 = t >> 3, tx4 = t & 7;
    constexpr int NL = VEC ? 4 : 16;  // loads of each operand per thread and chunk
    using V = typename std::conditional<VEC, float4, T>::type;
    const int nch = k1 > k0 ? (k1 - k0 + IB - 1) / IB : 0;
    for (int cb = 0; cb < nch; cb += 4 * KB2) {
        V va[KB2][NL], vb[KB2][NL];
#pragma unroll
        for (int u = 0; u < KB2; ++u) {
            const int ch = cb + grp + 4 * u;
            const int kc = k0 + ch * IB;
            const bool in = ch < nch;
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                if constexpr (VEC) {
                    // 4 rows x 128 bytes a warp: row (l / 8) + 4 (2 q + w), 16 bytes at 4 (l % 8)
                    const int i = (l >> 3) + 4 * (2 * q + w), j = 4 * (l & 7);
                    va[u][q] = (in && r0 + i < M && kc + j < M)
                                   ? *reinterpret_cast<const float4*>(A + (int64_t)(r0 + i) * M + kc + j)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    vb[u][q] = (in && kc + i < M && c0 + j < M)
                                   ? *reinterpret_cast<const float4*>(B + (int64_t)(kc + i) * M + c0 + j)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    // A: row (l % 4) + 4 (2 (q / 4) + w), k 4 (l / 4) + q % 4; B: k 2 q + w, column l
                    const int i = (l & 3) + 4 * (2 * (q >> 2) + w), j = 4 * (l >> 2) + (q & 3);
                    va[u][q] = (in && r0 + i < M && kc + j < M) ? A[(int64_t)(r0 + i) * M + kc + j] : T(0);
                    const int bi = 2 * q + w;
                    vb[u][q] = (in && kc + bi < M && c0 + l < M) ? B[(int64_t)(kc + bi) * M + c0 + l] : T(0);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < KB2; ++u) {
            if (cb + grp + 4 * u >= nch) break;  // uniform within the group
            group_bar(1 + grp);                   // the group's last chunk is consumed
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                if constexpr (VEC) {
                    const int i = (l >> 3) + 4 * (2 * q + w), j = 4 * (l & 7);
                    At[at_idx(j, i)] = va[u][q].x;
                    At[at_idx(j + 1, i)] = va[u][q].y;
                    At[at_idx(j + 2, i)] = va[u][q].z;
                    At[at_idx(j + 3, i)] = va[u][q].w;
                    *reinterpret_cast<float4*>(Bs + i * IB + j) = vb[u][q];
                } else {
                    const int i = (l & 3) + 4 * (2 * (q >> 2) + w), j = 4 * (l >> 2) + (q & 3);
                    At[at_idx(j, i)] = va[u][q];
                    Bs[(2 * q + w) * IB + l] = vb[u][q];
                }
            }
            group_bar(1 + grp);
#pragma unroll 8
            for (int k = 0; k < IB; ++k) {
                T a4[4], b4[4];
                ld4(At + at_idx(k, 4 * ty4), a4);
                ld4(Bs + k * IB + 4 * tx4, b4);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fma(a4[r], b4[c], acc[r][c]);
            }
        }
    }
}
template <typename T>
__device__ __forceinline__ void tile_mm4(const T* __restrict__ A, const T* __restrict__ B, int M, int r0, int c0,
                                         int k0, int k1, T (&out)[4], T* sm) {
    const int tid = threadIdx.x, grp = tid >> 6, t = tid & 63;
    const int ty4 = t >> 3, tx4 = t & 7;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
    T* At = sm + grp * 2 * IB * IB;
    T* Bs = At + IB * IB;
    if (sizeof(T) == 4 && (M & 3) == 0) {
        if constexpr (sizeof(T) == 4) tile_mm4_run<T, true>(A, B, M, r0, c0, k0, k1, acc, At, Bs);
    } else {
        tile_mm4_run<T, false>(A, B, M, r0, c0, k0, k1, acc, At, Bs);
    }
    __syncthreads();
    // partial tiles red[grp][row][col] (stride 33) over the staging buffers
    T* red = sm + grp * IB * (IB + 1);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) red[(4 * ty4 + r) * (IB + 1) + 4 * tx4 + c] = acc[r][c];
    __syncthreads();
    const int ry = tid >> 3, rx = (tid & 7) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        T v = T(0);
#pragma unroll
        for (int g = 0; g < 4; ++g) v += sm[g * IB * (IB + 1) + ry * (IB + 1) + rx + c];
        out[c] = v;
    }
    __syncthreads();
}

// Lt: L in the arithmetic type T (converted here when T is float; L itself
// when T is double); Wt: the result W in T (the float64 output itself when T
// is double; the float32 fit keeps no float64 copy); X: M x M scratch.
// At the end WT (Lt's buffer when T is float, X's when T is double) holds
// W^T in T on and above the diagonal, for the solve's W^T t; below it, WT is
// whatever the buffer held (the parts of L and X the phases used).
template <typename T>
__global__ void __launch_bounds__(NT) trinv_rec_kernel(const double* __restrict__ L, int M,
                                                       T* __restrict__ Lt, T* __restrict__ Wt,
                                                       T* __restrict__ X, T* __restrict__ WT, GpStatus* st,
                                                       GridBar* gb) {
    constexpr int LB = InvGeom<T>::LB, LD = InvGeom<T>::LD, XD = InvGeom<T>::XD;
    __shared__ T sa[IB][IB + 1];
    extern __shared__ __align__(16) unsigned char inv_raw[];
    T* sdyn = reinterpret_cast<T*>(inv_raw);  // level 0, then the tile products
    T* sL = sdyn;
    T* sW = sL + LB * LD;
    T* sX = sW + LB * LD;
    T* srd = sX + (LB / 2) * XD;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, ty = tid >> 3, tx = (tid & 7) * 4;
    const int G = gridDim.x;
    constexpr bool conv = sizeof(T) != sizeof(double);
    // ---- level 0: diagonal LB blocks (CTAs 0 .. nlb - 1), and outside them
    // zeros above the diagonal and L in T below it (the other CTAs, if any)
    const int nlb = (M + LB - 1) / LB;
    for (int b = blockIdx.x; b < nlb; b += G) {
        const int R0 = b * LB, wB = min(LB, M - R0);
        trinv_level0<T>(L, M, R0, wB, sL, sW, sX, srd);
        // the lower triangle of W and Wt (row i = warp + 8 t), and W^T above
        // the diagonal (row c, lanes across r >= c; the column reads of sW
        // cost a 4-way bank conflict, less than staging 32 x 32 transposes)
        for (int i = warp; i < wB; i += NT / 32) {
            for (int j = lane; j <= i; j += 32) {
                const int64_t o = (int64_t)(R0 + i) * M + R0 + j;
                Wt[o] = sW[i * LD + j];
            }
        }
        for (int c = warp; c < wB; c += NT / 32) {
            for (int r = c + lane; r < wB; r += 32) WT[(int64_t)(R0 + c) * M + R0 + r] = sW[r * LD + c];
        }
        __syncthreads();
    }
    {
        // CTAs nlb .. G - 1 (all, if there are no more than nlb): zeros above
        // the diagonal, L in T below the level-0 blocks
        const int c0 = G > nlb ? nlb : 0, nc = G - c0;
        if (blockIdx.x >= c0) {
            for (int i = (blockIdx.x - c0) * (NT / 32) + warp; i < M; i += nc * (NT / 32)) {
                const int bi = i / LB;
                const int64_t ro = (int64_t)i * M;
                for (int j = lane; j < M; j += 32) {
                    if (j > i) {
                        Wt[ro + j] = T(0);
                    } else if (conv && j / LB < bi) {
                        Lt[ro + j] = to_t(L[ro + j], (T*)nullptr);
                    }
                }
            }
        }
    }
    if (LB >= M) return;
    if (!grid_sync(gb, st)) return;
    const T* Lr = conv ? Lt : reinterpret_cast<const T*>(L);
    for (int h = LB; h < M; h *= 2) {
        const int hb = h / IB;                     // blocks per half
        const int ng = (M + 2 * h - 1) / (2 * h);  // pairs at this level
        const int ntile = ng * hb * hb;            // (S block, F block) tiles, full pairs
        // ---- A: X[S][F] = L[S][F] W[F][F]
        for (int t = blockIdx.x; t < ntile; t += G) {
            const int g = t / (hb * hb), si = (t / hb) % hb, fj = t % hb;
            const int F0 = g * 2 * h, S0 = F0 + h;
            const int r0 = S0 + si * IB, c0 = F0 + fj * IB;
            if (r0 >= M) continue;
            T acc[4] = {T(0), T(0), T(0), T(0)};
            tile_mm4<T>(Lr, Wt, M, r0, c0, c0, S0, acc, sdyn);  // W[k][c0..] = 0 for k < c0
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (r0 + ty < M) X[(int64_t)(r0 + ty) * M + c0 + tx + c] = acc[c];
        }
        if (!grid_sync(gb, st)) return;
        // ---- B: W[S][F] = -W[S][S] X[S][F], and its transpose into WT[F][S]
        for (int t = blockIdx.x; t < ntile; t += G) {
            const int g = t / (hb * hb), si = (t / hb) % hb, fj = t % hb;
            const int F0 = g * 2 * h, S0 = F0 + h;
            const int r0 = S0 + si * IB, c0 = F0 + fj * IB;
            if (r0 >= M) continue;
            T acc[4] = {T(0), T(0), T(0), T(0)};
            tile_mm4<T>(Wt, X, M, r0, c0, S0, min(r0 + IB, M), acc, sdyn);  // W[r][k] = 0 for k > r
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t o = (int64_t)(r0 + ty) * M + c0 + tx + c;
                if (r0 + ty < M) Wt[o] = -acc[c];
                sa[tx + c][ty] = -acc[c];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < IB * IB / NT; ++q) {
                const int e = tid + q * NT, i = e / IB, j = e % IB;
                if (r0 + j < M) WT[(int64_t)(c0 + i) * M + r0 + j] = sa[i][j];
            }
            // the next tile_mm4's barriers order these reads before sa is written again
        }
        if (2 * h < M && !grid_sync(gb, st)) return;
    }
}

// ---------------------------------------------------------------- c = A^{-1} b

// c = W^T (W b), then `refine` steps of c += W^T W (b - A c): the residual
// and c in float64; the products with W in T (float32 for the mixed fit,
// whose W is float32-accurate, so float32 products lose nothing the
// refinement would keep). One cooperative launch, a grid barrier between
// phases, every phase a warp per row:
//   Wv   t_i = sum_{j <= i} W_ij v_j
//   WTt  c_j (+)= sum_{i >= j} (W^T)_ji t_i     (W^T from the inverse)
//   res  r_i = b_i - sum_j A_ij c_j              (float64)
//
// A mixed fit (Wpack != NULL) also leaves the predict kernel's operands: the
// packed bf16 hi/lo blocks of the float32 W, written in the first phase (W is
// complete before this launch), and c in float32 after them, written with
// the final c.
template <typename T>
__global__ void __launch_bounds__(NT) solve_coop_kernel(const double* __restrict__ A, const T* __restrict__ W,
                                                        const T* __restrict__ WT, const double* __restrict__ b,
                                                        double* __restrict__ c, T* __restrict__ t,
                                                        T* __restrict__ r, int M, int refine, GpStatus* st,
                                                        GridBar* gb, uint8_t* __restrict__ Wpack, int Mpad) {
    if (status_code(st) != 0) return;  // set before this launch: every CTA leaves
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x;
    // row . vector over [lo, hi) by one warp, eight loads per lane in flight
    auto dotrow = [&](const T* row, const T* v, int lo, int hi) -> T {
        T s = T(0);
        for (int j0 = lo; j0 < hi; j0 += 32 * 8) {
            T a[8], x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + 32 * u + lane;
                a[u] = j < hi ? row[j] : T(0);
                x[u] = j < hi ? v[j] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) s = fma(a[u], x[u], s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
    };
    auto w_apply = [&](const T* v) {
        for (int i = blockIdx.x * (NT / 32) + warp; i < M; i += G * (NT / 32)) {
            const T s = dotrow(W + (int64_t)i * M, v, 0, i + 1);
            if (lane == 0) t[i] = s;
        }
    };
    float* cf = Wpack != nullptr ? reinterpret_cast<float*>(Wpack + (size_t)4 * Mpad * Mpad) : nullptr;
    auto wt_apply = [&](bool accumulate, bool last) {
        for (int j = blockIdx.x * (NT / 32) + warp; j < M; j += G * (NT / 32)) {
            const T s = dotrow(WT + (int64_t)j * M, t, j, M);
            if (lane == 0) {
                const double cj = (accumulate ? c[j] : 0.0) + (double)s;
                c[j] = cj;
                if constexpr (sizeof(T) == 4) {
                    if (last && cf != nullptr) cf[j] = (float)cj;
                }
            }
        }
    };
    for (int i = blockIdx.x * NT + tid; i < M; i += G * NT) r[i] = (T)b[i];
    if constexpr (sizeof(T) == 4) {
        if (Wpack != nullptr) {
            const int64_t items = pack_w_items(Mpad);
            for (int64_t i = (int64_t)blockIdx.x * NT + tid; i < items; i += (int64_t)G * NT)
                pack_w_item(W, M, Mpad, Wpack, i);
            for (int i = M + blockIdx.x * NT + tid; i < Mpad; i += G * NT) cf[i] = 0.f;
        }
    }
    if (!grid_sync(gb, st)) return;
    w_apply(r);
    if (!grid_sync(gb, st)) return;
    wt_apply(false, refine == 0);
    for (int it = 0; it < refine; ++it) {
        if (!grid_sync(gb, st)) return;
        for (int i = blockIdx.x * (NT / 32) + warp; i < M; i += G * (NT / 32)) {
            const double* row = A + (int64_t)i * M;
            double s = 0.0;
            for (int j0 = 0; j0 < M; j0 += 32 * 8) {
                double a[8], x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = j0 + 32 * u + lane;
                    a[u] = j < M ? row[j] : 0.0;
                    x[u] = j < M ? c[j] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) s = fma(a[u], x[u], s);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) r[i] = (T)(b[i] - s);
        }
        if (!grid_sync(gb, st)) return;
        w_apply(r);
        if (!grid_sync(gb, st)) return;
        wt_apply(true, it + 1 == refine);
    }
}

// CTAs of a cooperative launch of `kern` (one per SM) with `smem` bytes of
// dynamic shared memory (allowed beyond 48 KB here), cached per kernel and
// device: the occupancy query costs more host time than the launch itself.
int coop_grid(const void* kern, int dev, size_t smem = 0) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({kern, dev});
        if (it != cache.end()) return it->second;
    }
    int sms = 1, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
    if (occ < 1) occ = 1;
    const int g = sms * (occ < 2 ? occ : 1);
    std::lock_guard<std::mutex> lk(mu);
    cache[{kern, dev}] = g;
    return g;
}

}  // namespace

size_t factor_work_bytes(int M, bool fp32_inverse) {
    // inverse: L and W in float32 plus X (mixed), or X alone (float64)
    const size_t inv = fp32_inverse ? 3 * sizeof(float) * (size_t)M * M : sizeof(double) * (size_t)M * M;
    const size_t chol = sizeof(double) * (size_t)M;  // 1 / L_jj
    return CHOL_RSD_OFFSET + (inv > chol ? inv : chol);
}

// A grid capped at max_ctas (> 0), never below lo: the batched fit runs many
// problems' factorisations side by side, each on a few CTAs (every phase of
// these kernels walks its work with grid strides, so any grid size is correct).
int cap_grid(int g, int max_ctas, int lo = 1) {
    if (max_ctas > 0 && g > max_ctas) g = max_ctas;
    return g < lo ? lo : g;
}

// CTAs for the Cholesky of an M x M matrix: about two trailing-update tiles
// per CTA in the first step (one CTA when there is none), at most one per SM,
// so that small problems -- e.g. the many problems of a batch running side by
// side -- do not claim the whole GPU.
int chol_grid(int M, int dev, bool f32_update) {
    if (M <= CB) return 1;
    // about two 16-row (one 64-row, float32) trailing-update tiles per CTA in
    // the first step; with float32 tiles also at least one panel row per warp
    // (the float64 panel solves then set the step time at small M)
    const int T = f32_update ? (M - CB + UF - 1) / UF : (M - CB + UT - 1) / UT;
    const int want = f32_update ? std::max(T * (T + 1) / 2, (M - CB + NT / 32 - 1) / (NT / 32))
                                : (T * (T + 1) / 2 + 1) / 2;
    const int g = coop_grid((const void*)chol_coop_kernel<false>, dev);
    return want < 2 ? 2 : (want > g ? g : want);
}

namespace {
// failure-detection test hooks (gp_debug_barrier_timeout)
std::atomic<unsigned long long> g_chol_wait_ns{0};  // 0: GP_WAIT_NS
std::atomic<int> g_chol_skip_cta{-1};               // one-shot
}  // namespace

void factor_debug_barrier_timeout(double limit_s, int skip_cta) {
    g_chol_wait_ns.store(limit_s > 0.0 ? (unsigned long long)(limit_s * 1e9) : 0ull);
    g_chol_skip_cta.store(skip_cta >= 0 ? skip_cta : -1);
}

cudaError_t launch_cholesky(double* L, int M, GpStatus* st, void* work, cudaStream_t stream, bool f32_update,
                            int max_ctas) {
    int dev = 0;
    cudaGetDevice(&dev);
    CholWork* cw = (CholWork*)work;
    cudaMemsetAsync(cw, 0, CHOL_RSD_OFFSET, stream);
    dim3 grid((unsigned)cap_grid(chol_grid(M, dev, f32_update), max_ctas, M > CB ? 2 : 1)), block(NT);
    const unsigned long long lim = g_chol_wait_ns.load();
    uint64_t wait_ns = lim ? (uint64_t)lim : (uint64_t)GP_WAIT_NS;
    int skip = g_chol_skip_cta.exchange(-1);
    void* args[] = {&L, &M, &st, &cw, &wait_ns, &skip};
    gp_note_launches(1);
    const void* k = f32_update ? (const void*)chol_coop_kernel<true> : (const void*)chol_coop_kernel<false>;
    return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
}

namespace {
// widest phase of the inverse: the diagonal blocks of level 0, or the tiles
// of the last level's pairs
int trinv_want(int M, int LB) {
    const int nlb = (M + LB - 1) / LB;
    if (LB >= M) return nlb;
    int hmax = LB;
    while (hmax * 2 < M) hmax *= 2;
    const int hb = hmax / IB;
    return std::max(nlb, ((M + 2 * hmax - 1) / (2 * hmax)) * hb * hb);
}
}  // namespace

cudaError_t launch_tri_inverse(const double* L, double* W, int M, bool fp32, GpStatus* st, void* work,
                               cudaStream_t stream, int max_ctas) {
    int dev = 0;
    cudaGetDevice(&dev);
    GridBar* gb = (GridBar*)((char*)work + TRINV_BAR_OFFSET);  // zeroed by launch_cholesky
    char* base = (char*)work + CHOL_RSD_OFFSET;
    gp_note_launches(1);
    const size_t M2 = (size_t)M * M;
    if (fp32) {
        float* Lt = (float*)base;
        float* Wt = Lt + M2;
        float* X = Wt + M2;
        float* WT = Lt;  // W^T goes where L in float is no longer read
        const void* k = (const void*)trinv_rec_kernel<float>;
        const size_t smem = trinv_smem_bytes<float>();
        dim3 grid((unsigned)cap_grid(std::min(trinv_want(M, InvGeom<float>::LB), coop_grid(k, dev, smem)), max_ctas)),
            block(NT);
        void* args[] = {(void*)&L, &M, &Lt, &Wt, &X, &WT, &st, &gb};
        return cudaLaunchCooperativeKernel(k, grid, block, args, smem, stream);
    }
    double* Lt = nullptr;
    double* Wt = W;
    double* X = (double*)base;
    double* WT = X;  // above the diagonal, where X is never used
    const void* k = (const void*)trinv_rec_kernel<double>;
    const size_t smem = trinv_smem_bytes<double>();
    dim3 grid((unsigned)cap_grid(std::min(trinv_want(M, InvGeom<double>::LB), coop_grid(k, dev, smem)), max_ctas)),
        block(NT);
    void* args[] = {(void*)&L, &M, &Lt, &Wt, &X, &WT, &st, &gb};
    return cudaLaunchCooperativeKernel(k, grid, block, args, smem, stream);
}

size_t solve_refine_work_elems(int M) {
    return 32 + 2 * (size_t)M;  // 256 bytes unused (alignment), t, r
}

cudaError_t launch_solve_refine(const double* A, const double* W, const void* fwork, bool fp32, const double* b,
                                double* c, double* work, int M, int refine, GpStatus* st, cudaStream_t stream,
                                uint16_t* Wpack, int max_ctas) {
    uint8_t* wp = fp32 ? reinterpret_cast<uint8_t*>(Wpack) : nullptr;
    int Mpad = (int)gp_round_up(M, PREDTC_KB);
    int dev = 0;
    cudaGetDevice(&dev);
    GridBar* gb = (GridBar*)((char*)const_cast<void*>(fwork) + SOLVE_BAR_OFFSET);  // zeroed by launch_cholesky
    const int want = (M + NT / 32 - 1) / (NT / 32);
    gp_note_launches(1);
    const char* fbase = (const char*)fwork + CHOL_RSD_OFFSET;
    if (fp32) {
        // the float32 W and W^T left in the inverse's workspace
        const float* WTf = (const float*)fbase;
        const float* Wf = WTf + (size_t)M * M;
        float* t = (float*)(work + 32);
        float* r = t + M;
        const void* k = (const void*)solve_coop_kernel<float>;
        dim3 grid((unsigned)cap_grid(std::min(want, coop_grid(k, dev)), max_ctas)), block(NT);
        void* args[] = {(void*)&A, (void*)&Wf, (void*)&WTf, (void*)&b, &c, &t, &r, &M, &refine, &st, &gb, &wp, &Mpad};
        return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
    }
    const double* WTd = (const double*)fbase;
    double* t = work + 32;
    double* r = t + M;
    const void* k = (const void*)solve_coop_kernel<double>;
    dim3 grid((unsigned)cap_grid(std::min(want, coop_grid(k, dev)), max_ctas)), block(NT);
    void* args[] = {(void*)&A, (void*)&W, (void*)&WTd, (void*)&b, &c, &t, &r, &M, &refine, &st, &gb, &wp, &Mpad};
    return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
}
