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
constexpr int NHELP = 16; // CTAs sharing the next diagonal block's update

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

// Cholesky workspace header: the grid barrier, the counter of finished
// next-diagonal-block updates, then (from byte 256) 1 / L_jj for every j.
struct CholWork {
    GridBar bar;
    unsigned int helped;
};
constexpr int CHOL_RSD_OFFSET = 256;

constexpr int PSLOT = 4;  // pivot slots (the owner of pivot j reuses the slot of pivot j - 4)

struct PotrfSmem {
    uint64_t full[PSLOT];   // slot s holds pivot j (j mod PSLOT = s): arrives when u and r are written
    uint64_t empty[PSLOT];  // every warp arrives once it has applied that pivot to its columns
    double u[PSLOT][CB];    // pivot column j after steps < j (lane i: a_ij)
    double l[PSLOT][CB];    // multipliers a_ij / d_j (i > j; 0 elsewhere)
    double r[PSLOT];        // 1 / d_j
    double d[CB];       // pivots d_j
    double s[CB];       // sqrt(d_j)
    double rs[CB];      // 1 / sqrt(d_j)
    int bad;
    int fail;
};

// Named barriers of the pivot chain: U(s) hands the pivot column of slot s,
// R(s) its reciprocal, from the owner of pivot j to the owner of pivot j + 1.
constexpr int POTRF_BAR_U = 1;           // ids 1..PSLOT
constexpr int POTRF_BAR_R = 1 + PSLOT;   // ids PSLOT+1..2 PSLOT

// col[q] (column warp + 8q) -= l[lane] u[column] for the owned columns m > mlo.
__device__ __forceinline__ void potrf_apply(double (&col)[4], const double* l, const double* u, int mlo,
                                            int w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double lv = l[lane];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = warp + 8 * q;
        if (m > mlo && m < w) col[q] = fma(-lv, u[m], col[q]);
    }
}

// The owner of pivot j publishes column j (already updated by all earlier
// pivots) and then its reciprocal. A pivot outside [2^-1022, 2^1021) -- zero,
// negative, NaN, or beyond any value a Gram matrix plus the clamped noise
// diagonal reaches -- is checked on the high word (no float64 instruction),
// recorded as not positive definite and replaced by NaN, so control flow
// never depends on the data.
__device__ __forceinline__ void potrf_publish(double v, int j, int w, int kb, GpStatus* st, PotrfSmem& sm,
                                              bool handoff) {
    const int lane = threadIdx.x & 31;
    const int sl = j % PSLOT;
    sm.u[sl][lane] = v;
    __syncwarp();
    if (handoff) named_bar_arrive(POTRF_BAR_U + sl, 64);
    const double piv = __shfl_sync(0xffffffffu, v, j);
    const int hi = __double2hiint(piv);
    const bool ok = hi >= 0x00100000 && hi < 0x7FD00000;
    const double r = ok ? fast_rcp(piv) : __longlong_as_double(0x7FF8000000000000ll);
    if (lane == 0) {
        sm.r[sl] = r;
        sm.d[j] = piv;
        if (!ok) {
            sm.bad = 1;
            gp_set_status(st, GP_ENOTPD, kb + j);
        }
    }
    __syncwarp();
    if (handoff) named_bar_arrive(POTRF_BAR_R + sl, 64);
    // the multipliers, once, for every warp that applies this pivot
    sm.l[sl][lane] = (lane > j && lane < w) ? v * r : 0.0;
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.full[sl]);
}

// Factor the w x w diagonal block at (kb, kb) in place (one CTA, w <= 32).
// Right-looking L D L^T elimination in registers: lane i holds row i, warp
// q owns columns q, q + 8, q + 16, q + 24, and pivot j subtracts
// (a_ij / d_j) a_mj from every later column m. The critical path is the chain
// of pivots, so it is cut to one reciprocal and one FMA per pivot: the owner
// of pivot j publishes column j before forming 1 / d_j, the owner of pivot
// j + 1 multiplies a_ij a_{j+1,j} meanwhile and, once the reciprocal arrives,
// finishes its column with one FMA and publishes it in turn. These handoffs
// use pairs of named barriers; the other warps follow through PSLOT pivot
// slots guarded by mbarriers (bounded waits), applying each pivot to their
// columns off the critical path. The owner of pivot j + 2 applies pivot j
// to that column alone and the rest of its columns after its own turn, so it
// is never late for the chain. Every warp runs the same sequence of
// barrier operations whatever the data, so nothing can wait for an arrival
// that never comes. At the end L_jj = sqrt(d_j), L_ij = a_ij / sqrt(d_j) and
// rsd[kb + j] = 1 / L_jj. Returns false on a non-positive pivot (GP_ENOTPD)
// or an expired wait (GP_ETIMEOUT).
__device__ __forceinline__ bool chol_potrf(double* __restrict__ L, int M, int kb, int w, GpStatus* st,
                                           double* __restrict__ rsd, PotrfSmem& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double col[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = warp + 8 * q;
        col[q] = (m < w && lane < w && lane >= m) ? L[(int64_t)(kb + lane) * M + kb + m] : 0.0;
    }
    if (tid == 0) {
        sm.bad = 0;
        sm.fail = 0;
        for (int q = 0; q < PSLOT; ++q) {
            mbar_init(&sm.full[q], 1);
            mbar_init(&sm.empty[q], NT / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) potrf_publish(col[0], 0, w, kb, st, sm, w > 1);
    int pend = -1;  // pivot this warp has applied to its next pivot column only
    for (int j = 0; j + 1 < w; ++j) {
        const int sl = j % PSLOT, jn = j + 1, sn = jn % PSLOT;
        if (warp == (jn & 7)) {
            // ---- the pivot chain: finish column jn and publish it
            named_bar_sync(POTRF_BAR_U + sl, 64);
            const double p = sm.u[sl][lane] * sm.u[sl][jn];
            // slot sn last held pivot jn - PSLOT: every warp must be done with it
            if (jn >= PSLOT && !*(volatile int*)&sm.fail &&
                !mbar_wait(&sm.empty[sn], (uint32_t)(jn / PSLOT - 1) & 1u)) {
                if (lane == 0) {
                    sm.fail = 1;
                    gp_set_status(st, GP_ETIMEOUT, 103);
                }
            }
            named_bar_sync(POTRF_BAR_R + sl, 64);
            const double r = sm.r[sl];
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q == (jn >> 3)) {
                    col[q] = fma(-p, r, col[q]);
                    v = col[q];
                }
            potrf_publish(v, jn, w, kb, st, sm, jn + 1 < w);
            // then the rest of this warp's columns (all > jn): pivot j - 1 if put
            // off, and pivot j
            if (pend >= 0) {
                const int sp = pend % PSLOT;
                potrf_apply(col, sm.l[sp], sm.u[sp], jn, w);
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[sp]);
                pend = -1;
            }
            // pivot j's multipliers were written after its reciprocal's handoff
            if (!*(volatile int*)&sm.fail && !mbar_wait(&sm.full[sl], (uint32_t)(j / PSLOT) & 1u)) {
                if (lane == 0) {
                    sm.fail = 1;
                    gp_set_status(st, GP_ETIMEOUT, 104);
                }
            }
            potrf_apply(col, sm.l[sl], sm.u[sl], jn, w);
        } else {
            // ---- follow pivot j
            if (!*(volatile int*)&sm.fail && !mbar_wait(&sm.full[sl], (uint32_t)(j / PSLOT) & 1u)) {
                if (lane == 0) {
                    sm.fail = 1;
                    gp_set_status(st, GP_ETIMEOUT, 102);
                }
            }
            const int jnn = jn + 1;
            if (jnn < w && warp == (jnn & 7)) {
                // owner of the next pivot: column jnn now, the others after its turn
                const double lv = sm.l[sl][lane];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q == (jnn >> 3)) col[q] = fma(-lv, sm.u[sl][jnn], col[q]);
                pend = j;
                continue;  // its empty arrival for pivot j comes with the deferred update
            }
            potrf_apply(col, sm.l[sl], sm.u[sl], j, w);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[sl]);
    }
    __syncthreads();
    if (sm.bad || sm.fail) return false;  // uniform: read after the barrier
    if (tid < w) {
        const double sq = sqrt(sm.d[tid]);
        const double rs = 1.0 / sq;
        sm.s[tid] = sq;
        sm.rs[tid] = rs;
        rsd[kb + tid] = rs;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = warp + 8 * q;
        if (m < w && lane < w && lane >= m)
            L[(int64_t)(kb + lane) * M + kb + m] = (lane == m) ? sm.s[m] : col[q] * sm.rs[m];
    }
    __syncthreads();
    return true;
}

// L[r0.., c0..] -= L[r0.., kb..kb+w) L[c0.., kb..kb+w)^T on one 16 x 16 lower tile.
__device__ void chol_update_tile(double* __restrict__ L, int M, int kb, int w, int r0, int c0,
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

// Share `part` of `nparts` of the next diagonal block's update
// L[r0 + I][r0 + J] -= sum_l L[r0 + I][kb + l] L[r0 + J][kb + l] (J <= I < wn,
// r0 = kb + w): four threads per entry, each summing every fourth l.
__device__ void chol_next_diag(double* __restrict__ L, int M, int kb, int w, int wn, int part,
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
__global__ void __launch_bounds__(NT) chol_coop_kernel(double* __restrict__ L, int M, GpStatus* st,
                                                       CholWork* cw) {
    __shared__ double a[CB][CB + 1];
    __shared__ double ti[UT][CB + 1];
    __shared__ double tj[UT][CB + 1];
    __shared__ double rdiag[CB];
    __shared__ PotrfSmem sm;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = (M + CB - 1) / CB;
    const int G = gridDim.x;
    const int nh = (G > 1) ? min(NHELP, G - 1) : 1;
    double* rsd = (double*)((char*)cw + CHOL_RSD_OFFSET);
    GridBar* gb = &cw->bar;
    if (blockIdx.x == 0) chol_potrf(L, M, 0, min(CB, M), st, rsd, sm);
    if (!grid_sync(gb, st)) return;
    if (status_code(st) != 0) return;
    for (int k = 0; k < nb; ++k) {
        const int kb = k * CB, w = min(CB, M - kb);
        const int rest = M - kb - w;
        if (rest == 0) break;
        // ---- B: panel rows, x L_kk^T = a (lane j owns x_j). With s_j = 1 / L_jj,
        // x_j = a_j s_j - sum_{l<j} x_l (L_jl s_j): lane j holds the scaled row of
        // L_kk in registers, and each step is one shuffle and one FMA.
        if ((int)blockIdx.x < rest) {
            double v[CB * CB / NT];
#pragma unroll
            for (int q = 0; q < CB * CB / NT; ++q) {
                const int e = tid + q * NT, i = e / CB, j = e % CB;
                v[q] = (i < w && j <= i) ? L[(int64_t)(kb + i) * M + kb + j] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < CB * CB / NT; ++q) {
                const int e = tid + q * NT;
                a[e / CB][e % CB] = v[q];
            }
            if (tid < CB) rdiag[tid] = tid < w ? rsd[kb + tid] : 0.0;
            __syncthreads();
            const double rd = rdiag[lane];
            double ls[CB];
#pragma unroll
            for (int l = 0; l < CB; ++l) ls[l] = a[lane][l] * rd;
            for (int rr = blockIdx.x + G * warp; rr < rest; rr += G * (NT / 32)) {
                double* row = L + (int64_t)(kb + w + rr) * M + kb;
                double acc = lane < w ? row[lane] * rd : 0.0;
#pragma unroll
                for (int l = 0; l < CB; ++l) {
                    if (l < w) {
                        const double xl = __shfl_sync(0xffffffffu, acc, l);
                        if (lane > l) acc = fma(-xl, ls[l], acc);
                    }
                }
                if (lane < w) row[lane] = acc;
            }
            __syncthreads();
        }
        if (!grid_sync(gb, st)) return;
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
                        if ((++it & 1023u) == 0 && globaltimer_ns() - t0 > GP_WAIT_NS) {
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

// float32 inverse by column strips (M <= STRIP_MAX_M). Block column J of W
// depends on no other block column, so after one grid barrier (the diagonal
// block inverses D_I) each CTA walks its strips down the rows with no further
// synchronisation:
//   W_IJ = D_I (delta_IJ I - sum_{J <= K < I} L_IK W_KJ).
// The strip's finished blocks stay in shared memory (M x 32 float32), and the
// K sum streams L in chunks of SKC columns whose global loads are issued one
// chunk ahead, into registers, while the current chunk is multiplied.
constexpr int SKC = 128;
constexpr int STRIP_MAX_M = 1024;
constexpr int SPF = IB * SKC / NT;  // chunk elements per thread

size_t strip_smem_bytes(int M) {
    return sizeof(float) * ((size_t)M * IB + (size_t)IB * (SKC + 1) + 2 * IB * (IB + 1));
}

__global__ void __launch_bounds__(NT) trinv_strip_kernel(const double* __restrict__ L,
                                                         double* __restrict__ W, int M,
                                                         float* __restrict__ Dinv, GpStatus* st,
                                                         GridBar* gb) {
    extern __shared__ __align__(16) float smem_f[];
    float* sS = smem_f;                               // [M][IB]   the strip
    float (*sL)[SKC + 1] = (float (*)[SKC + 1])(sS + (size_t)M * IB);
    float (*sa)[IB + 1] = (float (*)[IB + 1])(&sL[IB][0]);
    float (*sb)[IB + 1] = sa + IB;
    const int tid = threadIdx.x;
    const int nb = (M + IB - 1) / IB;
    // ---- 0: D_I = L_II^{-1}
    for (int I = blockIdx.x; I < nb; I += gridDim.x) {
        const int r0 = I * IB, wI = min(IB, M - r0);
        float v[IB * IB / NT];
#pragma unroll
        for (int q = 0; q < IB * IB / NT; ++q) {
            const int e = tid + q * NT, i = e / IB, j = e % IB;
            v[q] = (i < wI && j <= i) ? (float)L[(int64_t)(r0 + i) * M + r0 + j] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < IB * IB / NT; ++q) {
            const int e = tid + q * NT;
            sa[e / IB][e % IB] = v[q];
            sb[e / IB][e % IB] = 0.0f;
        }
        __syncthreads();
        if (tid < wI) {
            const int j = tid;
            sb[j][j] = 1.0f / sa[j][j];
            for (int i = j + 1; i < wI; ++i) {
                float s = 0.0f;
                for (int k = j; k < i; ++k) s = fmaf(sa[i][k], sb[k][j], s);
                sb[i][j] = -s / sa[i][i];
            }
        }
        __syncthreads();
        for (int e = tid; e < IB * IB; e += NT) Dinv[(int64_t)I * IB * IB + e] = sb[e / IB][e % IB];
        __syncthreads();
    }
    if (!grid_sync(gb, st)) return;
    // ---- 1: strips
    const int ty = tid >> 3, tx = (tid & 7) * 4;
    for (int J = blockIdx.x; J < nb; J += gridDim.x) {
        const int c0 = J * IB, wJ = min(IB, M - c0);
        for (int e = tid; e < c0 * IB; e += NT) {  // rows above the strip's diagonal block
            const int i = e / IB, j = e % IB;
            if (j < wJ) W[(int64_t)i * M + c0 + j] = 0.0;
        }
        // chunk prefetch: (pI, pkc) is the next chunk to be consumed
        int pI = J + 1, pkc = c0;
        float pf[SPF];
        auto load_chunk = [&](int I, int kc) {
            const int r0 = I * IB, wI = min(IB, M - r0);
#pragma unroll
            for (int q = 0; q < SPF; ++q) {
                const int e = tid + q * NT, i = e / SKC, l = e % SKC;
                pf[q] = (i < wI && kc + l < r0) ? (float)L[(int64_t)(r0 + i) * M + kc + l] : 0.0f;
            }
        };
        if (pI < nb) load_chunk(pI, pkc);
        for (int I = J; I < nb; ++I) {
            const int r0 = I * IB, wI = min(IB, M - r0);
            float acc[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = (I == J && ty == tx + c) ? 1.0f : 0.0f;
            for (int kc = c0; kc < r0; kc += SKC) {
                __syncthreads();
#pragma unroll
                for (int q = 0; q < SPF; ++q) {
                    const int e = tid + q * NT;
                    sL[e / SKC][e % SKC] = pf[q];
                }
                __syncthreads();
                if (pkc + SKC < pI * IB) {
                    pkc += SKC;
                } else {
                    ++pI;
                    pkc = c0;
                }
                if (pI < nb) load_chunk(pI, pkc);
                const int kn = min(SKC, r0 - kc);
                const float* srow = sS + (size_t)kc * IB + tx;
                for (int l = 0; l < kn; ++l) {
                    const float av = sL[ty][l];
                    const float4 w4 = *reinterpret_cast<const float4*>(srow + (size_t)l * IB);
                    acc[0] = fmaf(-av, w4.x, acc[0]);
                    acc[1] = fmaf(-av, w4.y, acc[1]);
                    acc[2] = fmaf(-av, w4.z, acc[2]);
                    acc[3] = fmaf(-av, w4.w, acc[3]);
                }
            }
            float dv[IB * IB / NT];
#pragma unroll
            for (int q = 0; q < IB * IB / NT; ++q) dv[q] = Dinv[(int64_t)I * IB * IB + tid + q * NT];
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 4; ++c) sb[ty][tx + c] = acc[c];
#pragma unroll
            for (int q = 0; q < IB * IB / NT; ++q) {
                const int e = tid + q * NT;
                sa[e / IB][e % IB] = dv[q];
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float o = 0.0f;
                for (int l = 0; l <= ty; ++l) o = fmaf(sa[ty][l], sb[l][tx + c], o);
                const bool ok = ty < wI && tx + c < wJ;
                if (r0 + ty < M) sS[(size_t)(r0 + ty) * IB + tx + c] = ok ? o : 0.0f;
                if (ok) W[(int64_t)(r0 + ty) * M + c0 + tx + c] = (double)o;
            }
        }
        __syncthreads();
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
    const size_t inv = el * ((size_t)M * M + nb * IB * IB);
    const size_t chol = sizeof(double) * (size_t)M;  // 1 / L_jj
    return CHOL_RSD_OFFSET + (inv > chol ? inv : chol);
}

// CTAs for the Cholesky of an M x M matrix: about two trailing-update tiles
// per CTA in the first step (one CTA when there is none), at most one per SM,
// so that small problems -- e.g. the many problems of a batch running side by
// side -- do not claim the whole GPU.
int chol_grid(int M, int dev) {
    if (M <= CB) return 1;
    const int T = (M - CB + UT - 1) / UT;
    const int want = (T * (T + 1) / 2 + 1) / 2;
    const int g = coop_grid((const void*)chol_coop_kernel, dev);
    return want < 2 ? 2 : (want > g ? g : want);
}

cudaError_t launch_cholesky(double* L, int M, GpStatus* st, void* work, cudaStream_t stream) {
    int dev = 0;
    cudaGetDevice(&dev);
    CholWork* cw = (CholWork*)work;
    cudaMemsetAsync(cw, 0, CHOL_RSD_OFFSET, stream);
    dim3 grid((unsigned)chol_grid(M, dev)), block(NT);
    void* args[] = {&L, &M, &st, &cw};
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
    if (fp32 && M <= STRIP_MAX_M) {
        float* D = (float*)base;
        const void* k = (const void*)trinv_strip_kernel;
        const size_t smem = strip_smem_bytes(M);
        gp_allow_max_smem((const void*)k);
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        dim3 grid((unsigned)((int)nb < sms ? (int)nb : sms)), block(NT);  // one CTA per strip
        void* args[] = {(void*)&L, &W, &M, &D, &st, &gb};
        return cudaLaunchCooperativeKernel(k, grid, block, args, smem, stream);
    }
    if (fp32) {
        float* R = (float*)base;
        float* D = R + (size_t)M * M;
        const void* k = (const void*)trinv_coop_kernel<float>;
        dim3 grid((unsigned)coop_grid(k, dev)), block(NT);
        void* args[] = {(void*)&L, &W, &M, &R, &D, &st, &gb};
        return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
    }
    double* R = (double*)base;
    double* D = R + (size_t)M * M;
    const void* k = (const void*)trinv_coop_kernel<double>;
    dim3 grid((unsigned)coop_grid(k, dev)), block(NT);
    void* args[] = {(void*)&L, &W, &M, &R, &D, &st, &gb};
    return cudaLaunchCooperativeKernel(k, grid, block, args, 0, stream);
}
