// gp_common.cuh -- shared definitions of the GB300 decomposed-kernel GP library.
//
// Host/device structures for one problem, the device status word, the
// eigenfunction-table window of a column tile (Sec. 2.3, Eq. 18-19: a
// column of Phi is a product of one table row per input dimension), and
// error-handling helpers. Nothing here launches a kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gpfagp.h"

#define GP_PMAX 32           // largest supported input dimension p

// ---------------------------------------------------------------------------
// Device status word: written by kernels, read back once per call by the host.
// ---------------------------------------------------------------------------
struct GpStatus {
    int32_t code;            // GP_OK or a negative status
    int32_t pad;
    int64_t detail;          // pivot column, timeout site, ...
};

// float64 -> float32, rounded to nearest even, in integer arithmetic: on
// GB300 the conversion instruction runs on the float64 pipe (64 cycles per
// warp instruction per scheduler), integer operations do not. A normal
// result takes the top 23 mantissa bits plus the rounding of the 29 below
// (a carry moves into the exponent, and to infinity at the top); tiny
// results become subnormal or zero, large ones infinity, NaN stays NaN.
__device__ __forceinline__ float gp_d2f_rn(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7FFu, sgn = hi & 0x80000000u;
    if (e - 897u < 254u || e == 0u) {  // float exponent 1 .. 254 before rounding, or zero
        const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29), rem = lo & 0x1FFFFFFFu;
        const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
        return __uint_as_float(e == 0u ? sgn : sgn | ((((e - 896u) << 23) | m) + up));
    }
    if (e == 0x7FFu) return __uint_as_float(sgn | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x00400000u : 0u));
    if (e > 1150u) return __uint_as_float(sgn | 0x7F800000u);
    // |x| < 2^-126: q = round(x 2^149) = round(sig 2^(e - 926)), sig with its hidden bit
    const int sh = 926 - (int)e;
    if (e == 0u || sh > 63) return __uint_as_float(sgn);
    const uint64_t sig = (1ull << 52) | ((uint64_t)(hi & 0xFFFFFu) << 32) | lo;
    uint64_t q = sig >> sh;
    const uint64_t rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    return __uint_as_float(sgn | (uint32_t)q);
}
// float -> float64 without the float64 pipe (exact for normal floats and
// zero; float subnormals, below 1.2e-38, become signed zero)
__device__ __forceinline__ double gp_f2d_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (e == 0xFFu) return (double)f;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}
// x is finite (neither infinite nor NaN), from its exponent bits: the
// float64 comparison would take the float64 pipe
__device__ __forceinline__ bool gp_isfinite_bits(double x) {
    return ((__double2hiint(x) >> 20) & 0x7FF) != 0x7FF;
}

__device__ __forceinline__ void gp_set_status(GpStatus* st, int code, int64_t detail) {
    // first error wins
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// ---------------------------------------------------------------------------
// One problem's shape and SE eigen-parameters (Eq. 14-16), per input
// dimension j (one eps_j and rho_j per dimension: the ARD kernel of Eq. 17;
// all equal for the isotropic kernel of Eq. 13), computed on the host in
// float64 (and rounded to float there for the float32 tables) and passed by
// value to kernels.
// ---------------------------------------------------------------------------
struct GpShape {
    int64_t N;               // data rows (training or test points)
    int64_t Npad;            // rows of the eigenfunction tables (multiple of 128)
    int     p, n;            // input dimensions, eigenfunctions per dimension
    int     M;               // n^p
    int     Mpad;            // M rounded up to the tile size of the kernel in use
    int     stride[GP_PMAX]; // n^(p-1-j): column m has digit (m / stride[j]) % n
    double  ab[GP_PMAX];     // rho_j beta_j   (Hermite argument scale, Eq. 15)
    double  d2[GP_PMAX];     // delta_j^2      (envelope exponent, Eq. 15)
    double  sb[GP_PMAX];     // gamma_1 = sqrt(beta_j)
    float   abf[GP_PMAX], d2f[GP_PMAX], sbf[GP_PMAX];  // the same rounded to float
};

// ---------------------------------------------------------------------------
// Table window of a tile of consecutive columns [m0, m0 + TW).
//
// Each column of Phi multiplies one eigenfunction table row per dimension.
// For dimension j, the digits of consecutive columns are consecutive values
// mod n, so a tile needs count_j <= n rows of dimension j starting at digit
// first_j (mod n). Window row r = base_j + ((digit - first_j) mod n).
// ---------------------------------------------------------------------------
struct TileWindow {
    int nrows;
    int base[GP_PMAX];
    int first[GP_PMAX];
    int count[GP_PMAX];
};

__host__ __device__ inline void tile_window(const GpShape& s, int m0, int TW, TileWindow* w) {
    int m1 = m0 + TW;
    if (m1 > s.M) m1 = s.M;
    int rows = 0;
    for (int j = 0; j < s.p; ++j) {
        int st = s.stride[j];
        int f = (m0 / st) % s.n;
        int cnt = 0;
        if (m1 > m0) {
            long span = (long)((m1 - 1) / st) - (long)(m0 / st) + 1;
            cnt = span < s.n ? (int)span : s.n;
        }
        w->base[j] = rows;
        w->first[j] = f;
        w->count[j] = cnt;
        rows += cnt;
    }
    w->nrows = rows;
}

// window row of dimension j for column m (m inside the tile)
__host__ __device__ inline int window_row(const GpShape& s, const TileWindow& w, int j, int m) {
    int d = (m / s.stride[j]) % s.n;
    int pos = d - w.first[j];
    if (pos < 0) pos += s.n;
    return w.base[j] + pos;
}

// global table row (dimension j, digit) for window row r
__host__ __device__ inline int window_table_row(const GpShape& s, const TileWindow& w, int r) {
    int j = 0;
    while (j + 1 < s.p && r >= w.base[j + 1]) ++j;
    int d = w.first[j] + (r - w.base[j]);
    if (d >= s.n) d -= s.n;
    return j * s.n + d;
}

// lower-triangular tile pair index q -> (I, J), I >= J, q = I(I+1)/2 + J
__host__ __device__ inline void tri_pair(int q, int* I, int* J) {
    // float estimate (double square roots are slow on the device), corrected below
    int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    if (i < 0) i = 0;
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    while (i * (i + 1) / 2 > q) --i;
    *I = i;
    *J = q - i * (i + 1) / 2;
}

// largest window (table rows) over the column tiles of width TW
static inline int gp_max_window_rows(const GpShape& s, int TW) {
    int mx = 1;
    for (int m0 = 0; m0 < s.M; m0 += TW) {
        TileWindow w;
        tile_window(s, m0, TW, &w);
        if (w.nrows > mx) mx = w.nrows;
    }
    return mx;
}

static inline int64_t gp_round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// Host-side helpers implemented in gp_api.cu
// ---------------------------------------------------------------------------
int gp_fill_shape(GpShape* s, int64_t N, int p, int n, double eps, double alpha, int tile);
// the same with eps_j, alpha_j per dimension (p values each)
int gp_fill_shape_ard(GpShape* s, int64_t N, int p, int n, const double* eps, const double* alpha, int tile);

// Let `kern` use as much dynamic shared memory as the device allows next to
// its static shared memory. Always the same value, so it can be set before
// every launch in any order (captured graphs and concurrent launches of the
// same kernel with different sizes see one limit); each launch's own size
// is checked against it at launch.
inline cudaError_t gp_allow_max_smem(const void* kern) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

// gp_prof.cu: kernel launch counter and CUDA-event timing of kernel groups
void gp_note_launches(int n);
void gp_prof_begin(const char* name, cudaStream_t s);
void gp_prof_end(const char* name, cudaStream_t s);
int gp_prof_suspend();
void gp_prof_resume(int state);

// RAII bracket of one kernel group on a stream
struct GpProf {
    const char* name;
    cudaStream_t s;
    GpProf(const char* n, cudaStream_t st) : name(n), s(st) { gp_prof_begin(n, st); }
    ~GpProf() { gp_prof_end(name, s); }
};
