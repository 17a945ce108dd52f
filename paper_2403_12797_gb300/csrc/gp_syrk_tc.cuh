// gp_syrk_tc.cuh -- device helpers shared by the tensor-core Gram kernels
// (gp_syrk_tc.cu: one CTA per 128 x 128 tile pair; gp_syrk_tc2.cu: a CTA pair
// per 256 x 256 tile pair): the table-window copy ranges of a column tile, the
// exact power-of-two scales, and the split of a scaled Phi value into the
// integer slice s1 and the fp16 remainder lo that the exact-block Gram sums.
#pragma once

#include "gp_kernels.cuh"
#include "gp_tc.cuh"

namespace gpsyrk {

constexpr int WS = SYRKTC_WS;  // floats per window row (36: bank-conflict padding)
constexpr uint32_t LBO = 128;  // K-adjacent core matrices of an operand tile

__host__ __device__ inline int max_ranges(int p) { return 4 * p + 1; }
__host__ __device__ inline int win_floats(int maxrows) { return (2 * maxrows + 1) * WS; }

// 2^k for -126 <= k <= 127, exactly
__device__ __forceinline__ float pow2i(int k) { return __int_as_float((127 + k) << 23); }
// 2^k for k <= 0, flushed to 0 below 2^-126 (a block whose column bound is
// that far below the column's global bound adds nothing representable)
__device__ __forceinline__ float pow2_down(int k) { return k < -126 ? 0.f : __int_as_float((127 + k) << 23); }

// Copy ranges of one tile's window (thread 0): dimension j's window rows
// are the digits first .. first+count-1 (mod n), i.e. at most two
// contiguous runs of table rows j*n + digit.
__device__ inline int tile_ranges(const GpShape& s, const TileWindow& w, int dst0, int* rng, int nr) {
    for (int j = 0; j < s.p; ++j) {
        const int cnt = w.count[j];
        if (cnt <= 0) continue;
        const int first = w.first[j];
        const int run = min(cnt, s.n - first);
        rng[3 * nr] = j * s.n + first;
        rng[3 * nr + 1] = run;
        rng[3 * nr + 2] = dst0 + w.base[j];
        ++nr;
        if (cnt > run) {
            rng[3 * nr] = j * s.n;
            rng[3 * nr + 1] = cnt - run;
            rng[3 * nr + 2] = dst0 + w.base[j] + run;
            ++nr;
        }
    }
    return nr;
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
// the magic K = 1.5 * 2^23 + 0x6480 (still in [2^23, 2^24), where floats
// are the integers) rounds w to the nearest integer k (ties to even), and
// the low 16 bits of the sum t are then 0x6480 + k -- the float16 bit
// pattern of 1152 + k (exponent 2^10) -- for |k| <= 128, with no carry out
// of the half word. One byte permute packs two of them and one exact half2
// subtraction of 1152 leaves k. Only the remainder takes a float16
// conversion.
template <uint32_t SBO>
__device__ __forceinline__ void store_slices(uint8_t* s1_tile, uint8_t* lo_tile, int r, int g,
                                             const float v[8], float sc) {
    constexpr float kMagic = 12608640.0f;  // 1.5 * 2^23 + 0x6480
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // v * sc is exact (sc is a power of two), so one rounding each: t rounds
        // v sc + K to an integer, a = rint(v sc), lo = v sc - a exactly
        const float t0 = __fmaf_rn(v[2 * q], sc, kMagic), t1 = __fmaf_rn(v[2 * q + 1], sc, kMagic);
        const float a0 = __fsub_rn(t0, kMagic), a1 = __fsub_rn(t1, kMagic);
        const uint32_t raw = __byte_perm((uint32_t)__float_as_int(t0), (uint32_t)__float_as_int(t1), 0x5410);
        uint32_t k2;
        asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(k2) : "r"(raw), "r"(0x64806480u));  // - (1152, 1152)
        h[q] = k2;
        l[q] = pack_half2(__fmaf_rn(v[2 * q], sc, -a0), __fmaf_rn(v[2 * q + 1], sc, -a1));
    }
    const uint32_t off = (uint32_t)(r >> 3) * SBO + (uint32_t)g * LBO + (uint32_t)(r & 7) * 16;
    *reinterpret_cast<uint4*>(s1_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// 32-bit shared-space accesses (no generic-address arithmetic). Volatile, so
// they keep their order relative to the pipeline's barrier waits.
__device__ __forceinline__ void lds_row8(uint32_t a, float v[8]) {
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(a));
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4+16];"
                 : "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(a));
}
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

// The split of store_slices into registers: s1 (h) and lo (l) of 8 values
// scaled by the power of two sc, two fp16 per word, low element first.
__device__ __forceinline__ void split8(const float v[8], float sc, uint32_t h[4], uint32_t l[4]) {
    constexpr float kMagic = 12608640.0f;  // 1.5 * 2^23 + 0x6480
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float t0 = __fmaf_rn(v[2 * q], sc, kMagic), t1 = __fmaf_rn(v[2 * q + 1], sc, kMagic);
        const float a0 = __fsub_rn(t0, kMagic), a1 = __fsub_rn(t1, kMagic);
        const uint32_t raw = __byte_perm((uint32_t)__float_as_int(t0), (uint32_t)__float_as_int(t1), 0x5410);
        uint32_t k2;
        asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(k2) : "r"(raw), "r"(0x64806480u));  // - (1152, 1152)
        h[q] = k2;
        l[q] = pack_half2(__fmaf_rn(v[2 * q], sc, -a0), __fmaf_rn(v[2 * q + 1], sc, -a1));
    }
}

}  // namespace gpsyrk

