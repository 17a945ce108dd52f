// gp_syrk_tc2.cu -- fused Phi generation + tensor-core Gram on CTA pairs
// (tcgen05 cta_group::2, 256 x 256 tile pairs).
//
// Computes G = Phi^T Phi (the product of Lambda-bar in Sec. 2.2; Phi of
// Eq. 19) with the arithmetic of gp_syrk_tc.cu; b = Phi^T y of these fits is
// formed by the exponent pass (launch_colexp) from the same Phi values, which
// keeps the producers within their 96 registers (accumulating b here made
// them spill and cost 4 % of the kernel's time). Per
// GP_PAIR_BLOCK-row block each column is scaled by 2^(6 - E_m) (|w| < 64) and split
// into the integer s1 = rint(w) and the fp16 remainder lo; s1 s1' is summed
// exactly in float32 TMEM, s1 lo' + lo s1' + lo lo' beside it; each block's
// sums are rescaled by exact powers of two and folded into the split's
// float-pair partial tile by an exact two-sum. The generated Phi values and
// their slices are bit-identical to the one-CTA kernel's.
//
// What differs is the shape of the work, chosen for the shared-memory
// bandwidth that bounds the one-CTA kernel (generation reads table windows
// and writes operand tiles through the same shared memory the MMAs read):
//   * A cluster of two CTAs owns one 256 x 256 tile pair (I2, J2) of G and one
//     row split. CTA r generates Phi columns 256 I2 + 128 r .. + 127 (its half
//     of A) and 256 J2 + 128 r .. + 127 (its half of B) into its shared
//     memory; the leader (r = 0) issues M = 256, N = 256 MMAs over the pair,
//     and each CTA's TMEM receives its 128 rows of the 256 x 256 block. Per
//     generated value the pair does twice the MMA work of a 128 x 128 tile,
//     and each B half is read from shared memory once for both SMs.
//   * A producer thread generates 8 data rows x 4 consecutive columns per
//     stage: the product of the upper dimensions' table rows (Eq. 19) is
//     formed once and reused for the 4 columns whenever they share those
//     digits, so a value costs one table-row read and one multiply. The 4
//     columns are visited in an order rotated by the thread's position so
//     that the 8 threads of a quarter-warp store into 8 different 16-byte
//     rows of a core matrix (no bank conflicts).
//   * TMEM holds acc1 (256 columns) and acc2 (256 columns): there is no room
//     for a float32 sum of blocks, so every block is folded into the split's
//     float64 partial tile as soon as it is done. In four rounds of 16
//     columns a producer warp reads its 32 rows of acc1 and acc2, rescales
//     the block sums (factors the loader warp prepared per block), turns them
//     into float64 exactly by integer bit manipulation (GB300's float64 pipe
//     is slow), stages the 4 KB in the operand slot of the block's last stage
//     (its MMAs are done) and hands it to the bulk-copy engine: a store for
//     the split's first block, an atomic float64 add (cp.reduce.async.bulk)
//     after that. The next block's MMAs wait only for the TMEM reads, not for
//     L2. Each drain first waits for the warp's previous bulk operations to
//     complete, so every element's additions happen in block order and the
//     result is bit-reproducible. The partial tile's layout
//     (gp_pair_tile_offset) makes each warp's round one contiguous 4 KB.
//
// Roles (576 threads per CTA, one CTA per SM):
//   warps 0-15  producers: generation (warps 0-7 the A half, 8-15 the B
//               half; a diagonal pair's B half is its A half) and the
//               per-block drain of TMEM;
//   warp 16     TMEM allocation (both CTAs); in the leader, one lane issues
//               the pair's MMAs and commits them to both CTAs' barriers;
//   warp 17     bulk (TMA) copies of this CTA's table windows, and each
//               block's rescaling factors for the drains.
// Handshakes across the pair: one lane of each producer warp of both CTAs
// arrives on the leader's `full` and `drained` barriers (the peer through its
// shared::cluster address, release at cluster scope) once the warp is done;
// the leader's commits arrive on `empty` and `accf` in both CTAs. Arriving
// per warp instead of per thread matters: a remote arrival crosses the SM
// pair, and 512 of them per stage cost more than the stage's MMAs. Every
// wait is bounded (GP_ETIMEOUT).
#include "gp_syrk_tc.cuh"

#include <algorithm>
#include <mutex>
#include <map>

namespace {

using namespace gpsyrk;

constexpr int TM = 128;                   // rows of a CTA's operand halves
constexpr int TP = 2 * TM;                // pair tile: MMA M = N = 256
constexpr int CW = SYRKTC_BK;             // 32 rows per table chunk
constexpr int H = 2;                      // table chunks per pipeline stage
constexpr int KS = CW * H;                // 64 rows per stage
constexpr int TILE = TM * KS * 2;         // bytes of one 16-bit operand tile
constexpr int SBYTES = 4 * TILE;          // A s1, A lo, B s1, B lo
constexpr uint32_t SBO = (KS / 8) * 128;  // 8-row core-matrix groups
constexpr int BLOCK = GP_PAIR_BLOCK / KS;  // stages per exact GP_PAIR_BLOCK-row block
constexpr int STAGES = 3;                 // deepest operand pipeline
constexpr int WRMAX = 8;                  // deepest window ring
constexpr int NPROD = 512;                // 16 producer warps
constexpr int NPW = NPROD / 32;
constexpr int MMA_WARP = NPW;
constexpr int NTHREADS = NPROD + 64;
constexpr int CPT = TP / 4;               // drained columns per thread
constexpr uint32_t TMEM_COLS = 512;       // acc1 | acc2
constexpr unsigned FULLMASK = 0xffffffffu;

struct Smem2 {
    uint8_t* stage;       // nst x SBYTES (1024-aligned)
    float* win;           // nwr x H x (2 maxrows + 1) x WS
    int* egI;             // TM: global exponents of this CTA's A-half columns
    int* egJ;             // TP: global exponents of the pair's B columns
    unsigned short* crI;  // TM x p: window row of (column, dimension), A half
    unsigned short* crJ;  // TM x p: B half
    int* rng;             // copy ranges (table row, rows, window row)
    float* msc;           // 2 x (TP + TM): per block (double-buffered by parity), the
                          // B columns' and A-half rows' scales 2^(E_blk - E_glob), from the loader
    uint64_t* full;       // STAGES: leader's, one arrival per producer warp of both CTAs
    uint64_t* empty;      // STAGES: one commit (multicast) per phase
    uint64_t* tfull;      // WRMAX: window landed
    uint64_t* wempty;     // WRMAX: every producer warp has read the window
    uint64_t* accf;       // the block's MMAs are done (multicast commit)
    uint64_t* drained;    // leader's: every producer warp of both CTAs has read the block's TMEM
    uint64_t* staged;     // every producer warp of this CTA has finished its drain's staging reads
    uint32_t* tmem_base;
};

__host__ __device__ inline size_t smem_tc2_layout(int maxrows, int p, int nst, int nwr, char* base, Smem2* L) {
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = (off + align - 1) / align * align;
        size_t o = off;
        off += bytes;
        return o;
    };
    size_t oS = take((size_t)nst * SBYTES, 1024);
    size_t oW = take(sizeof(float) * nwr * H * win_floats(maxrows), 16);
    size_t oEI = take(sizeof(int) * TM, 16);
    size_t oEJ = take(sizeof(int) * TP, 16);
    size_t oCI = take(sizeof(unsigned short) * TM * p, 16);
    size_t oCJ = take(sizeof(unsigned short) * TM * p, 16);
    size_t oR = take(sizeof(int) * 3 * max_ranges(p), 16);
    size_t oMS = take(sizeof(float) * 2 * (TP + TM), 16);
    size_t oF = take(sizeof(uint64_t) * STAGES, 8);
    size_t oE = take(sizeof(uint64_t) * STAGES, 8);
    size_t oX = take(sizeof(uint64_t) * WRMAX, 8);
    size_t oY = take(sizeof(uint64_t) * WRMAX, 8);
    size_t oA = take(sizeof(uint64_t), 8);
    size_t oD = take(sizeof(uint64_t), 8);
    size_t oG = take(sizeof(uint64_t), 8);
    size_t oT = take(sizeof(uint32_t), 8);
    if (L) {
        L->stage = (uint8_t*)(base + oS);
        L->win = (float*)(base + oW);
        L->egI = (int*)(base + oEI);
        L->egJ = (int*)(base + oEJ);
        L->crI = (unsigned short*)(base + oCI);
        L->crJ = (unsigned short*)(base + oCJ);
        L->rng = (int*)(base + oR);
        L->msc = (float*)(base + oMS);
        L->full = (uint64_t*)(base + oF);
        L->empty = (uint64_t*)(base + oE);
        L->tfull = (uint64_t*)(base + oX);
        L->wempty = (uint64_t*)(base + oY);
        L->accf = (uint64_t*)(base + oA);
        L->drained = (uint64_t*)(base + oD);
        L->staged = (uint64_t*)(base + oG);
        L->tmem_base = (uint32_t*)(base + oT);
    }
    return off + 1024;  // slack for aligning the dynamic base
}

// 8 consecutive window floats (one table row, the thread's 8 data rows)
__device__ __forceinline__ void ld_row8(const float* p, float v[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void mul_row8(const float* p, float v[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] *= a.x; v[1] *= a.y; v[2] *= a.z; v[3] *= a.w;
    v[4] *= b.x; v[5] *= b.y; v[6] *= b.z; v[7] *= b.w;
}

// P = p (1..4): offsets in registers, products unrolled.
template <int P>
__global__ void __launch_bounds__(NTHREADS, 1)
    syrk_tc2_kernel(GpShape s, const float* __restrict__ tabc, const signed char* __restrict__ ebx,
                    const int* __restrict__ colexp, SyrkSplit sp, int T, int maxrows, int nst, int nwr,
                    double* __restrict__ Gpart, GpStatus* st) {
    extern __shared__ __align__(1024) char smem_raw[];
    __shared__ TileWindow wI, wJ;
    __shared__ int s_nrng;
    char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    Smem2 sm;
    smem_tc2_layout(maxrows, P, nst, nwr, base, &sm);
    const uint32_t rank = cluster_ctarank();

    // work item of the pair -> (pair class, pair, split), as in the one-CTA
    // kernel on tiles of 256 columns: class 0 the diagonal pairs, 1 the pairs
    // (I2, 0), 2 the rest; the pair index runs fastest within a class
    int I2, J2, split, cls;
    {
        int item = (int)(blockIdx.x >> 1);
        const int n0 = T, n1 = T - 1, n2 = (T - 1) * (T - 2) / 2;
        if (item < n0 * sp.n[0]) {
            cls = 0;
            I2 = J2 = item % n0;
            split = item / n0;
        } else if ((item -= n0 * sp.n[0]) < n1 * sp.n[1]) {
            cls = 1;
            I2 = item % n1 + 1;
            J2 = 0;
            split = item / n1;
        } else {
            item -= n1 * sp.n[1];
            cls = 2;
            int a, b;
            tri_pair(item % n2, &a, &b);
            I2 = a + 2;
            J2 = b + 1;
            split = item / n2;
        }
    }
    const int npairs = T * (T + 1) / 2;
    const int q = I2 * (I2 + 1) / 2 + J2;
    const bool diag = (I2 == J2);
    const int I = 2 * I2 + (int)rank, J = 2 * J2 + (int)rank;  // this CTA's 128-column tiles
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    const int64_t rows_c = cls == 0 ? sp.rows[0] : (cls == 1 ? sp.rows[1] : sp.rows[2]);
    const int64_t r0 = (int64_t)split * rows_c;
    int64_t r1 = r0 + rows_c;
    if (r1 > s.Npad) r1 = s.Npad;
    const int nchunks = r0 < r1 ? (int)((r1 - r0) / KS) : 0;  // splits are whole blocks
    const int nblocks = (nchunks + BLOCK - 1) / BLOCK;
    const int64_t RC = (int64_t)(s.p * s.n + 1) * WS;  // floats per table chunk
    const int wsz1 = win_floats(maxrows);
    const int wsz = H * wsz1;

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
            mbar_init(&sm.full[i], 2 * NPW);
            mbar_init(&sm.empty[i], 1);
        }
        for (int i = 0; i < WRMAX; ++i) {
            mbar_init(&sm.tfull[i], 1);
            mbar_init(&sm.wempty[i], NPW);
        }
        mbar_init(sm.accf, 1);
        mbar_init(sm.drained, 2 * NPW);
        mbar_init(sm.staged, NPW);
        mbar_fence_init();
    }
    if (warp == MMA_WARP) tmem_alloc_pair(sm.tmem_base, TMEM_COLS);
    __syncthreads();
    for (int e = tid; e < TM * P; e += NTHREADS) {
        const int c = e / P, j = e % P;
        const int mi = I * TM + c, mj = J * TM + c;
        sm.crI[e] = (unsigned short)(mi < s.M ? window_row(s, wI, j, mi) : 0xFFFF);
        sm.crJ[e] = (unsigned short)(mj < s.M ? window_row(s, wJ, j, mj) : 0xFFFF);
    }
    for (int c = tid; c < TM; c += NTHREADS) sm.egI[c] = colexp[I * TM + c];
    for (int c = tid; c < TP; c += NTHREADS) sm.egJ[c] = colexp[J2 * TP + c];
    // both CTAs' barriers are initialised and the pair's TMEM is allocated
    // before either CTA arrives on the other's barriers
    tc_fence_before();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_base;
    const int nrowsI = wI.nrows;
    const int nwin = (diag ? nrowsI : nrowsI + wJ.nrows) + 1;

    if (warp < NPW) {
        // ------------------------------------------------------------ producers
        const int tsel = warp >> 3;              // 0: A half (tile I), 1: B half (tile J)
        const int wl = warp & 7;
        const int g8 = (wl >> 2) * 4 + (lane >> 3);  // 8-row group of the stage (0..7)
        const int hh = g8 >> 2, gg = g8 & 3;         // its table chunk, 8-row group in the chunk
        const int kq = (wl & 3) * 8 + (lane & 7);    // column quad of the tile (0..31)
        const int rot = (lane & 7) >> 1;
        const bool gen = !(diag && tsel == 1);
        const unsigned short* cr = tsel ? sm.crJ : sm.crI;
        // the tile column visited at step k (the rotation keeps a quarter-warp's
        // stores on 8 different core-matrix rows)
        auto colk = [&](int k) { return 4 * kq + ((k + rot) & 3); };
        // window offsets (floats) of the 4 columns, two 16-bit offsets a
        // register (0xFFFF: a padding column, Phi = 0); offsets stay below
        // (2 maxrows + 1) WS < 65535
        constexpr int PW = (P + 1) / 2;
        uint32_t wpk[4][PW];
        bool shared = true;  // the 4 columns share the upper dimensions' rows (and none is padding)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int j = 0; j < PW; ++j) wpk[k][j] = 0u;
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const unsigned short v = cr[colk(k) * P + j];
                const uint32_t o = v == 0xFFFF ? 0xFFFFu : (uint32_t)v * WS;
                wpk[k][j >> 1] |= o << (16 * (j & 1));
                if (o == 0xFFFFu) shared = false;
            }
        }
#pragma unroll
        for (int k = 1; k < 4; ++k)
#pragma unroll
            for (int j = 0; j + 1 < P; ++j)
                if (((wpk[k][j >> 1] >> (16 * (j & 1))) & 0xFFFFu) != ((wpk[0][j >> 1] >> (16 * (j & 1))) & 0xFFFFu))
                    shared = false;
        auto woff = [&](int k, int j) -> int { return (int)((wpk[k][j >> 1] >> (16 * (j & 1))) & 0xFFFFu); };
        // 32-bit shared-space addresses: the stage's operand tiles and the
        // window slot move per stage, the thread's offsets inside them do not
        const uint32_t stage_s = smem_u32(sm.stage) + (uint32_t)(tsel * 2 * TILE);
        const uint32_t win_s = smem_u32(sm.win) + 4u * (uint32_t)(hh * wsz1 + 8 * gg);
        uint32_t so[4];  // the columns' core-matrix rows in an operand tile (K group g8)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            so[k] = (uint32_t)(colk(k) >> 3) * SBO + (uint32_t)g8 * LBO + (uint32_t)(colk(k) & 7) * 16;
        const int twin = (tsel == 1 && !diag) ? nrowsI * WS : 0;  // this tile's window in the chunk window
        const int mtile = (tsel ? J : I) * TM;
        // drain: TMEM lanes 32 quarter .. (A-half rows), columns CPT cgrp ..
        const int quarter = warp & 3, cgrp = warp >> 2;
        const int drow = quarter * 32 + lane;
        // this warp's rounds of the split's partial tile: round r (16 columns
        // x 32 rows, 512 float64) at gtile + r * 2048 (gp_pair_tile_offset)
        double* gtile = Gpart + ((int64_t)split * npairs + q) * (TP * TP) +
                        (int64_t)gp_pair_tile_offset((int)rank * TM + quarter * 32, cgrp * CPT);
        const uint32_t lrow = ((uint32_t)(quarter * 32) << 16) + cgrp * CPT;
        const uint32_t full_l0 = mapa_shared(sm.full, 0);
        const uint32_t drained_l0 = mapa_shared(sm.drained, 0);
        bool fresh = true;  // the partial tile holds no block yet
        bool ok = true;
        auto arrive_leader = [&](uint64_t* local, uint32_t leader_addr) {
            if (rank == 0)
                mbar_arrive(local);
            else
                mbar_arrive_remote(leader_addr);
        };
        // float -> float64 bit pattern by integer operations: exact for normal
        // floats; zero and subnormals become +-2^-127-ish values, below any
        // block sum's rounding (the block sums are of order one or larger in
        // these units, and a column whose scale would underflow is flushed to
        // zero by pow2_down before this)
        auto f64bits = [](float g) -> uint2 {
            const uint32_t b = __float_as_uint(g);
            const uint32_t hi = (b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + 0x38000000u);
            return make_uint2(b << 29, hi);  // (low word, high word)
        };
        auto drain = [&](int d) -> bool {
            if (!__all_sync(FULLMASK, mbar_wait(sm.accf, d & 1))) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 14);
                return false;
            }
            tc_fence_after();
            // the previous block's bulk operations of this warp are complete:
            // its additions precede this block's
            if (lane == 0) bulk_wait_all();
            __syncwarp();
            // scales back to the global column scaling (the loader formed them
            // for this block and published them with the block's first window)
            const float* ms = sm.msc + (d & 1) * (TP + TM);
            const float mrow = ms[TP + drow];
            const float* mcp = ms + cgrp * CPT;
            // staging: the operand slot of the block's last stage, whose MMAs
            // are done and which the producers fill again only after this drain
            const int clast = min((d + 1) * BLOCK, nchunks) - 1;
            const uint32_t stg_s = smem_u32(sm.stage) + (uint32_t)((clast % nst) * SBYTES) + (uint32_t)warp * 4096u;
#pragma unroll
            for (int rnd = 0; rnd < CPT / 16; ++rnd) {
                uint32_t a1[16], a2[16];
                tmem_ld16_nowait(tmem + lrow + rnd * 16, a1);
                tmem_ld16_nowait(tmem + lrow + TP + rnd * 16, a2);
                tmem_wait_ld();
                if (rnd == CPT / 16 - 1) {
                    // every TMEM read of this warp is done: the next block's MMAs may begin
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) arrive_leader(sm.drained, drained_l0);
                }
                uint2 w[16];
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const float2 mc = *reinterpret_cast<const float2*>(mcp + rnd * 16 + i);
                    w[i] = f64bits((__uint_as_float(a1[i]) + __uint_as_float(a2[i])) * (mrow * mc.x));
                    w[i + 1] = f64bits((__uint_as_float(a1[i + 1]) + __uint_as_float(a2[i + 1])) * (mrow * mc.y));
                }
                if (rnd > 0) {
                    // the previous round has left the staging (its read overlapped
                    // this round's TMEM read and conversion)
                    if (lane == 0) bulk_wait_read<0>();
                    __syncwarp();
                }
#pragma unroll
                for (int qq = 0; qq < 8; ++qq)
                    sts128(stg_s + (uint32_t)((qq * 32 + lane) * 16), w[2 * qq].x, w[2 * qq].y, w[2 * qq + 1].x,
                           w[2 * qq + 1].y);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    const void* src = __cvta_shared_to_generic(stg_s);
                    if (fresh)
                        bulk_s2g(gtile + rnd * 2048, src, 4096);
                    else
                        bulk_add_f64_s2g(gtile + rnd * 2048, src, 4096);
                    bulk_commit();
                }
            }
            fresh = false;
            // the staging slot is written again by the next stages -- of any
            // producer warp, whose tiles span the slot: wait until every warp's
            // staging has been read
            if (lane == 0) {
                bulk_wait_read<0>();
                mbar_arrive(sm.staged);
            }
            if (!__all_sync(FULLMASK, mbar_wait(sm.staged, d & 1))) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 17);
                return false;
            }
            return true;
        };

        const int blk0 = (int)(r0 / GP_PAIR_BLOCK);
        // per-column block exponents, loaded one block ahead
        int e[4] = {0, 0, 0, 0};
        if (nblocks > 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] = ebx[(int64_t)blk0 * s.Mpad + mtile + colk(k)];
        }
        float sc[4] = {0.f, 0.f, 0.f, 0.f};
        int next_drain = 0;
        int stg = 0, sph = 0, wsl = 0, wph = 0;
        for (int c = 0; c < nchunks && ok; ++c) {
            bool w = c < nst || mbar_wait(&sm.empty[stg], sph ^ 1);
            w = w && mbar_wait(&sm.tfull[wsl], wph);
            if (!__all_sync(FULLMASK, w)) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 11);
                ok = false;
                break;
            }
            if (c % BLOCK == 0) {
                // a new block: quantisation scales 2^(6 - E_blk)
#pragma unroll
                for (int k = 0; k < 4; ++k) sc[k] = pow2i(6 - e[k]);
                const int nb = c / BLOCK + 1;
                if (nb < nblocks) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) e[k] = ebx[(int64_t)(blk0 + nb) * s.Mpad + mtile + colk(k)];
                }
            }
            if (gen) {
                const uint32_t sb = stage_s + (uint32_t)(stg * SBYTES);
                const uint32_t wb = win_s + 4u * (uint32_t)(wsl * wsz);
                const uint32_t wt = wb + 4u * (uint32_t)twin;
                if (P >= 2 && shared) {
                    // the upper dimensions' product once, then one row and one multiply a column
                    float pre[8];
                    lds_row8(wt + 4u * (uint32_t)woff(0, 0), pre);
#pragma unroll
                    for (int j = 1; j + 1 < P; ++j) {
                        float r[8];
                        lds_row8(wt + 4u * (uint32_t)woff(0, j), r);
#pragma unroll
                        for (int i = 0; i < 8; ++i) pre[i] *= r[i];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float v[8];
                        lds_row8(wt + 4u * (uint32_t)woff(k, P - 1), v);
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = pre[i] * v[i];
                        uint32_t h[4], l[4];
                        split8(v, sc[k], h, l);
                        sts128(sb + so[k], h[0], h[1], h[2], h[3]);
                        sts128(sb + TILE + so[k], l[0], l[1], l[2], l[3]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float v[8];
                        if (woff(k, 0) == 0xFFFF) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) v[i] = 0.f;
                        } else {
                            lds_row8(wt + 4u * (uint32_t)woff(k, 0), v);
#pragma unroll
                            for (int j = 1; j < P; ++j) {
                                float r[8];
                                lds_row8(wt + 4u * (uint32_t)woff(k, j), r);
#pragma unroll
                                for (int i = 0; i < 8; ++i) v[i] *= r[i];
                            }
                        }
                        uint32_t h[4], l[4];
                        split8(v, sc[k], h, l);
                        sts128(sb + so[k], h[0], h[1], h[2], h[3]);
                        sts128(sb + TILE + so[k], l[0], l[1], l[2], l[3]);
                    }
                }
            }
            // every lane's operand writes are ordered before the async proxy's
            // reads, then one arrival for the warp (release: it carries the
            // lanes' writes, ordered before it by the warp barrier)
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.wempty[wsl]);  // this warp is done with the window
                arrive_leader(&sm.full[stg], full_l0 + 8u * (uint32_t)stg);
            }
            if (++stg == nst) {
                stg = 0;
                sph ^= 1;
            }
            if (++wsl == nwr) {
                wsl = 0;
                wph ^= 1;
            }
            // drain a finished block once one stage of the next one is queued
            while (next_drain < nblocks && min((next_drain + 1) * BLOCK, nchunks) <= c) {
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
        if (nblocks == 0) {  // a split without rows: its partial tile is zero
            for (int k = lane; k < (CPT / 16) * 512 / 4; k += 32)
                reinterpret_cast<double4*>(gtile)[(k / 128) * 512 + (k % 128)] = make_double4(0.0, 0.0, 0.0, 0.0);
        }
        // every bulk operation of this warp has completed before the CTA ends
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer (leader CTA)
        if (rank == 0 && lane == 0) {
            const uint32_t idesc = idesc_f16_f32(TP, TP);
            // descriptors of stage 0's four tiles; a stage adds SBYTES / 16 and
            // a 16-row K step 2 LBO / 16 to the address field (no carry out of
            // it: shared addresses stay below 256 KB)
            const uint64_t dA1_0 = smem_desc(smem_u32(sm.stage), LBO, SBO);
            const uint64_t dA2_0 = dA1_0 + (uint64_t)(TILE >> 4);
            const uint64_t dB1_0 = diag ? dA1_0 : dA1_0 + (uint64_t)(2 * TILE >> 4);
            const uint64_t dB2_0 = diag ? dA2_0 : dA1_0 + (uint64_t)(3 * TILE >> 4);
            int stg = 0, sph = 0, issued = 0;
            for (int c = 0; c < nchunks; ++c) {
                const int d = c / BLOCK, cb = c % BLOCK;
                // both CTAs have folded block d - 1 out of acc1 and acc2
                if (cb == 0 && d >= 1 && !mbar_wait_cl(sm.drained, (d - 1) & 1)) {
                    gp_set_status(st, GP_ETIMEOUT, 15);
                    break;
                }
                if (!mbar_wait_cl(&sm.full[stg], sph)) {
                    gp_set_status(st, GP_ETIMEOUT, 13);
                    break;
                }
                tc_fence_after();
                const uint32_t acc1 = tmem;
                const uint32_t acc2 = tmem + TP;
                const uint64_t so = (uint64_t)(stg * (SBYTES >> 4));
#pragma unroll
                for (int ks = 0; ks < KS / 16; ++ks) {
                    const uint64_t ko = so + (uint64_t)(ks * (2 * LBO >> 4));
                    const uint32_t acc = (cb > 0 || ks > 0) ? 1u : 0u;
                    mma_f16_pair(acc1, dA1_0 + ko, dB1_0 + ko, idesc, acc);  // s1 s1'  (exact)
                    mma_f16_pair(acc2, dA1_0 + ko, dB2_0 + ko, idesc, acc);  // s1 lo'
                    mma_f16_pair(acc2, dA2_0 + ko, dB1_0 + ko, idesc, 1u);   // lo s1'
                    mma_f16_pair(acc2, dA2_0 + ko, dB2_0 + ko, idesc, 1u);   // lo lo'
                }
                mma_commit_pair(&sm.empty[stg], (uint16_t)3);
                if (cb == BLOCK - 1 || c == nchunks - 1) mma_commit_pair(sm.accf, (uint16_t)3);
                ++issued;
                if (++stg == nst) {
                    stg = 0;
                    sph ^= 1;
                }
            }
            // before leaving, wait (bounded) for the last issued MMAs
            if (issued > 0) {
                const int lc = issued - 1;
                mbar_wait(&sm.empty[lc % nst], (lc / nst) & 1);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ window loader (bulk copies)
        const int nr = s_nrng;
        const uint32_t wbytes = (uint32_t)(H * nwin * WS * 4);
        int rdst = 0, rsrc = 0, rlen = 0;
        for (int k = lane; k < nr; k += 32) {
            rdst = sm.rng[3 * k + 2] * WS;
            rsrc = sm.rng[3 * k] * WS;
            rlen = sm.rng[3 * k + 1] * WS * 4;
        }
        const int blk0 = (int)(r0 / GP_PAIR_BLOCK);
        int c = 0, wsl = 0, wph = 0;
        for (; c < nchunks; ++c) {
            const bool e = c < nwr || mbar_wait(&sm.wempty[wsl], wph ^ 1);
            if (!__all_sync(FULLMASK, e)) {
                if (lane == 0) gp_set_status(st, GP_ETIMEOUT, 16);
                break;
            }
            if (c % BLOCK == 0) {
                // the block's rescaling factors 2^(E_blk - E_glob) for the drains
                // (exact powers of two); the buffer of this parity was last read
                // by the drain of block d - 2, which every producer warp finished
                // before releasing the window slot this copy waited for; the
                // arrival below publishes them with the block's first window
                const int d = c / BLOCK;
                const signed char* eb = ebx + (int64_t)(blk0 + d) * s.Mpad;
                float* ms = sm.msc + (d & 1) * (TP + TM);
                for (int k = lane; k < TP + TM; k += 32)
                    ms[k] = k < TP ? pow2_down((int)eb[J2 * TP + k] - sm.egJ[k])
                                   : pow2_down((int)eb[I * TM + (k - TP)] - sm.egI[k - TP]);
                __syncwarp();
            }
            if (lane == 0) mbar_arrive_expect_tx(&sm.tfull[wsl], wbytes);
            __syncwarp();
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float* src = tabc + ((r0 + (int64_t)c * KS) / CW + h) * RC;
                float* dst = sm.win + wsl * wsz + h * wsz1;
                if (lane < nr) bulk_g2s(dst + rdst, src + rsrc, (uint32_t)rlen, &sm.tfull[wsl]);
            }
            if (++wsl == nwr) {
                wsl = 0;
                wph ^= 1;
            }
        }
        for (int k = c - nwr; k < c; ++k)
            if (k >= 0) mbar_wait(&sm.tfull[k % nwr], (k / nwr) & 1);
        __syncwarp();
    }
    // the peer may still arrive on the leader's barriers, and the leader's MMAs
    // read both CTAs' shared memory, until both reach this point
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, TMEM_COLS);
    }
}

// Pipeline depth: the deepest (<= STAGES operand stages, then <= WRMAX window
// slots, at least two of each) whose dynamic shared memory fits one CTA next
// to the kernel's static shared memory. Returns the operand stages (0: none fits).
int syrk_tc2_stages(const GpShape& s, int maxrows, int* nwr, size_t* smem) {
    constexpr size_t kDynamicBudget = (227 - 2) * 1024;
    for (int nst = STAGES; nst >= 2; --nst)
        for (int w = WRMAX; w >= 2; --w) {
            *smem = smem_tc2_layout(maxrows, s.p, nst, w, nullptr, nullptr);
            if (*smem <= kDynamicBudget) {
                *nwr = w;
                return nst;
            }
        }
    return 0;
}

template <int P>
cudaError_t go2(const GpShape& s, const float* tabc, const signed char* ebx, const int* colexp, const SyrkSplit& sp,
                int T, int maxrows, int nst, int nwr, size_t smem, double* Gpart, GpStatus* st,
                cudaStream_t stream) {
    const void* kern = (const void*)syrk_tc2_kernel<P>;
    cudaError_t e = gp_allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)T * sp.n[0] + (int64_t)(T - 1) * sp.n[1] + (int64_t)(T - 1) * (T - 2) / 2 * sp.n[2];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * items));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, syrk_tc2_kernel<P>, s, tabc, ebx, colexp, sp, T, maxrows, nst, nwr, Gpart, st);
}

}  // namespace

bool syrktc2_supported(const GpShape& s) {
    if (s.p < 1 || s.p > 4 || s.Mpad % TP != 0 || s.Npad % KS != 0) return false;
    size_t smem = 0;
    int nwr = 0;
    return syrk_tc2_stages(s, gp_max_window_rows(s, TM), &nwr, &smem) > 0;
}

int syrktc2_max_clusters(const GpShape& s, int dev) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;  // (device, p) -> clusters
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({dev, s.p});
        if (it != cache.end()) return it->second;
    }
    const int maxrows = gp_max_window_rows(s, TM);
    size_t smem = 0;
    int nwr = 0;
    int n = 0;
    if (syrk_tc2_stages(s, maxrows, &nwr, &smem) > 0) {
        const void* kern = nullptr;
        switch (s.p) {
            case 1: kern = (const void*)syrk_tc2_kernel<1>; break;
            case 2: kern = (const void*)syrk_tc2_kernel<2>; break;
            case 3: kern = (const void*)syrk_tc2_kernel<3>; break;
            default: kern = (const void*)syrk_tc2_kernel<4>; break;
        }
        if (gp_allow_max_smem(kern) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2);
            cfg.blockDim = dim3(NTHREADS);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
                (void)cudaGetLastError();
                n = 0;
            }
        }
    }
    if (n < 1) {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = std::max(1, sms / 2);
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[{dev, s.p}] = n;
    return n;
}

cudaError_t launch_syrk_tc2(const GpShape& s, const float* tabc, const SyrkSplit& sp, double* Gpart, int* colexp, signed char* ebx,
                            GpStatus* st, cudaStream_t stream) {
    if (!syrktc2_supported(s)) return cudaErrorInvalidValue;
    for (int c = 0; c < 3; ++c)
        if (sp.n[c] < 1 || sp.rows[c] < GP_PAIR_BLOCK || sp.rows[c] % GP_PAIR_BLOCK != 0) return cudaErrorInvalidValue;
    // the exponents of the pair blocks (launch_colexp writes them after the scale blocks')
    const signed char* ebx4 = syrktc_pair_exponents(s, ebx);
    const int maxrows = gp_max_window_rows(s, TM);
    size_t smem = 0;
    int nwr = 0;
    const int nst = syrk_tc2_stages(s, maxrows, &nwr, &smem);
    const int T = s.Mpad / TP;
    switch (s.p) {
        case 1: return go2<1>(s, tabc, ebx4, colexp, sp, T, maxrows, nst, nwr, smem, Gpart, st, stream);
        case 2: return go2<2>(s, tabc, ebx4, colexp, sp, T, maxrows, nst, nwr, smem, Gpart, st, stream);
        case 3: return go2<3>(s, tabc, ebx4, colexp, sp, T, maxrows, nst, nwr, smem, Gpart, st, stream);
        default: return go2<4>(s, tabc, ebx4, colexp, sp, T, maxrows, nst, nwr, smem, Gpart, st, stream);
    }
}
