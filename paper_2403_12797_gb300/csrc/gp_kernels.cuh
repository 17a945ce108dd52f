// gp_kernels.cuh -- launchers of the library's CUDA kernels (host side).
#pragma once

#include "gp_common.cuh"

constexpr int SYRKTC_TM = 128;  // tile of the mixed-precision Gram
constexpr int SYRKTC_BK = 32;   // rows per pipeline chunk of it

// ---- eigenfunction tables (gp_tables.cu) ------------------------------------
void launch_eig_tables_f64(const GpShape& s, const double* X, const double* y, double* tab,
                           GpStatus* st, cudaStream_t stream);
void launch_eig_tables_f32(const GpShape& s, const double* X, const double* y, float* tab,
                           GpStatus* st, cudaStream_t stream);

// Rows per block of the mixed-precision Gram's column scales: each block
// scales its columns by their own exact maxima (|w| < 64), and the one-CTA
// kernel's tensor-core integer sums (at most 1024 * 64^2 = 2^22) are exact over
// one block. Row splits are whole blocks.
constexpr int GP_TAB_BLOCK = 1024;
// Rows per exact block of the CTA-pair kernel: four scale blocks under the
// largest of their exponents (4096 * 64^2 = 2^24); its row splits are whole
// pair blocks.
constexpr int GP_PAIR_BLOCK = 4096;
// Chunk-major float32 table of the mixed-precision Gram: chunk q of 32 rows
// holds table row R = j*n + k at tabc[q*RC + R*SYRKTC_WS + i%32] and y in row
// p*n, RC = (p*n + 1) * SYRKTC_WS (row stride 36 floats, 4 of them zero).
constexpr int SYRKTC_WS = 36;
size_t syrktc_table_floats(const GpShape& s);
void launch_eig_tables_chunked(const GpShape& s, const double* X, const double* y, float* tabc, GpStatus* st,
                               cudaStream_t stream);

// ---- float64 Gram (gp_syrk64.cu) ---------------------------------------------
// Tile 64 x 64, lower-triangular tile pairs x N splits.
constexpr int SYRK64_TM = 64;
constexpr int SYRK64_BK = 16;
size_t syrk64_smem_bytes(const GpShape& s);
cudaError_t launch_syrk64(const GpShape& s, const double* tab, const double* ypad, int nsplit,
                          int64_t rows_per_split, double* Gpart, double* bpart, cudaStream_t stream);

// ---- bf16x3 tensor-core Gram (gp_syrk_tc.cu) ---------------------------------
// Row splits of the tensor-core Gram per class of tile pair (I, J): 0 the
// diagonal pairs, 1 the pairs (I, 0), I > 0 (which also form Phi^T y), 2 the
// other off-diagonal pairs. The classes cost different amounts per row (a
// diagonal pair generates one operand tile, the others two), so each gets its
// own split count n[c] and rows per split rows[c] (a multiple of
// GP_TAB_BLOCK). Pair (I, J) of class c has partial tiles for splits
// 0 .. n[c] - 1; smax is the largest n[c].
struct SyrkSplit {
    int n[3];
    int64_t rows[3];
    int smax;
};
__host__ __device__ __forceinline__ int syrk_pair_class(int I, int J) { return I == J ? 0 : (J == 0 ? 1 : 2); }
size_t syrktc_smem_bytes(const GpShape& s);
// bytes of the per-block column exponents the launch needs (ebx argument)
size_t syrktc_ebx_bytes(const GpShape& s);
// Gpart holds column-scaled partial tiles as float pairs hi + lo (units
// 2^(12 - E_m - E_m')) at (split * npairs + pair), with colexp and ebx formed
// before by launch_colexp, bpart the unscaled float64 Phi^T y partials at
// (split * Mpad + m), from the pairs (I, 0).
cudaError_t launch_syrk_tc(const GpShape& s, const float* tabc, const SyrkSplit& sp, float2* Gpart, double* bpart,
                           int* colexp, signed char* ebx, GpStatus* st, cudaStream_t stream);

// One problem of a batched Gram launch: the arguments launch_syrk_tc takes
// (its column exponents already formed by launch_colexp), and the launch's
// first item of this problem (problems in ascending item0).
struct SyrkBatchProb {
    GpShape s;
    const float* tabc;
    const signed char* ebx;
    const int* colexp;
    SyrkSplit sp;
    int T;
    float2* Gpart;
    double* bpart;
    GpStatus* st;
    int64_t item0;
};
constexpr size_t SYRK_BATCH_SHAPE_BYTES = (sizeof(GpShape) + 1023) / 1024 * 1024;
// CTAs (work items) of launch_syrk_tc for this shape and split plan
int64_t syrktc_items(const GpShape& s, const SyrkSplit& sp);
// The Grams of several problems with the same p in one launch: items in
// [probs[k].item0, probs[k].item0 + syrktc_items) are problem k's; maxrows
// bounds every problem's tile window (gp_max_window_rows(s, 128)).
cudaError_t launch_syrk_tc_batch(const SyrkBatchProb* probs, int nprob, int64_t items, int p, int maxrows,
                                 cudaStream_t stream);
// ebx (syrktc_ebx_bytes): ebx[b * Mpad + m] = E_m of GP_TAB_BLOCK-row block b
// (the exact maximum of |Phi[:, m]| over the block's rows is below 2^E_m),
// then the largest E_m of each GP_PAIR_BLOCK-row block at
// syrktc_pair_exponents(s, ebx), then the pass's scratch; colexp[m] = the
// largest E_m over all blocks. With bblk (colexp_b_floats(s) floats of
// scratch) and b (M float64) it also forms b = Phi^T y from the same Phi
// values: float32 partials per block and row range, summed in float64 in a
// fixed order (bit-reproducible).
void launch_colexp(const GpShape& s, const float* tabc, int* colexp, signed char* ebx, cudaStream_t stream,
                   float* bblk = nullptr, double* b = nullptr);
size_t colexp_b_floats(const GpShape& s);
const signed char* syrktc_pair_exponents(const GpShape& s, const signed char* ebx);

// ---- split-N reduction and assembly (gp_assemble.cu) --------------------------
// A = sum_s Gpart[s] + diag(d) (M x M, full symmetric, row-major, lda = M);
// b = sum_s bpart[s]. d may be NULL (plain Gram).
void launch_assemble_f64(const double* Gpart, const double* bpart, int nsplit, int tile, int Mpad,
                         int M, const double* d, double* A, double* b, cudaStream_t stream);
// Optional extras of the fit's assembly: the noise diagonal d_m computed in
// the kernel (from loglam and sigma2, stored to dout and added to A's
// diagonal; d is then ignored), and a copy of A's lower triangle written to L.
struct AssembleExtra {
    const GpShape* shape;
    const double* loglam;
    double sigma2;
    double* dout;
    double* L;
};
// ---- the tensor-core Gram on CTA pairs (gp_syrk_tc2.cu) --------------------------
// 256 x 256 tile pairs, one cluster of two CTAs each (tcgen05 cta_group::2); the
// same arithmetic as launch_syrk_tc with tiles of 256: s.Mpad a multiple of
// 256, SyrkSplit classes over the 256-column tiles, Gpart (split * npairs +
// pair) x 256 x 256 float64 partials. It forms G only: b = Phi^T y of its
// fits comes from launch_colexp. For p <= 4 when the pipeline fits shared
// memory (syrktc2_supported).
bool syrktc2_supported(const GpShape& s);
// Partial tiles of the CTA-pair kernel: float64, one 256 x 256 tile per (split,
// pair) at (split * npairs + pair) * 65536, element (R, C) of the tile (R the
// A index, C the B index) at the offset below -- the order in which each warp
// of the kernel drains TMEM (CTA rank, column group, round of 16 columns, lane
// quarter; inside a round, column pairs, lane, column), so that one warp's
// round (32 rows x 16 columns) is 4 KB contiguous and is staged in shared
// memory without bank conflicts.
__host__ __device__ __forceinline__ int gp_pair_tile_offset(int R, int C) {
    const int rank = R >> 7, quarter = (R >> 5) & 3, lane = R & 31;
    const int cgrp = C >> 6, rnd = (C >> 4) & 3, cc = C & 15;
    return ((((rank * 4 + cgrp) * 4 + rnd) * 4 + quarter) << 9) + (((cc >> 1) * 32 + lane) << 1) + (cc & 1);
}
// clusters of the kernel that are resident at once on device dev
int syrktc2_max_clusters(const GpShape& s, int dev);
cudaError_t launch_syrk_tc2(const GpShape& s, const float* tabc, const SyrkSplit& sp, double* Gpart, int* colexp,
                            signed char* ebx, GpStatus* st, cudaStream_t stream);

// float-pair partials of the tensor-core Gram (tile x tile partial tiles, tile
// 128 or 256): A[m][m'] = split sum * 2^(E_m + E_m' - 12) (+ d)
void launch_assemble_scaled(const float2* Gpart, const double* bpart, const int* colexp, const SyrkSplit& sp,
                            int tile, int Mpad, int M, const double* d, double* A, double* b,
                            cudaStream_t stream, const AssembleExtra* ex = nullptr);
// the same from the CTA-pair kernel's float64 partial tiles (gp_pair_tile_offset); bpart NULL:
// b is left alone (the CTA-pair path forms it in launch_colexp)
void launch_assemble_pair(const double* Gpart, const double* bpart, const int* colexp, const SyrkSplit& sp,
                          int Mpad, int M, const double* d, double* A, double* b, cudaStream_t stream,
                          const AssembleExtra* ex = nullptr);
// d_m = sigma2 * exp(-sum_j loglam[m_j]) clamped at 1e200 (Eq. 16, 20)
void launch_noise_diag(const GpShape& s, const double* loglam, double sigma2, double* d,
                       cudaStream_t stream);

// ---- allocation-free float64 Gram (gp_static.cu) --------------------------------
// Device pointers only; returns a GP_* status, *detail as in gp_last_error_detail.
int gp_static_gram(const double* X, const double* y, int64_t N, int p, int n, double eps,
                   double alpha, double* G, double* b, cudaStream_t stream, int64_t* detail);

// ---- factorisation, inverse and solve (gp_factor.cu) ---------------------------
// Device workspace (bytes) for launch_cholesky and launch_tri_inverse.
size_t factor_work_bytes(int M, bool fp32_inverse);
// In-place lower Cholesky of the M x M row-major matrix L (upper part ignored,
// then zeroed), float64, one cooperative launch. Non-positive pivot ->
// status GP_ENOTPD, detail = column. It zeroes the workspace header, which
// holds the grid barriers of launch_tri_inverse and launch_solve_refine too:
// those two run after it, on the same workspace.
// f32_update: the trailing-update products in float32, subtracted from the
// float64 trailing matrix (mixed-precision fits); the diagonal blocks and
// panel solves are float64 either way.
// max_ctas > 0 caps the grid of this and the two launches below (the
// batched fit runs several problems' factorisations side by side).
cudaError_t launch_cholesky(double* L, int M, GpStatus* st, void* work, cudaStream_t stream,
                            bool f32_update = false, int max_ctas = 0);
// Test hook of gp_debug_barrier_timeout: the Cholesky's bounded waits give up
// after limit_s seconds (<= 0: GP_WAIT_NS), and the next launch's CTA
// skip_cta (< 0: none) leaves before its first grid-barrier arrival.
void factor_debug_barrier_timeout(double limit_s, int skip_cta);
// W = L^{-1} (lower, M x M row-major, upper part zeroed), one cooperative
// launch: in float64 into W (fp32 = false), or in float32 into the workspace
// (fp32 = true; W is not written and may be NULL), where the solve finds it
// and its transpose.
cudaError_t launch_tri_inverse(const double* L, double* W, int M, bool fp32, GpStatus* st, void* work,
                               cudaStream_t stream, int max_ctas = 0);
// c = A^{-1} b through W = L^{-1}: c = W^T (W b), then `refine` steps of
// c += W^T W (b - A c) with the float64 residual, one cooperative launch.
// fp32: the products use the float32 W that launch_tri_inverse left in
// fwork (its workspace); otherwise W itself.
// fp32 with Wpack != NULL: also the predict kernel's operands into Wpack
// (predtc_wpack_bytes), from the float32 W and the final c.
cudaError_t launch_solve_refine(const double* A, const double* W, const void* fwork, bool fp32, const double* b,
                                double* c, double* work, int M, int refine, GpStatus* st, cudaStream_t stream,
                                uint16_t* Wpack = nullptr, int max_ctas = 0);
size_t solve_refine_work_elems(int M);

// ---- float64 predict (gp_predict64.cu) -----------------------------------------
constexpr int PRED64_TT = 64;   // test points per CTA
constexpr int PRED64_TK = 64;   // columns of Z = Phi_* W^T per CTA
size_t predict64_part_elems(int64_t Ns, int M);
// zout (optional): Z = Phi_* W^T, Npad x zld row-major, zld = 64 * ceil(M / 64)
cudaError_t launch_predict64(const GpShape& s, const double* tab, const double* W, const double* c,
                             double sigma2, double* part, double* mean, double* var,
                             cudaStream_t stream, double* zout = nullptr);
size_t predict64_z_elems(int64_t Npad, int M);

// ---- bf16x3 tensor-core predict (gp_predict_tc.cu) ------------------------------
constexpr int PREDTC_TT = 128;  // test points per CTA (MMA M)
constexpr int PREDTC_BK = 32;   // Phi_* columns per pipeline stage (MMA K chunk)
constexpr int PREDTC_KB = 128;  // rows of W per MMA (MMA N)
constexpr int PREDTC_SUPER = 4; // MMA N-blocks held in TMEM at once (4 x 128 = 512 columns)
size_t predtc_wpack_bytes(int M);
// The predict kernel's operands (predtc_wpack_bytes): bf16 hi/lo blocks of
// W = L^{-1} (pack_w_item in gp_tc.cuh), then c in float32 (Mpad floats, zero
// beyond M); written by the solve (launch_solve_refine) of a mixed fit.
size_t predtc_smem_bytes(const GpShape& s);
// Chunk table of the predict kernel (ints): built once per fitted model.
size_t predtc_cinfo_ints(const GpShape& s);
void predtc_build_cinfo(const GpShape& s, int* out);
// One predict request of a mixed-precision model, as the predict kernel and
// the batched table kernel read it (device tables of these, or one by value).
struct PredReq {
    int64_t Ns, Npad;       // test points; table rows (a multiple of 128)
    int p, n, M, Mpad;      // the model's basis; Mpad a multiple of 128
    int maxrows;            // the model's largest chunk window (= its zero window row)
    int pad_;
    const double* Xs;       // Ns x p test points
    const float* consts;    // 3p floats: rho_j beta_j, sqrt(beta_j), delta_j^2 (batched tables)
    float* tab;             // the eigenfunction tables of X*: (j n + k) Npad + i
    const uint8_t* Wpack;   // the model's operand blocks (predtc_wpack_bytes)
    const float* cf;        // the model's float32 c (in Wpack)
    const int* cinfo;       // the model's chunk table (predtc_build_cinfo)
    double sigma2;
    double* mean;           // Ns outputs
    double* var;            // Ns outputs, or NULL
    uint8_t* zpack;         // optional rows of Z (predtc_zpack_bytes)
    double* vpart;          // with var and more than one super-tile: the items' partial
                            // variances, predtc_vpart_elems (summed by the reduce launch)
    GpStatus* st;           // this request's status word
};
int predtc_window_rows(const GpShape& s);  // a model's PredReq::maxrows
// Super-tiles of W rows (512 each) of a model with M columns: the items of a
// request are its (128-point tile, super-tile) pairs when the variance or
// Z is wanted, else its tiles' last super-tiles only (the mean).
int predtc_nsuper(int M);
size_t predtc_vpart_elems(int64_t Npad, int M);  // 0 when there is one super-tile

// The batched form (one launch per basis dimension p): the kernel's CTAs walk
// items[0 .. nitems) = (request, tile * nsuper + super-tile) in a fixed
// round-robin order; maxrows_all bounds the requests' windows (it sizes the
// pipeline stages). Every request's p must equal `p`. Requests with several
// super-tiles and a variance then need launch_predict_reduce_batch.
cudaError_t launch_predict_tc_batch(const PredReq* reqs, const int2* items, int nitems, int p, int maxrows_all,
                                    cudaStream_t stream);
// var = sigma2 * (the sum of the partial variances over the super-tiles, in
// their order) for every request of the table with several super-tiles and a
// variance (max_npad bounds the requests' Npad).
void launch_predict_reduce_batch(const PredReq* reqs, int nreq, int64_t max_npad, cudaStream_t stream);
size_t predtc_batch_smem_bytes(int maxrows_all, int p);
// Tables of every request of a batch: the grid's blocks [boff[r], boff[r+1])
// belong to request r (256 points x one dimension each; boff has nreq + 1
// entries); max_n bounds the requests' n.
void launch_eig_tables_batch(const PredReq* reqs, const int* boff, int nreq, int nblocks, int max_n,
                             cudaStream_t stream);

// zpack (optional, predtc_zpack_bytes): the rows of Z = Phi_* W^T as bf16
// hi/lo, per 128-point tile and 32-column chunk an 8 KB hi block and an 8 KB
// lo block in the K-major core-matrix layout of a tcgen05 operand
// vpart: predtc_vpart_elems(s.Npad, s.M) doubles of scratch, needed when var
// is given and the model has more than one super-tile
cudaError_t launch_predict_tc(const GpShape& s, const float* tab, const uint16_t* Wpack,
                              const int* cinfo, double sigma2, double* mean, double* var,
                              GpStatus* st, cudaStream_t stream, uint8_t* zpack = nullptr,
                              double* vpart = nullptr);
size_t predtc_zpack_bytes(int64_t Npad, int M);

// ---- predictive covariance block (gp_cov.cu) ------------------------------------
// cov (Ns x Ns row-major, leading dimension Ns) = sigma2 Z Z^T (+ sigma2 on
// the diagonal when noisy): from the packed Z of launch_predict_tc (tensor
// cores, 128 x 128 tiles) or the float64 Z of launch_predict64 (CUDA cores)
cudaError_t launch_cov_tc(const uint8_t* zpack, int64_t Ns, int64_t Npad, int M, double sigma2, int noisy,
                          double* cov, GpStatus* st, cudaStream_t stream);
cudaError_t launch_cov64(const double* Z, int64_t Ns, int zld, double sigma2, int noisy, double* cov,
                         cudaStream_t stream);

// ---- log marginal likelihood terms (gp_lml.cu) ----------------------------------
// out[0..3] = y^T y, b^T c, sum_j log L_jj, sum_m log d_m (float64, fixed
// summation order), through nparts per-CTA partials in part (4 nparts doubles).
int lml_partial_count(int sms);
void launch_lml_terms(const double* y, int64_t N, const double* L, const double* b, const double* c,
                      const double* d, int M, int nparts, double* part, double* out, cudaStream_t stream);
// out[m] = (A^{-1})_mm = sum_k W_km^2 for W = L^{-1} (M x M row-major, lower;
// float32 or float64), in float64
void launch_ainv_diag(const void* W, bool fp32, int M, double* out, cudaStream_t stream);
// out[0..2] = c^T E c, tr(A^{-1} E), unclamped columns (E = d/sigma^2 on them),
// through nparts per-CTA partials in part (4 nparts doubles); out[3] = 0
void launch_lml_grad_terms(const double* c, const double* d, const double* ainv, double sigma2, int M, int nparts,
                           double* part, double* out, cudaStream_t stream);
