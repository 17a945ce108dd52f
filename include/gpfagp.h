/*
 * gpfagp.h -- C ABI of the GB300 decomposed-kernel (FAGP) Gaussian process.
 *
 * The library fits and evaluates the Gaussian-process posterior of Sec. 2.2
 * of "Parallel Gaussian Process with Kernel Approximation in CUDA"
 * (arXiv 2403.12797) with the squared-exponential kernel expanded in its
 * Hermite eigenfunctions (Sec. 2.3, Eq. 14-16), taken as a tensor product
 * over the p input dimensions (Eq. 18-20): M = n^p basis columns.
 *
 *   fit:      Phi (N x M, never stored), A = Phi^T Phi + sigma^2 Lambda^{-1},
 *             b = Phi^T y, A = L L^T, c = A^{-1} b          (Eq. 10-12, Woodbury form)
 *   predict:  mean_i = phi(x*_i)^T c,
 *             var_i  = sigma^2 |L^{-1} phi(x*_i)|^2           (diagonal of Eq. 12)
 *
 * Conventions shared by every entry point
 *  - X and X* are row-major (N x p), (Ns x p) float64; y, mean, var float64.
 *  - alpha is the eigen-decomposition's global scale factor (rho, Sec. 2.3);
 *    eps the SE shape parameter (epsilon, Eq. 13); sigma2 the noise
 *    variance (sigma^2, Eq. 1). One eps and one alpha serve all dimensions.
 *  - The column order of Phi is m = sum_j m_j n^(p-1-j) (last dimension
 *    fastest); results do not depend on it.
 *  - Ownership: the caller owns every array it passes; the library copies
 *    what it needs and keeps no caller pointer after a call returns. A
 *    gp_model is owned by the library until gp_free.
 *  - Errors: every int-returning call returns GP_OK (0) or a negative
 *    status; gp_last_error() returns the calling thread's last status and
 *    gp_last_error_detail() an integer detail (the failing pivot column for
 *    GP_ENOTPD, the CUDA error code for GP_ECUDA). No call traps or aborts.
 *  - Streams: the _ex variants take a cudaStream_t (NULL = the legacy
 *    default stream). With dev_ptrs = 1 all array arguments are device
 *    pointers and the call is asynchronous with respect to the host except
 *    for the final status read back (one 8-byte device-to-host copy);
 *    with dev_ptrs = 0 they are host pointers and the call returns after
 *    the results are in host memory.
 *  - Thread safety: a fitted gp_model is immutable; concurrent predicts on
 *    the same model (on different streams) are safe.
 */
#ifndef GPFAGP_H
#define GPFAGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GPFAGP_API __attribute__((visibility("default")))
#else
#define GPFAGP_API
#endif

typedef struct gp_model gp_model;

/* ---- status codes ------------------------------------------------------- */
#define GP_OK        0
#define GP_EINVAL   (-1)  /* bad argument: N<1, p<1, n<1, p>32, M=n^p > GP_MAX_M,
                             non-finite or non-positive eps/alpha/sigma2,
                             NaN/Inf in X, y or X* (detected on the device)   */
#define GP_ENOMEM   (-2)  /* a device allocation failed                       */
#define GP_ENOTPD   (-3)  /* A is not numerically positive definite; detail =
                             first failing pivot column                         */
#define GP_ECUDA    (-4)  /* a CUDA runtime call failed; detail = cudaError_t  */
#define GP_ETIMEOUT (-5)  /* a bounded device-side wait ran out (pipeline
                             barrier of a tensor-core kernel)                   */
#define GP_ENODEV   (-6)  /* no usable sm_103 device                           */

/* ---- precision modes ---------------------------------------------------- */
/* GP_PREC_FP64:  every step in float64 on the CUDA cores.
 * GP_PREC_MIXED: Phi generated in float32; the contractions run on the
 *                tensor cores with 16-bit operands:
 *                - Phi^T Phi: within each row block (1024 rows, or 4096 on
 *                  CTA pairs) every column is scaled by the power of two
 *                  that its exact block maximum sets, so that |w| < 64, and
 *                  split into the integer s1 = rint(w) (exact in fp16) and
 *                  lo = fp16(w - s1); s1*s1' is summed EXACTLY in float32
 *                  TMEM over the block, s1*lo' + lo*s1' + lo*lo' beside it;
 *                  the block sums are rescaled exactly and folded into float
 *                  pairs hi + lo by an exact two-sum (no truncation drift);
 *                - Phi_* L^{-T} (variance): bf16 hi/lo split of both
 *                  operands, hi*hi + hi*lo + lo*hi in float32;
 *                Phi^T y and the predictive mean use float32 products;
 *                split-N partials are summed and A assembled in float64;
 *                the Cholesky keeps its trailing matrix in float64 and
 *                takes its pivots and panel solves (on power-of-two
 *                equilibrated blocks and rows) and its update products in
 *                float32; W = L^{-1} is float32; c is solved through W and
 *                refined against A in float64. A mixed fit whose float32
 *                pivot is not a positive normal number redoes its Gram and
 *                factorisation in float64.                                 */
#define GP_PREC_FP64   0
#define GP_PREC_MIXED  3

/* Largest supported M = n^p (the M x M float64 factor must fit in memory). */
#define GP_MAX_M  32768

/* ---- spec entry points -------------------------------------------- */

/* Fit the posterior of Sec. 2.2 on host arrays X (N x p) and y (N), in the
 * GP_PREC_MIXED mode on the current device and the legacy default stream.
 * Returns a model handle, or NULL on failure (gp_last_error() tells why). */
GPFAGP_API gp_model* gp_fit(const double* X, const double* y, int64_t N, int p, int n,
                            double eps, double alpha, double sigma2);

/* Predictive mean and variance (Eq. 11-12, diagonal) at Ns host points Xs
 * (Ns x p) into host arrays mean (Ns) and var (Ns). var may be NULL (the
 * variance is then not computed). Ns = 0 is a no-op. */
GPFAGP_API int gp_predict(const gp_model* h, const double* Xs, int64_t Ns,
                          double* mean, double* var);

/* Release a model (NULL is a no-op). Synchronises the model's device. */
GPFAGP_API void gp_free(gp_model* h);

GPFAGP_API int gp_last_error(void);
GPFAGP_API int64_t gp_last_error_detail(void);
/* For GP_ECUDA: the library step whose CUDA call failed (static string,
 * "" otherwise). */
GPFAGP_API const char* gp_last_error_where(void);
GPFAGP_API const char* gp_strerror(int status);

/* ---- extended entry points ---------------------------------------------- */

/* gp_fit with an explicit precision mode, stream and pointer kind.
 * On GP_OK *out receives the model. */
GPFAGP_API int gp_fit_ex(const double* X, const double* y, int64_t N, int p, int n,
                         double eps, double alpha, double sigma2, int prec,
                         void* cuda_stream, int dev_ptrs, gp_model** out);

/* gp_fit_ex for the ARD kernel (Eq. 17): eps[j] and alpha[j], j = 0 .. p-1
 * (host arrays of p values, copied), give dimension j its own SE shape
 * parameter epsilon_j and eigen-decomposition scale rho_j, hence its own
 * eigenvalues and eigenfunctions (Eq. 14-16 per dimension); the
 * tensor-product basis (Eq. 18-20) and everything after it are unchanged.
 * With all eps[j] equal and all alpha[j] equal it computes exactly what
 * gp_fit_ex computes. The model predicts, reports its likelihood and serves
 * like any other. Errors as gp_fit_ex (GP_EINVAL for a non-positive or
 * non-finite eps[j] or alpha[j], or NULL arrays). */
GPFAGP_API int gp_fit_ard_ex(const double* X, const double* y, int64_t N, int p, int n,
                             const double* eps, const double* alpha, double sigma2, int prec,
                             void* cuda_stream, int dev_ptrs, gp_model** out);

/* gp_predict with an explicit stream and pointer kind. The prediction uses
 * the model's precision mode. */
GPFAGP_API int gp_predict_ex(const gp_model* h, const double* Xs, int64_t Ns,
                             double* mean, double* var, void* cuda_stream, int dev_ptrs);

/* The full predictive covariance block of Eq. 12 at Ns test points:
 *   cov[i * Ns + j] = sigma^2 phi(x*_i)^T A^{-1} phi(x*_j)
 * (Ns x Ns, row-major, exactly symmetric, the covariance of the latent f;
 * with noisy != 0, sigma^2 is added on the diagonal: the covariance of the
 * noisy observations y*). Its diagonal is gp_predict_ex's variance, up to
 * the precision mode's rounding. Formed as sigma^2 Z Z^T with
 * Z = Phi_* L^{-T}: the mixed model takes Z from the predict kernel as
 * bf16 hi/lo and multiplies on the tensor cores (hi*hi + hi*lo + lo*hi,
 * float32 accumulation); the float64 model in float64. mean (Ns values) may
 * be NULL; it is the predictive mean as gp_predict_ex computes it. Xs, mean
 * and cov are device pointers when dev_ptrs != 0, else host (cov then needs
 * Ns^2 doubles of device scratch). GP_EINVAL for Ns > GP_COV_MAX_NS
 * (detail 6), a NULL Xs or cov, or a model on another device (detail 5). */
#define GP_COV_MAX_NS 65536
GPFAGP_API int gp_predict_cov_ex(const gp_model* h, const double* Xs, int64_t Ns,
                                 double* mean, double* cov, int noisy,
                                 void* cuda_stream, int dev_ptrs);

/* gp_fit_ex followed by gp_predict_ex on the fitted model (Sec. 2.2 and
 * Eq. 8-9, the same kernels), with the prediction enqueued right behind the
 * fit and a single status read at the end, so the device does not wait for
 * the host between the two. Arguments as in gp_fit_ex (X, y, N, ...,
 * dev_ptrs, out) and gp_predict_ex (Xs, Ns, mean, var; var may be NULL);
 * every pointer is of the kind dev_ptrs names. A mixed fit that the float64
 * Gram must redo (see gp_model_flags) is redone, and its prediction with it.
 * On GP_OK *out receives the model and mean/var hold the prediction; on
 * error *out is NULL and mean/var are unspecified. */
GPFAGP_API int gp_fit_predict_ex(const double* X, const double* y, int64_t N, int p, int n,
                                 double eps, double alpha, double sigma2, int prec,
                                 const double* Xs, int64_t Ns, double* mean, double* var,
                                 void* cuda_stream, int dev_ptrs, gp_model** out);

/* Log marginal likelihood of the fitted model: log p(y) = log N(y; 0,
 * K + sigma^2 I) for the truncated kernel K = Phi Lambda Phi^T (Eq. 1-2,
 * 7-9), the quantity hyperparameter learning maximises (Sec. 4, future
 * work). From the fit's factors, by the matrix determinant lemma and the
 * Woodbury identity (Eq. 10):
 *   log p(y) = -1/2 [ (y^T y - b^T c) / sigma^2 + N log sigma^2
 *                     + 2 sum_j log L_jj - sum_m log d_m + N log 2 pi ].
 * y: the N training targets the model was fitted on (the model does not keep
 * them), host or device memory per dev_ptrs. The sums run on the device in
 * float64 in a fixed order; *out receives log p(y). Returns GP_OK, GP_EINVAL
 * (NULL h, y or out, or N different from the fit's), or an error status. */
GPFAGP_API int gp_model_log_marginal(const gp_model* h, const double* y, int64_t N, double* out,
                                     void* cuda_stream, int dev_ptrs);

/* log p(y) as gp_model_log_marginal, and its derivative with respect to the
 * noise variance sigma^2 at fixed eps and alpha -- the noise part of the
 * gradient that hyperparameter learning follows (Sec. 4, future work).
 * Differentiating the terms above, with A = G + diag(d), d_m = sigma^2 /
 * lambda_m and E = dA / d sigma^2 = diag(e), e_m = d_m / sigma^2 (0 where d_m
 * is clamped at 1e200):
 *   d log p / d sigma^2 = -1/2 [ c^T E c / sigma^2 - (y^T y - b^T c) / sigma^4
 *                                + N / sigma^2 + tr(A^{-1} E) - n_u / sigma^2 ],
 * n_u the unclamped columns, tr(A^{-1} E) = sum_m e_m |W[:, m]|^2 with
 * W = L^{-1}. The float64 model keeps W; for a mixed model W is formed again
 * from L in float64 during the call (float32's exponent range loses
 * (A^{-1})_mm where d_m nears its clamp, and the gradient weights those
 * entries by d_m / sigma^2). Sums in
 * float64, fixed order. y, N, pointer kind and errors as
 * gp_model_log_marginal; *lml and *dlml_dsigma2 receive the results. */
GPFAGP_API int gp_model_log_marginal_grad(const gp_model* h, const double* y, int64_t N, double* lml,
                                          double* dlml_dsigma2, void* cuda_stream, int dev_ptrs);

/* Model shape and mode: any output pointer may be NULL. */
GPFAGP_API int gp_model_info(const gp_model* h, int64_t* M, int* p, int* n, int* prec);

/* Model flags: GP_MODEL_GRAM_FP64 when a mixed-precision fit recomputed its
 * Gram in float64. The mixed Gram keeps its row-block sums exact and folds
 * the blocks into ~46-bit float pairs; when A = G + sigma^2 Lambda^{-1} is
 * conditioned beyond what that and the float32 pivots carry (large N with a
 * small noise variance) the Cholesky meets a pivot that is not a positive
 * normal number, and the fit (gp_fit_ex, gp_fit_batch, server refits) then
 * redoes the Gram with the float64 kernel and factors again in float64
 * instead of failing. */
#define GP_MODEL_GRAM_FP64 1
GPFAGP_API int gp_model_flags(const gp_model* h);

/* Copy a fitted quantity of the model to host memory, in float64.
 *   GP_FIELD_L: the Cholesky factor L (M x M row-major, lower; upper = 0)
 *   GP_FIELD_C: c = A^{-1} b (M)
 *   GP_FIELD_B: b = Phi^T y (M)
 *   GP_FIELD_D: the diagonal sigma^2 / lambda_m (clamped at 1e200) (M)
 * dst must hold M*M (L) or M (others) doubles. */
#define GP_FIELD_L 1
#define GP_FIELD_C 2
#define GP_FIELD_B 3
#define GP_FIELD_D 4
GPFAGP_API int gp_model_read(const gp_model* h, int field, double* dst);

/* The fused Phi generation + contraction step on its own (Sec. 2.2: the
 * Phi^T Sigma_n^{-1} Phi and Phi^T y products of Lambda-bar and W):
 * G = Phi^T Phi (M x M, full symmetric, row-major) and b = Phi^T y (M),
 * in float64, computed in mode prec. Pointer kind as in gp_fit_ex. */
GPFAGP_API int gp_gram_ex(const double* X, const double* y, int64_t N, int p, int n,
                          double eps, double alpha, int prec, double* G, double* b,
                          void* cuda_stream, int dev_ptrs);

/* ---- allocation-free Gram ------------------------------------------------- */

/* Size of the library's fixed device scratch array used by gp_gram_static. */
#define GP_STATIC_SCRATCH_BYTES (32u << 20)

/* gp_gram_ex in GP_PREC_FP64 mode for callers that cannot allocate device
 * memory during the call (a fixed, pre-carved memory budget, a real-time
 * loop that must not enter the allocator, an allocator hook that must not
 * be re-entered). The paper has no counterpart: this is a deployment
 * variant of the Gram step. It calls no cudaMalloc/cudaFree (nor any
 * allocating library routine): its scratch (tables, partial tiles, status)
 * lives in one static device array of GP_STATIC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.
 *   X (N x p), y (N): device inputs; G (M x M) and b (M): device outputs,
 *   same layout and meaning as gp_gram_ex. Returns after the results are
 *   written (the status word is read back).
 * Errors: GP_EINVAL for bad arguments and for problems whose scratch would
 * exceed GP_STATIC_SCRATCH_BYTES (gp_last_error_detail() = the bytes needed).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current: make it before any
 * stream capture. The address is kept for the life of the process, so do
 * not call this again after resetting the device (cudaDeviceReset). Every
 * call shares the one array, so calls that overlap on the GPU race;
 * serialise them. */
GPFAGP_API int gp_gram_static(const double* X, const double* y, int64_t N, int p, int n,
                              double eps, double alpha, double* G, double* b, void* cuda_stream);

/* ---- batched fit -------------------------------------------------------- */

/* One independent problem of a batched fit. Pointer kind as in the call. */
/* Fit from a given Gram: G = Phi^T Phi (M x M, full symmetric, row-major,
 * float64) and b = Phi^T y (M) of N training rows -- e.g. the sums of the
 * per-GPU Grams of a row-sharded training set after one all-reduce (each
 * rank then factors the same A). Continues the fit exactly as gp_fit_ex does
 * after its Gram step: A = G + sigma^2 Lambda^{-1} (Eq. 11, 16), Cholesky,
 * W = L^{-1}, c with float64 refinement. G and b are device pointers when
 * dev_ptrs != 0, else host pointers; they are copied, not kept. Errors as
 * gp_fit_ex (GP_ENOTPD when G + diag(d) is not positive definite). */
GPFAGP_API int gp_fit_gram_ex(const double* G, const double* b, int64_t N, int p, int n, double eps,
                              double alpha, double sigma2, int prec, void* cuda_stream, int dev_ptrs,
                              gp_model** out);

/* The exchange step of a row-sharded fit, in one buffer. G = Phi^T Phi and
 * b = Phi^T y are sums over training rows (Sec. 2.2), so ranks that hold
 * disjoint row blocks of one training set sum their partial Grams with one
 * all-reduce of M (M + 1) / 2 + M float64 values and then each factor the
 * same A.
 * gp_gram_packed_ex: the Gram of X (N x p), y (N), as gp_gram_ex computes
 *   it, written as packed[i (i + 1) / 2 + j] = G[i][j] for j <= i (the lower
 *   triangle row by row), then packed[M (M + 1) / 2 + m] = b[m].
 * gp_fit_gram_packed_ex: gp_fit_gram_ex from such a buffer (N = all ranks'
 *   rows together).
 * Pointers are device pointers when dev_ptrs != 0, else host; errors as
 * gp_gram_ex and gp_fit_gram_ex. */
GPFAGP_API int gp_gram_packed_ex(const double* X, const double* y, int64_t N, int p, int n,
                                 double eps, double alpha, int prec, double* packed,
                                 void* cuda_stream, int dev_ptrs);
GPFAGP_API int gp_fit_gram_packed_ex(const double* packed, int64_t N, int p, int n, double eps,
                                     double alpha, double sigma2, int prec, void* cuda_stream,
                                     int dev_ptrs, gp_model** out);

typedef struct gp_fit_args {
    const double* X;   /* N x p */
    const double* y;   /* N     */
    int64_t N;
    int p, n;
    double eps, alpha, sigma2;
} gp_fit_args;

/* Fit `count` independent problems of uneven N, p and n (and precision
 * `prec` for all) side by side (Sec. 2.2 per problem).
 *   - Inputs, model buffers and the shape-only tables are staged first.
 *   - Mixed precision runs stage-major: every problem's eigenfunction tables
 *     and column exponents on its stream; then the Grams of ALL problems in
 *     one tensor-core launch per basis dimension p, whose CTAs find their
 *     (problem, tile pair, row split) in a device table of the problems --
 *     each problem's splits sized to its share of k waves of the GPU in
 *     proportion to its contraction work; then every problem's assembly,
 *     Cholesky, inverse and solve on its stream. Float64: each problem's own
 *     steps on its stream.
 *   - The plan (streams S in {8, 16, 32}, at most `count`; k in {1, 2, 4};
 *     and whether each problem's Cholesky, inverse and solve run on at most
 *     max(4, SMs / S) CTAs, so that more problems' factorisations overlap)
 *     comes from an autotuner that runs the whole batch once per
 *     candidate after one untimed warm-up run, timed on the host clock from
 *     call to return, the first time a batch of its kind is seen (the
 *     multiset of p, n, N rounded down to a power of two and precision, on
 *     the same GPU model and library version). It keeps the fastest for the
 *     process and, if the environment variable GPFAGP_TUNE_CACHE names a
 *     file, appends it there and reads that file in later processes
 *     (gp_batch_plan reports the plan and whether it came from the cache).
 *   - The run is captured into ONE CUDA graph and launched once; if CUDA
 *     refuses to capture or instantiate it, the same launches run directly
 *     on the streams (gp_batch_info reports which ran).
 *   - All statuses are read back once at the end; a mixed problem whose
 *     Cholesky met a non-positive pivot is refit with the float64 Gram.
 * out[i] receives problem i's model, or NULL if it failed; the return value
 * is GP_OK when every problem succeeded, else the first failing problem's
 * status with gp_last_error_detail() = its index. X, y are device pointers
 * when dev_ptrs != 0, else host pointers (copied during the call). Each
 * model equals the one gp_fit_ex computes for the same problem up to the
 * order of the Gram's split sums (the plan's split count), i.e. within the
 * precision mode's tolerance. Blocks until the batch has run. */
GPFAGP_API int gp_fit_batch(int count, const gp_fit_args* args, int prec,
                            void* cuda_stream, int dev_ptrs, gp_model** out);

/* Of the last gp_fit_batch on this thread: *used_graph = 1 if the batch ran
 * as one captured graph (0 if directly on streams), *tuned_k = the Gram
 * budget factor of its plan. Either pointer may be NULL. */
GPFAGP_API int gp_batch_info(int* used_graph, int* tuned_k);

/* Of the last gp_fit_batch on this thread: its plan (*streams, *k; k = 0
 * for float64 batches; *factor_ctas = the CTA cap of each problem's
 * Cholesky, inverse and solve, 0 if uncapped), *from_cache = 1 if the plan
 * came from the tuning cache (this process's or GPFAGP_TUNE_CACHE's) rather
 * than from timing the candidates in this call, and *tuned_ms = the plan's
 * timed run (host time from call to return). Any pointer may be NULL. */
GPFAGP_API int gp_batch_plan(int* streams, int* k, int* factor_ctas, int* from_cache, double* tuned_ms);

/* One predict request of a batched predict. */
typedef struct gp_predict_args {
    const gp_model* model;
    const double* Xs;  /* Ns x p */
    int64_t Ns;
    double* mean;      /* Ns */
    double* var;       /* Ns, or NULL */
} gp_predict_args;

/* Run `count` predict requests against (possibly different) models as one
 * batch (Eq. 11-12 per request). The requests against mixed-precision
 * models share one upload of a request table, one launch that evaluates
 * every request's eigenfunction tables, and one persistent tensor-core
 * predict launch per basis dimension p among them, whose CTAs walk the
 * (request, 128-point tile) items, heavier models first. Requests against
 * float64 models run their own kernels on up to 8 streams behind
 * `cuda_stream`. The call then waits once and reads every request's
 * status. Device pointers only. Each result is bitwise the same as
 * gp_predict_ex on that request alone (the same per-point arithmetic in the
 * same order). Returns the first failing request's status (detail = its
 * index; GP_EINVAL with detail 7 if a model's predict stages do not fit in
 * shared memory). */
GPFAGP_API int gp_predict_batch(int count, const gp_predict_args* args, void* cuda_stream);

/* ---- request server (continuous batching over resident models) ----------- */

/* A server keeps fitted models resident on the device and runs predict and
 * refit requests on `slots` CUDA streams from a worker thread. Requests queue
 * in arrival order; the queue head is admitted as soon as a slot is free and
 * its scratch-memory estimate fits under the budget (always, when nothing is
 * running), so requests that arrive while others run start as room frees up
 * and the admitted ones overlap on the device. Every request runs exactly the
 * kernels of gp_predict_ex / gp_fit_ex with the same launch plans, so its
 * result does not depend on the mix it ran in. Host buffers are staged
 * through pinned memory; the caller keeps them alive until gp_server_wait
 * has returned for the request. A refit fits a new model on the resident
 * model's p, n, eps, alpha, sigma2 and precision and swaps it in at
 * completion; predicts admitted before the swap finish on the old model,
 * which is freed after them. gp_server_add_model hands the model to the
 * server: the caller must not free it; gp_server_destroy frees every model
 * the server holds. gp_server_model returns the model currently serving an
 * id (valid until the next refit of that id completes or the server is
 * destroyed). */
typedef struct gp_server gp_server;

typedef struct gp_server_report {
    int64_t predicts_done;  /* finished predict requests (GP_OK)            */
    int64_t refits_done;    /* finished refits                              */
    int64_t points;         /* test points of the finished predicts         */
    double p50_ms, p99_ms, max_ms;  /* predict latency, submit to results   */
    double wall_s;          /* first submit to last completion              */
    double points_per_s;    /* points / wall_s                              */
    int peak_inflight;      /* most requests on the device at once          */
    int peak_batch;         /* most predicts in one batch                   */
    int64_t batches;        /* predict batches started                      */
} gp_server_report;

/* slots: 1..64 concurrent jobs (a refit, or a batch of the predicts queued
 * at the head: up to 256 requests and 2^20 points, all test points in one
 * upload, one table launch and one persistent predict launch per basis
 * dimension p, all results in one download); mem_budget_bytes: scratch
 * budget (<= 0: half the free device memory at creation). */
GPFAGP_API int gp_server_create(int slots, int64_t mem_budget_bytes, gp_server** out);
/* Register (and hand over) a fitted model; *model_id identifies it in requests. */
GPFAGP_API int gp_server_add_model(gp_server* s, gp_model* m, int* model_id);
/* The model currently serving model_id (changes when a refit completes). */
GPFAGP_API gp_model* gp_server_model(gp_server* s, int model_id);
/* Queue a predict of Ns >= 1 host rows Xs (Ns x p); mean (and var, or NULL)
 * are host outputs of Ns doubles, written before gp_server_wait returns. */
GPFAGP_API int gp_server_submit_predict(gp_server* s, int model_id, const double* Xs, int64_t Ns,
                                        double* mean, double* var, int64_t* req_id);
/* Queue a refit of model_id on N host rows X (N x p), y (N). */
GPFAGP_API int gp_server_submit_refit(gp_server* s, int model_id, const double* X, const double* y,
                                      int64_t N, int64_t* req_id);
/* Wait for a request (timeout_s <= 0: no limit); returns its status
 * (GP_ETIMEOUT if the limit passed first; the request stays queued). */
GPFAGP_API int gp_server_wait(gp_server* s, int64_t req_id, double timeout_s);
GPFAGP_API int gp_server_stats(gp_server* s, gp_server_report* out);
/* Start a new measurement window (requests still running are not counted). */
GPFAGP_API int gp_server_reset_stats(gp_server* s);
/* Finish every queued request, then stop the worker and release the streams. */
GPFAGP_API void gp_server_destroy(gp_server* s);

/* ---- test hooks ----------------------------------------------------------- */

/* Make the k-th device allocation from now fail with GP_ENOMEM (k >= 1);
 * k = 0 disarms. For error-path tests. */
GPFAGP_API void gp_debug_fail_alloc_after(int k);

/* Make the next k mixed-precision fits report a non-positive pivot on their
 * first attempt (k = 0 disarms), to exercise the float64 escalation. */
GPFAGP_API void gp_debug_force_escalation(int k);

/* Test hook: which mixed-precision Gram kernel the fits run. 0 (default):
 * automatic -- for M > 384 (p <= 4) a cluster of two CTAs per 256 x 256 tile
 * pair of G (tcgen05 cta_group::2), else one CTA per 128 x 128 tile pair;
 * 1: always one CTA per 128 x 128 tile pair; 2: CTA pairs wherever they
 * apply (p <= 4). Both compute the same arithmetic (the mixed mode above);
 * the tests compare them with each other and with the FP64 oracle. */
GPFAGP_API void gp_debug_gram_kernel(int kind);

/* Failure-detection test hook: the Cholesky's bounded grid-barrier
 * waits give up after limit_s seconds (limit_s <= 0 restores the 2 s
 * default), and in the next Cholesky launch the CTA with index skip_cta
 * (skip_cta < 0: none) returns before its first grid-barrier arrival, so
 * that the other CTAs' waits run out: the call then returns GP_ETIMEOUT
 * (detail 100, the grid barrier) and the device stays usable. Nothing
 * faults or hangs. The skip is one-shot; the limit stays until reset. */
GPFAGP_API void gp_debug_barrier_timeout(double limit_s, int skip_cta);

/* Test hook, host only: the mixed Gram's row-split plan for T 128-column tile
 * rows, Npad padded rows and a budget of target_ctas CTAs. out[0..2]: split
 * counts of the pair classes (0 diagonal, 1 pairs (I, 0), 2 other pairs),
 * out[3..5]: their rows per split, out[6]: the CTAs of the launch. Returns
 * GP_OK, or GP_EINVAL for T < 1, Npad < 1, target_ctas < 1 or out NULL. */
GPFAGP_API int gp_debug_gram_splits(int T, int64_t Npad, int target_ctas, int64_t* out);

/* Test hook: the mixed Gram's column exponents for the rows X (N x p,
 * row-major float64, host) and the hyperparameters (n, eps, alpha), as the
 * fits form them: for every 1024-row block b (rows padded to a multiple of
 * 128 are zero) and column m < M = n^p, ebx[b * M + m] = E, where the exact
 * maximum of |Phi[i, m]| over the block's rows (Eq. 19, float32 tables)
 * times (1 + 2^-20) lies in [2^(E-1), 2^E), except that E is at least -100
 * (a column that is zero in the block, or below 2^-101 there, gets -100). ebx4[b * M + m]: the largest E of each
 * 4096-row block (the CTA-pair kernel's); colexp[m]: the largest E over all
 * blocks. ebx holds ceil(Npad / 1024) x M bytes, ebx4 ceil(Npad / 4096) x M,
 * colexp M ints (Npad = N rounded up to 128); all are host memory owned by
 * the caller. Returns GP_OK, GP_EINVAL for bad arguments, or a CUDA error. */
GPFAGP_API int gp_debug_column_exponents(const double* X, int64_t N, int p, int n, double eps, double alpha,
                                         signed char* ebx, signed char* ebx4, int* colexp);

/* Library build tag (static string). *//* Library build tag (static string). */
GPFAGP_API const char* gp_version(void);

/* ---- measurement hooks ------------------------------------------------------ */

/* Number of CUDA kernels this library has launched since it was loaded. */
GPFAGP_API int64_t gp_kernel_launches(void);

/* Enable (1) or disable (0) CUDA-event timing of the library's kernel groups:
 * "eig_tables", "syrk64", "syrk_tc", "assemble", "cholesky", "tri_inverse",
 * "solve_refine", "pack_w", "predict64", "predict_tc". Each group is bracketed
 * by two events on the stream it runs on. */
GPFAGP_API void gp_profile_enable(int on);
/* Clear the accumulated group timings. */
GPFAGP_API void gp_profile_reset(void);
/* Wait for the recorded events of group `name` and report how many times it
 * ran and its total device time in milliseconds since the last reset.
 * Returns GP_EINVAL (and zeros) if the group has not run. */
GPFAGP_API int gp_profile_query(const char* name, int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* GPFAGP_H */
