// gp_lml.cu -- the reductions of the log marginal likelihood of a fitted model.
//
// log p(y) = log N(y; 0, K + sigma^2 I) for the truncated kernel
// K = Phi Lambda Phi^T (Eq. 1-2, 7-9), the quantity that hyperparameter
// learning (named as future work in Sec. 4) maximises. With A = L L^T the
// fit's M x M matrix, b = Phi^T y, c = A^{-1} b and d_m = sigma^2 / lambda_m,
// the matrix determinant lemma and the Woodbury identity (Eq. 10) give
//   log p(y) = -1/2 [ (y^T y - b^T c) / sigma^2 + N log sigma^2
//                     + 2 sum_j log L_jj - sum_m log d_m + N log 2 pi ].
// The kernels here form the four sums in float64, in a fixed order (per-CTA
// partials in grid-stride order, then one CTA adds the partials), so the
// result does not depend on scheduling; the caller combines them.
#include "gp_kernels.cuh"

#include <math.h>

namespace {

constexpr int LML_NT = 256;

// block sum of v, in a fixed tree order; the result in thread 0
__device__ double block_sum(double v, double* sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int w = LML_NT / 2; w > 0; w >>= 1) {
        if (tid < w) sh[tid] += sh[tid + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// part[blockIdx.x][0..3] = this CTA's shares of y^T y, b^T c, sum log L_jj,
// sum log d_m (grid-stride over N and M)
__global__ void __launch_bounds__(LML_NT) lml_partials_kernel(const double* __restrict__ y, int64_t N,
                                                             const double* __restrict__ L,
                                                             const double* __restrict__ b,
                                                             const double* __restrict__ c,
                                                             const double* __restrict__ d, int M,
                                                             double* __restrict__ part) {
    __shared__ double sh[LML_NT];
    const int64_t stride = (int64_t)gridDim.x * LML_NT;
    const int64_t i0 = (int64_t)blockIdx.x * LML_NT + threadIdx.x;
    double yy = 0.0, bc = 0.0, ll = 0.0, ld = 0.0;
    for (int64_t i = i0; i < N; i += stride) yy = fma(y[i], y[i], yy);
    for (int64_t m = i0; m < M; m += stride) {
        bc = fma(b[m], c[m], bc);
        ll += log(L[m * (int64_t)M + m]);
        ld += log(d[m]);
    }
    const double s0 = block_sum(yy, sh), s1 = block_sum(bc, sh), s2 = block_sum(ll, sh), s3 = block_sum(ld, sh);
    if (threadIdx.x == 0) {
        double* o = part + 4 * (int64_t)blockIdx.x;
        o[0] = s0;
        o[1] = s1;
        o[2] = s2;
        o[3] = s3;
    }
}

// out[k] = sum over the nparts partials of term k, in partial order
__global__ void __launch_bounds__(LML_NT) lml_total_kernel(const double* __restrict__ part, int nparts,
                                                          double* __restrict__ out) {
    __shared__ double sh[LML_NT];
    for (int k = 0; k < 4; ++k) {
        double v = 0.0;
        for (int q = threadIdx.x; q < nparts; q += LML_NT) v += part[4 * (int64_t)q + k];
        const double s = block_sum(v, sh);
        if (threadIdx.x == 0) out[k] = s;
    }
}

// (A^{-1})_mm = sum_k (L^{-1})_km^2 (A = L L^T): the squared norm of column m
// of W = L^{-1} (lower triangular, row-major, rows k >= m), in float64 in
// increasing k; one thread per column, consecutive threads read consecutive
// columns of a row.
template <typename T>
__global__ void __launch_bounds__(LML_NT) ainv_diag_kernel(const T* __restrict__ W, int M,
                                                          double* __restrict__ out) {
    const int m = blockIdx.x * LML_NT + threadIdx.x;
    if (m >= M) return;
    double acc = 0.0;
    for (int k = m; k < M; ++k) {
        const double w = (double)W[(int64_t)k * M + m];
        acc = fma(w, w, acc);
    }
    out[m] = acc;
}

// part[blockIdx.x][0..2] = this CTA's shares of c^T E c, tr(A^{-1} E) and the
// number of unclamped columns, with E = diag(e), e_m = d_m / sigma^2 where
// d_m < 1e200 (d_m = sigma^2 / lambda_m moves with sigma^2) and 0 where d_m
// is clamped (it does not)
__global__ void __launch_bounds__(LML_NT) lml_grad_partials_kernel(const double* __restrict__ c,
                                                                  const double* __restrict__ d,
                                                                  const double* __restrict__ ainv, double inv_s2,
                                                                  int M, double* __restrict__ part) {
    __shared__ double sh[LML_NT];
    const int64_t stride = (int64_t)gridDim.x * LML_NT;
    const int64_t i0 = (int64_t)blockIdx.x * LML_NT + threadIdx.x;
    double cec = 0.0, tr = 0.0, nu = 0.0;
    for (int64_t m = i0; m < M; m += stride) {
        if (d[m] < 1e200) {
            const double e = d[m] * inv_s2;
            cec = fma(e * c[m], c[m], cec);
            tr = fma(e, ainv[m], tr);
            nu += 1.0;
        }
    }
    const double s0 = block_sum(cec, sh), s1 = block_sum(tr, sh), s2 = block_sum(nu, sh);
    if (threadIdx.x == 0) {
        double* o = part + 4 * (int64_t)blockIdx.x;
        o[0] = s0;
        o[1] = s1;
        o[2] = s2;
        o[3] = 0.0;
    }
}

}  // namespace

int lml_partial_count(int sms) { return sms > 0 ? sms : 1; }

void launch_ainv_diag(const void* W, bool fp32, int M, double* out, cudaStream_t stream) {
    const unsigned g = (unsigned)((M + LML_NT - 1) / LML_NT);
    if (fp32)
        ainv_diag_kernel<float><<<g, LML_NT, 0, stream>>>((const float*)W, M, out);
    else
        ainv_diag_kernel<double><<<g, LML_NT, 0, stream>>>((const double*)W, M, out);
}

void launch_lml_grad_terms(const double* c, const double* d, const double* ainv, double sigma2, int M, int nparts,
                           double* part, double* out, cudaStream_t stream) {
    lml_grad_partials_kernel<<<(unsigned)nparts, LML_NT, 0, stream>>>(c, d, ainv, 1.0 / sigma2, M, part);
    lml_total_kernel<<<1, LML_NT, 0, stream>>>(part, nparts, out);
}

void launch_lml_terms(const double* y, int64_t N, const double* L, const double* b, const double* c,
                      const double* d, int M, int nparts, double* part, double* out, cudaStream_t stream) {
    lml_partials_kernel<<<(unsigned)nparts, LML_NT, 0, stream>>>(y, N, L, b, c, d, M, part);
    lml_total_kernel<<<1, LML_NT, 0, stream>>>(part, nparts, out);
}
