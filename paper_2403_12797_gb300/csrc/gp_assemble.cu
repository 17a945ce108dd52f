// gp_assemble.cu -- split-N reduction and assembly of A = Phi^T Phi + sigma^2 Lambda^{-1}.
//
// A is sigma^2 times the Lambda-bar of Sec. 2.2 (with Sigma_n = sigma^2 I);
// its diagonal term d_m = sigma^2 / lambda_m uses the tensor-product
// eigenvalues lambda_m = prod_j lambda_{m_j} of Eq. 20 with lambda_k of
// Eq. 16, evaluated in log space and clamped at 1e200 so that eigenvalues
// that underflow stay finite.
//
// The partial Gram tiles of the N splits are summed in split order (float64
// for the float64 Gram, float pairs for the mixed one), so the result does
// not depend on scheduling. The mixed fit's assembly also forms d itself
// (one warp per diagonal block) and writes A's lower triangle into L, the
// Cholesky's input, which saves a kernel and a copy per fit.
#include "gp_kernels.cuh"

#include <math.h>

namespace {

// a partial value as float64 (float pairs hold hi + lo)
__device__ __forceinline__ double to_f64(double v) { return v; }

template <typename P, typename PB = P>
__global__ void __launch_bounds__(256) assemble_kernel(const P* __restrict__ Gpart,
                                                       const PB* __restrict__ bpart,
                                                       const PB* __restrict__ dpart,
                                                       const int* __restrict__ colexp, int nsplit,
                                                       int tile, int Mpad, int M,
                                                       const double* __restrict__ d,
                                                       double* __restrict__ A,
                                                       double* __restrict__ b) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y;
    if (col >= M) return;
    const int T = Mpad / tile;
    const int npairs = T * (T + 1) / 2;
    // read the lower-triangle element (r >= c), so A is exactly symmetric
    const int r = row >= col ? row : col;
    const int c = row >= col ? col : row;
    const int I = r / tile, J = c / tile;
    const int q = I * (I + 1) / 2 + J;
    const int64_t off = (int64_t)q * tile * tile + (int64_t)(r % tile) * tile + (c % tile);
    const int64_t sstride = (int64_t)npairs * tile * tile;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += to_f64(Gpart[off + s * sstride]);
    if (row == col && dpart != nullptr)
        for (int s = 0; s < nsplit; ++s) acc += to_f64(dpart[(int64_t)s * Mpad + row]);
    if (colexp != nullptr) acc = ldexp(acc, colexp[r] + colexp[c] - 12);
    if (row == col && d != nullptr) acc += d[row];
    A[(int64_t)row * M + col] = acc;
    if (row == 0) {
        double bb = 0.0;
        for (int s = 0; s < nsplit; ++s) bb += to_f64(bpart[(int64_t)s * Mpad + col]);
        b[col] = bb;
    }
}

// The mixed-precision Gram's assembly, per 32 x 32 block (bi >= bj) of the
// lower triangle of A: the float-pair partial tiles (TT x TT) of the splits (column-
// scaled by 2^(6 - E_m)) are read coalesced along their rows, summed in split
// order as an unevaluated float pair (exact two-sum, ~46 bits), converted to
// float64 once and unscaled by the exact power of two 2^(E_r + E_c - 12); the
// block is written to A and, through shared memory, transposed into the
// upper triangle (A is exactly symmetric). Diagonal blocks also sum b.
// d_m = sigma2 / lambda_m = exp(log sigma2 - sum_j log lambda^(j)_{m_j}) (Eq. 16,
// 20; with ARD, Eq. 17, each dimension has its own eigenvalues), clamped at
// 1e200; loglam[j * n + k] = log lambda_k of dimension j
__device__ __forceinline__ double noise_diag_entry(const GpShape& s, const double* __restrict__ loglam,
                                                   double log_sigma2, int m) {
    double ll = 0.0;
    for (int j = 0; j < s.p; ++j) ll += loglam[j * s.n + (m / s.stride[j]) % s.n];
    const double logd = log_sigma2 - ll;
    const double lclamp = 460.51701859880913680;  // log(1e200)
    return logd >= lclamp ? 1e200 : exp(logd);
}

// With loglam given, the diagonal of A gets d_m computed here (and stored in
// dout) instead of read from d; with L given, the lower triangle of A is also
// written there (the Cholesky's input), which saves a separate copy.
// PAIR: float64 partials of the CTA-pair kernel (256 x 256 tiles in the order
// of gp_pair_tile_offset), summed in split order in float64; otherwise
// float-pair partials (TT x TT, row-major) summed as float pairs.
template <bool PAIR>
__global__ void __launch_bounds__(1024) assemble_scaled_kernel(const void* __restrict__ Gpv,
                                                              const double* __restrict__ bpart,
                                                              const int* __restrict__ colexp, SyrkSplit spl,
                                                              int TT, int Mpad, int M, const double* __restrict__ d,
                                                              double* __restrict__ A, double* __restrict__ b,
                                                              GpShape sh, const double* __restrict__ loglam,
                                                              double log_sigma2, double* __restrict__ dout,
                                                              double* __restrict__ Lc) {
    constexpr int B = 32;  // TT: the Gram's tile (128, or 256 for the CTA-pair kernel)
    __shared__ double t[B][B + 1];
    __shared__ double sd[B];
    int bi, bj;
    tri_pair(blockIdx.x, &bi, &bj);
    const int r0 = bi * B, c0 = bj * B;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // one element per thread
    if (bi == bj) {
        // the block's diagonal entries of d, all by warp 0 (a float64
        // instruction costs its scheduler the same for one lane as for 32,
        // so one entry in each of 32 warps would cost 32 times as much)
        if (threadIdx.x < B) {
            const int r = r0 + threadIdx.x;
            double dr = 0.0;
            if (r < M) {
                if (loglam != nullptr) {
                    dr = noise_diag_entry(sh, loglam, log_sigma2, r);
                    dout[r] = dr;
                } else if (d != nullptr) {
                    dr = d[r];
                }
            }
            sd[threadIdx.x] = dr;
        }
        __syncthreads();
    }
    const int T = Mpad / TT;
    const int64_t sstride = (int64_t)(T * (T + 1) / 2) * TT * TT;
    auto add2 = [](float& hi, float& lo, float v) {  // hi + v = s + e exactly; lo collects e
        const float sum = __fadd_rn(hi, v);
        const float tt = __fsub_rn(sum, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, tt)), __fsub_rn(v, tt));
        hi = sum;
        lo = __fadd_rn(lo, e);
    };
    {
        const int r = r0 + ty, c = c0 + tx;
        double v = 0.0;
        if (r < M && c < M && c <= r) {
            const int I = r / TT, J = c / TT;
            const int pc = syrk_pair_class(I, J);
            const int nsplit = pc == 0 ? spl.n[0] : (pc == 1 ? spl.n[1] : spl.n[2]);  // this pair's splits
            double sum;
            if constexpr (PAIR) {
                const double* Gpart = reinterpret_cast<const double*>(Gpv);
                const int64_t off = (int64_t)(I * (I + 1) / 2 + J) * TT * TT + gp_pair_tile_offset(r % TT, c % TT);
                sum = 0.0;
                for (int sp = 0; sp < nsplit; ++sp) sum += Gpart[off + sp * sstride];
            } else {
                const float2* Gpart = reinterpret_cast<const float2*>(Gpv);
                const int64_t off = (int64_t)(I * (I + 1) / 2 + J) * TT * TT + (int64_t)(r % TT) * TT + (c % TT);
                float hi = 0.f, lo = 0.f;
                for (int sp = 0; sp < nsplit; ++sp) {
                    const float2 g = Gpart[off + sp * sstride];
                    add2(hi, lo, g.x);
                    lo = __fadd_rn(lo, g.y);
                }
                sum = (double)hi + (double)lo;
            }
            const int e = colexp[r] + colexp[c] - 12;  // |e| well inside float64's exponent range
            v = sum * __hiloint2double((e + 1023) << 20, 0);
            if (r == c) v += sd[ty];
            A[(int64_t)r * M + c] = v;
            if (Lc != nullptr) Lc[(int64_t)r * M + c] = v;
        }
        t[ty][tx] = v;
    }
    __syncthreads();
    {
        const int rr = ty;  // row of the transposed block (a column of the lower block)
        if (bi != bj) {
            const int row = c0 + rr, col = r0 + tx;
            if (row < M && col < M) A[(int64_t)row * M + col] = t[tx][rr];
        } else if (tx > rr && r0 + rr < M && c0 + tx < M) {
            A[(int64_t)(r0 + rr) * M + c0 + tx] = t[tx][rr];
        }
    }
    if (bpart != nullptr && bi == bj && threadIdx.x < B) {  // (the CTA-pair path forms b elsewhere)
        const int col = c0 + threadIdx.x;
        if (col < M) {
            double bb = 0.0;
            const int nsb = col / TT == 0 ? spl.n[0] : spl.n[1];  // splits of the pair (I, 0) that formed it
            for (int sp = 0; sp < nsb; ++sp) bb += bpart[(int64_t)sp * Mpad + col];
            b[col] = bb;
        }
    }
}

__global__ void noise_diag_kernel(GpShape s, const double* __restrict__ loglam, double log_sigma2,
                                  double* __restrict__ d) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= s.M) return;
    d[m] = noise_diag_entry(s, loglam, log_sigma2, m);
}

}  // namespace

void launch_assemble_f64(const double* Gpart, const double* bpart, int nsplit, int tile, int Mpad,
                         int M, const double* d, double* A, double* b, cudaStream_t stream) {
    dim3 grid((unsigned)((M + 255) / 256), (unsigned)M);
    assemble_kernel<double, double><<<grid, 256, 0, stream>>>(Gpart, bpart, nullptr, nullptr, nsplit, tile,
                                                      Mpad, M, d, A, b);
}

void launch_assemble_scaled(const float2* Gpart, const double* bpart, const int* colexp, const SyrkSplit& spl,
                            int tile, int Mpad, int M, const double* d, double* A, double* b,
                            cudaStream_t stream, const AssembleExtra* ex) {
    const int nb = (M + 31) / 32;
    GpShape sh{};
    const double* loglam = nullptr;
    double lsig = 0.0;
    double *dout = nullptr, *Lc = nullptr;
    if (ex != nullptr) {
        sh = *ex->shape;
        loglam = ex->loglam;
        lsig = log(ex->sigma2);
        dout = ex->dout;
        Lc = ex->L;
    }
    assemble_scaled_kernel<false><<<(unsigned)(nb * (nb + 1) / 2), 1024, 0, stream>>>(
        Gpart, bpart, colexp, spl, tile, Mpad, M, d, A, b, sh, loglam, lsig, dout, Lc);
}

void launch_assemble_pair(const double* Gpart, const double* bpart, const int* colexp, const SyrkSplit& spl,
                          int Mpad, int M, const double* d, double* A, double* b, cudaStream_t stream,
                          const AssembleExtra* ex) {
    const int nb = (M + 31) / 32;
    GpShape sh{};
    const double* loglam = nullptr;
    double lsig = 0.0;
    double *dout = nullptr, *Lc = nullptr;
    if (ex != nullptr) {
        sh = *ex->shape;
        loglam = ex->loglam;
        lsig = log(ex->sigma2);
        dout = ex->dout;
        Lc = ex->L;
    }
    assemble_scaled_kernel<true><<<(unsigned)(nb * (nb + 1) / 2), 1024, 0, stream>>>(
        Gpart, bpart, colexp, spl, 256, Mpad, M, d, A, b, sh, loglam, lsig, dout, Lc);
}

void launch_noise_diag(const GpShape& s, const double* loglam, double sigma2, double* d,
                       cudaStream_t stream) {
    noise_diag_kernel<<<(s.M + 255) / 256, 256, 0, stream>>>(s, loglam, log(sigma2), d);
}
