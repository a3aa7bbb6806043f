// Least-squares estimation of the APH coefficients (Sec. 2.2):
//   h = (Psi^H Psi)^{-1} Psi^H t,  Psi = basis matrix of Eq. 2 built from u.
//
// Real form.  With A = [Re Psi | Re t | Im Psi | Im t] (n x C, C = 2K + 2),
// every quantity needed is a block of S = A^T A:
//   Re G_ab = S[a][b] + S[K+1+a][K+1+b],   Im G_ab = S[a][K+1+b] - S[K+1+a][b]
//   Re g_a  = S[a][K] + S[K+1+a][2K+1],    Im g_a  = S[a][2K+1] - S[K+1+a][K]
//   t^H t   = S[K][K] + S[2K+1][2K+1]
// (G = Psi^H Psi, g = Psi^H t).  S is a dense contraction over the n rows, so
// it runs on the tensor cores: each CTA generates R rows of A at a time (the
// basis, recomputed from u, never stored in global memory) into shared memory
// as operand rows (one per column of A, K-major, 128-byte swizzle), split into
// a high and a low part (BF16 or TF32), and issues
//   S += hi^T hi + hi^T lo + lo^T hi
// as tcgen05 MMAs accumulating in tensor memory (FP32), in two 128-row tiles
// that cover the upper triangle of S only.  Each CTA writes its partial S;
// the partials are summed in FP64 in a fixed order.  The K x K system is then
// equilibrated and factored in FP64 (Cholesky), and refined against the FP32
// residual t - Psi h computed by the filter and adjoint kernels.
#pragma once

#include "dpd_internal.h"

namespace dpd {

struct GramProblem {
    const float2 *u;   // basis input (n samples)
    const float2 *t;   // target (n samples) or null
    int64_t n;
};

constexpr int kGramRows = 256;   // real-form columns, padded (two 128-row MMA tiles)
constexpr int kGramCols = 208;   // widest accumulator tile (N <= 208 covers C <= 196)

struct GramArgs {
    const GramProblem *probs;
    int nprob;
    int cpp;               // CTAs per problem (row chunks)
    int Bp, Bq, T, K;
    float *partials;       // [nprob * cpp][kGramRows][kGramCols]
    int *status;
};

// Precision of the Gram contraction.
enum : int { kPrecFP32 = 0, kPrecTF32x3 = 1, kPrecBF16x3 = 2 };

cudaError_t launch_gram(int precision, const GramArgs &a, cudaStream_t s);
// S[p][i][j] (i <= j < 2K+2) = sum over the problem's CTAs of the partials, in FP64.
cudaError_t launch_gram_reduce(const float *partials, int nprob, int cpp, int K, double *S, cudaStream_t s);
// G (K x K, row-major), g (K) and t^H t per problem from S.
cudaError_t launch_gram_assemble(const double *S, int nprob, int K, double2 *G, double2 *g, double *tt,
                                 cudaStream_t s);
// Equilibrated Cholesky factorisation of every G: D G D = L L^H, D = diag(G)^{-1/2}.
// L (lower, row-major K x K) and d (K) per problem; info[p] = 0 or the failing pivot + 1.
cudaError_t launch_chol(const double2 *G, int nprob, int K, double2 *L, double *d, int *info, cudaStream_t s);
// x = G^{-1} rhs using the factorisation; if accumulate, h += x instead of h = x.
cudaError_t launch_chol_solve(const double2 *L, const double *d, const int *info, const double2 *rhs, int nprob,
                              int K, double2 *h, int accumulate, cudaStream_t s);
// Complex64 copy of the FP64 coefficients.
cudaError_t launch_h_to_f32(const double2 *h, int n, float2 *out, cudaStream_t s);
// e = t - y (n samples).
cudaError_t launch_residual(const float2 *t, const float2 *y, int64_t n, float2 *e, cudaStream_t s);
// out[0] = sum |e|^2, out[1] = sum |t|^2 in FP64 (part: 2 * 1024 doubles of scratch).
cudaError_t launch_sqnorm2(const float2 *e, const float2 *t, int64_t n, double *part, double *out, cudaStream_t s);
// Like launch_adj_finalize, summed to FP64.
cudaError_t launch_adj_finalize64(const float2 *partials, int rows, int K, double2 *out, cudaStream_t s);

}  // namespace dpd
