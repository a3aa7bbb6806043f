// Least-squares estimation of the APH coefficients (Sec. 2.2):
//   h = (Psi^H Psi)^{-1} Psi^H t,  Psi = basis matrix of Eq. 2 built from u.
//
// Real form.  With A = [Re Psi | Re t | Im Psi | Im t] (n x (2K + 2)), every
// quantity needed is a block of A^T A:
//   Re G_ab = <Re a, Re b> + <Im a, Im b>,   Im G_ab = <Re a, Im b> - <Im a, Re b>
//   Re g_a  = <Re a, Re t> + <Im a, Im t>,   Im g_a  = <Re a, Im t> - <Im a, Re t>
//   t^H t   = <Re t, Re t> + <Im t, Im t>
// (G = Psi^H Psi, g = Psi^H t).  The conjugate branch's basis is the conjugate
// of the main branch's (Eq. 2), so Re conj(z) = Re z and Im conj(z) = -Im z:
// every real column of A is +-1 times one of D = 2 B T + 3 distinct columns
// X (B = max(Bp, Bq)), or zero (Im of the constant column):
//   d = b T + k          Re psi_b(u_{n-k})    (b < B, k < T)
//   d = B T + b T + k    Im psi_b(u_{n-k})
//   d = 2 B T            1
//   d = 2 B T + 1, + 2   Re t, Im t
// and S = X^T X (D x D, D <= 99) holds all of A^T A up to signs.
//
// S is a contraction over the n rows, run on the tensor cores.  Every distinct
// column is one of 15 signals (Re / Im psi_b, Re / Im t, the constant) read at
// a tap, so an entry of S is a lagged correlation of two signals, less the
// products that fall off the end of the record; the tensor kernel computes the
// 15 x 14 x 8 lagged correlations (the basis recomputed from u, never stored
// in global memory), as a polyphase product whose operands hold each signal
// once per sample, split into a high and a low part (BF16 or TF32), X = hi +
// lo, with hi hi + hi lo + lo hi summed in FP32 in tensor memory.  Per-CTA
// partial sums are added in FP64 in a fixed order and S is filled from them
// and the last samples of the record.  The K x K system is then equilibrated
// and factored in FP64 (Cholesky), and refined against the FP32 residual
// t - Psi h computed by the filter and adjoint kernels.
#pragma once

#include "dpd_internal.h"

namespace dpd {

struct GramProblem {
    const float2 *u;   // basis input (n samples)
    const float2 *t;   // target (n samples) or null
    int64_t n;
};

constexpr int kGramS = 112;             // distinct columns, padded (D <= 99); row stride of S
constexpr int kGramRows = 128;          // rows of a partial (the MMA's M)
constexpr int kGramPartCols = 2 * kGramS;   // a partial: P in columns [0, 112), Q in [112, 224)

__host__ __device__ constexpr int gram_distinct(int B, int T) { return 2 * B * T + 3; }

// Distinct column and sign of the real and imaginary parts of complex column j
// of Psi (stacking order of Sec. 2.2); sign 0 marks a zero column.
struct ColRef {
    int d, sign;
};
__host__ __device__ inline void psi_column_refs(int j, int K, int Bp, int B, int T, ColRef &re, ColRef &im)
{
    if (j == K - 1) {   // the constant column (LO leakage term c)
        re = ColRef{2 * B * T, 1};
        im = ColRef{0, 0};
        return;
    }
    const bool conj = j >= Bp * T;
    const int jj = conj ? j - Bp * T : j;
    const int b = jj / T, k = jj % T;
    re = ColRef{b * T + k, 1};
    im = ColRef{B * T + b * T + k, conj ? -1 : 1};
}

struct GramArgs {
    const GramProblem *probs;   // device array of nprob problems, or null: the one problem below
    GramProblem one;
    int nprob;
    int cpp;               // CTAs per problem (row chunks)
    int Bp, Bq, T, K;
    float *partials;       // FP32 kernel: [nprob * cpp][kGramRows][kGramPartCols] floats;
                           // tensor kernel: [nprob * cpp][kLagEntries] float pairs
    int *status;
    // Basis of the psi columns: per problem a kMaxB x kMaxB matrix U (row-major,
    // U[a][b] multiplies |u|^{2a} u in basis function b, upper triangular), or
    // null for the monomials |u|^{2b} u themselves.
    const float *ubasis;
};
constexpr int kUSize = kMaxB * kMaxB;

// Precision of the Gram contraction.
enum : int { kPrecFP32 = 0, kPrecTF32x3 = 1, kPrecBF16x3 = 2 };

cudaError_t launch_gram(int precision, const GramArgs &a, cudaStream_t s);
// S[p][i][c] (i < D, c < 2 kGramS) = sum over the problem's CTAs of the partial P and Q
// blocks, in FP64 and a fixed order (S = P + Q + Q^T is formed by the assembly).
cudaError_t launch_gram_reduce(const float *partials, int nprob, int cpp, int D, double *S, cudaStream_t s);
// Tensor-core precisions: each CTA's partial is kLagEntries lag sums C[a][b][d]
// (a < 15, b < 14, d < kMaxT), each an FP32 pair (sum, rounding error); this sums them per
// problem into C (FP64, fixed order).
// G, g and t^H t are assembled from C directly (the entries of S on the fly), into G / g
// / tt at K x K, K, 1 per problem; probs may be null for one problem passed as `one`.
constexpr int kLagEntries = 15 * 14 * kMaxT;
cudaError_t launch_gram_lag_finish(const float *partials, const GramProblem *probs, GramProblem one,
                                   const float *ubasis, int nprob, int cpp, int K, int Bp, int B, int T, double *C,
                                   double2 *G, double2 *g, double *tt, cudaStream_t s);
// G (K x K, row-major), g (K) and t^H t per problem from S.
cudaError_t launch_gram_assemble(const double *S, int nprob, int K, int Bp, int B, int T, double2 *G, double2 *g,
                                 double *tt, cudaStream_t s);
// Power sums of r = |u|^2 per problem: mom[p][k - 1] = sum_n r_n^k, k = 1 .. 2 kMaxB - 1,
// in a fixed order: per thread as exact FP32 two-sum pairs, then FP64 (part: nprob *
// kMomBlocks * kMomK doubles of scratch).
constexpr int kMomK = 2 * kMaxB - 1;
constexpr int kMomBlocks = 64;
cudaError_t launch_moments(const GramProblem *probs, int nprob, double *part, double *mom, cudaStream_t s);
// Coefficient vectors between the monomial basis and the basis U (both
// branches, every tap; the constant unchanged), per problem:
//   to_monomial: out = W in       (h = W h_U)
//   otherwise:   out = W^T in     (g_U = W^T g for right-hand sides)
cudaError_t launch_basis_transform(const double2 *in, double2 *out, const double *U, int nprob, int K, int Bp,
                                   int Bq, int T, int to_monomial, cudaStream_t s);
// CTAs per row chunk the launch wants for nprob problems of up to n rows.
int gram_ctas_per_problem(int precision, int sm_count, int nprob, int64_t n);
// Equilibrated Cholesky factorisation of every G: D G D = L L^H, D = diag(G)^{-1/2}.
// L (lower, row-major K x K) and d (K) per problem; info[p] = 0 or the failing pivot + 1.
cudaError_t launch_chol(const double2 *G, int nprob, int K, double2 *L, double *d, int *info, cudaStream_t s);
// x = G^{-1} rhs using the factorisation; if accumulate, h += x instead of h = x.
cudaError_t launch_chol_solve(const double2 *L, const double *d, const int *info, const double2 *rhs, int nprob,
                              int K, double2 *h, int accumulate, cudaStream_t s);
// Single problem: Linv = L^{-1} (lower, row-major K x K) of the factorisation,
// then x = G^{-1} rhs = D Linv^H Linv D rhs as two parallel matrix-vector
// products (tmp: K values of scratch); both skip a failed factorisation.
cudaError_t launch_chol_invert(const double2 *L, const int *info, int K, double2 *Linv, cudaStream_t s);
cudaError_t launch_solve_inverse(const double2 *Linv, const double *d, const int *info, const double2 *rhs, int K,
                                 double2 *tmp, double2 *h, int accumulate, cudaStream_t s);
// Complex64 copy of the FP64 coefficients.
cudaError_t launch_h_to_f32(const double2 *h, int n, float2 *out, cudaStream_t s);
// e = t - y (n samples).
cudaError_t launch_residual(const float2 *t, const float2 *y, int64_t n, float2 *e, cudaStream_t s);
// e = t - y together with out[0] = sum |e|^2, out[1] = sum |t|^2 in FP64
// (part: 2 * 1024 doubles of scratch).
cudaError_t launch_residual_norm(const float2 *t, const float2 *y, int64_t n, float2 *e, double *part, double *out,
                                 cudaStream_t s);
// Like launch_adj_finalize, summed to FP64.
cudaError_t launch_adj_finalize64(const float2 *partials, int rows, int K, double2 *out, cudaStream_t s);
// The same for `count` problems, each with `rows` rows (outputs K apart).
cudaError_t launch_adj_finalize64_many(const float2 *partials, int rows, int K, int count, double2 *out,
                                       cudaStream_t s);

}  // namespace dpd
