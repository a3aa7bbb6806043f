// libdpd C ABI, least-squares part: dpd_gram, dpd_estimate and
// dpd_estimate_batched (contracts in include/dpd.h, method in dpd_gram.cuh).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <system_error>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dpd.h"
#include "dpd_batched.cuh"
#include "dpd_gram.cuh"
#include "dpd_handle.h"

namespace {

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

template <class T>
bool grow(T *&p, size_t have, size_t need)
{
    if (need <= have && p) return true;
    cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T)) == cudaSuccess;
}

// Make sure the workspace holds nprob problems with cpp Gram CTAs each and
// nsamp samples of refinement buffers.  Synchronises the device when it grows.
dpd_status reserve(dpd_handle h, int nprob, int cpp, int64_t nsamp)
{
    EstimateWorkspace &w = h->est;
    const int K = h->K;
    bool ok = true;
    if (nprob > w.nprob || cpp * nprob > w.cpp * w.nprob) {
        cudaDeviceSynchronize();
        const size_t np = (size_t)nprob, parts = (size_t)nprob * cpp;
        ok = ok && grow(reinterpret_cast<dpd::GramProblem *&>(w.probs), 0, np);
        ok = ok && grow(w.partials, 0, parts * dpd::kGramRows * dpd::kGramPartCols);
        ok = ok && grow(w.S, 0, np * dpd::kGramS * dpd::kGramPartCols) && grow(w.Clag, 0, np * dpd::kLagEntries);
        ok = ok && grow(w.G, 0, np * K * K) && grow(w.L, 0, np * K * K);
        ok = ok && grow(w.g, 0, np * K) && grow(w.h64, 0, np * K) && grow(w.delta, 0, np * K);
        ok = ok && grow(w.d, 0, np * K) && grow(w.tt, 0, np) && grow(w.info, 0, np);
        ok = ok && grow(w.hf, 0, (size_t)K) && grow(w.tab, 0, (size_t)dpd::wl_table_floats(h->B, h->T));
        // partial pairs, the two results, the completion counter (zero)
        ok = ok && grow(w.norm_part, 0, (size_t)2 * dpd::kFwdNormSlots + 3) &&
             cudaMemset(w.norm_part, 0, ((size_t)2 * dpd::kFwdNormSlots + 3) * sizeof(double)) == cudaSuccess;
        ok = ok && grow(w.ubasis, 0, np * dpd::kUSize) && grow(w.ubasis64, 0, np * dpd::kUSize);
        ok = ok && grow(w.mom, 0, np * dpd::kMomK) && grow(w.mom_part, 0, np * dpd::kMomBlocks * dpd::kMomK);
        ok = ok && grow(w.hm64, 0, np * K);
        ok = ok && grow(w.Linv, 0, (size_t)K * K) && grow(w.tmpv, 0, (size_t)K);
        if (!ok) return DPD_ERR_ALLOC;
        w.nprob = nprob;
        w.cpp = cpp;
    }
    if (w.hK != K || !w.h_G) {
        cudaFreeHost(w.h_G);
        cudaFreeHost(w.h_Linv);
        cudaFreeHost(w.h_info);
        cudaFreeHost(w.h_norm);
        w.h_G = nullptr;
        w.h_Linv = nullptr;
        w.h_info = nullptr;
        w.h_norm = nullptr;
        w.hK = 0;
        if (cudaMallocHost(&w.h_G, sizeof(double2) * K * K) != cudaSuccess ||
            cudaMallocHost(&w.h_Linv, sizeof(double2) * K * K) != cudaSuccess ||
            cudaMallocHost(&w.h_info, sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&w.h_norm, 2 * sizeof(double)) != cudaSuccess)
            return DPD_ERR_ALLOC;
        w.hK = K;
    }
    if (!w.ev_L && cudaEventCreateWithFlags(&w.ev_L, cudaEventDisableTiming) != cudaSuccess) return DPD_ERR_CUDA;
    if (!w.ev_G && cudaEventCreateWithFlags(&w.ev_G, cudaEventDisableTiming) != cudaSuccess) return DPD_ERR_CUDA;
    if (nsamp > w.nsamp) {
        cudaDeviceSynchronize();
        ok = grow(w.y, 0, (size_t)nsamp) && grow(w.e, 0, (size_t)nsamp);
        if (!ok) return DPD_ERR_ALLOC;
        w.nsamp = nsamp;
    }
    return DPD_OK;
}

bool valid_precision(int p) { return p == DPD_PREC_FP32 || p == DPD_PREC_TF32X3 || p == DPD_PREC_BF16X3; }

bool ortho(dpd_handle h) { return h->est_basis == DPD_BASIS_ORTHOGONAL; }

// Basis of statistically orthogonal polynomials (Sec. 2.1) for every problem
// in w.probs: with mu_k = sum_n r_n^k (r = |u|^2), the moment matrix
// M[a][b] = mu_{a+b+1} / n is the Gram matrix of the monomials |u|^{2a} u;
// M = L L^T (FP64 Cholesky on the host) and U = L^{-T} make
// sum_a U[a][b] |u|^{2a} u orthonormal.  U is rounded to FP32 for the Gram
// kernels and the same values are kept in FP64 for the coefficient
// transforms.  A problem whose moment matrix is not positive definite keeps
// the monomials (U = I).
dpd_status compute_basis(dpd_handle h, const std::vector<int64_t> &n, cudaStream_t s)
{
    EstimateWorkspace &w = h->est;
    const int nprob = (int)n.size(), B = h->B;
    if (dpd::launch_moments(static_cast<const dpd::GramProblem *>(w.probs), nprob, w.mom_part, w.mom, s) !=
        cudaSuccess)
        return DPD_ERR_CUDA;
    std::vector<double> mom((size_t)nprob * dpd::kMomK);
    if (cudaMemcpyAsync(mom.data(), w.mom, sizeof(double) * mom.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DPD_ERR_CUDA;
    std::vector<float> uf((size_t)nprob * dpd::kUSize, 0.f);
    std::vector<double> ud((size_t)nprob * dpd::kUSize, 0.0);
    for (int p = 0; p < nprob; ++p) {
        double M[dpd::kMaxB][dpd::kMaxB], L[dpd::kMaxB][dpd::kMaxB] = {}, U[dpd::kMaxB][dpd::kMaxB] = {};
        for (int a = 0; a < B; ++a)
            for (int b = 0; b < B; ++b) M[a][b] = mom[(size_t)p * dpd::kMomK + a + b] / (double)n[p];
        bool spd = true;
        for (int i = 0; i < B && spd; ++i)
            for (int j = 0; j <= i; ++j) {
                double v = M[i][j];
                for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
                if (i == j) {
                    if (!(v > 0.0) || !std::isfinite(v)) {
                        spd = false;
                        break;
                    }
                    L[i][i] = std::sqrt(v);
                } else {
                    L[i][j] = v / L[j][j];
                }
            }
        if (spd) {   // U = L^{-T}: L^T U = I, solved column by column (back substitution)
            for (int b = 0; b < B; ++b)
                for (int a = B - 1; a >= 0; --a) {
                    double v = a == b ? 1.0 : 0.0;
                    for (int k = a + 1; k < B; ++k) v -= L[k][a] * U[k][b];
                    U[a][b] = v / L[a][a];
                }
        }
        for (int a = 0; a < dpd::kMaxB; ++a)
            for (int b = 0; b < dpd::kMaxB; ++b) {
                const double v = (a < B && b < B) ? (spd ? U[a][b] : (a == b ? 1.0 : 0.0)) : 0.0;
                uf[(size_t)p * dpd::kUSize + a * dpd::kMaxB + b] = (float)v;
                ud[(size_t)p * dpd::kUSize + a * dpd::kMaxB + b] = (double)(float)v;
            }
    }
    if (cudaMemcpyAsync(w.ubasis, uf.data(), sizeof(float) * uf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.ubasis64, ud.data(), sizeof(double) * ud.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DPD_ERR_CUDA;
    return DPD_OK;
}

// FP64 coefficients of problems [p0, p0 + np) in the monomial basis (w.hm64).
const double2 *monomial_h(dpd_handle h, int p0, int np, cudaStream_t s, dpd_status &st)
{
    EstimateWorkspace &w = h->est;
    const size_t off = (size_t)p0 * h->K;
    st = DPD_OK;
    if (!ortho(h)) return w.h64 + off;
    if (dpd::launch_basis_transform(w.h64 + off, w.hm64 + off, w.ubasis64 + (size_t)p0 * dpd::kUSize, np, h->K,
                                    h->Bp, h->Bq, h->T, 1, s) != cudaSuccess)
        st = DPD_ERR_CUDA;
    return w.hm64 + off;
}

int gram_cpp(dpd_handle h, int nprob, int64_t n, int precision)
{
    return dpd::gram_ctas_per_problem(precision, h->sm_count, nprob, n);
}

// Gram (+ reduction + assembly) of nprob problems described in w.probs, or of
// the single problem *one (passed by value to the kernels, no copy); G and g
// go to G_out / g_out when given, else to the workspace.  The basis is the
// handle's estimate basis, or the monomials of Eq. 2 with `monomial`.
dpd_status run_gram(dpd_handle h, int nprob, int cpp, int precision, cudaStream_t s,
                    const dpd::GramProblem *one = nullptr, double2 *G_out = nullptr, double2 *g_out = nullptr,
                    bool monomial = false)
{
    EstimateWorkspace &w = h->est;
    dpd::GramArgs a;
    a.probs = one ? nullptr : static_cast<const dpd::GramProblem *>(w.probs);
    a.one = one ? *one : dpd::GramProblem{nullptr, nullptr, 0};
    a.nprob = nprob;
    a.cpp = cpp;
    a.Bp = h->Bp;
    a.Bq = h->Bq;
    a.T = h->T;
    a.K = h->K;
    a.partials = w.partials;
    a.status = h->d_status;
    a.ubasis = ortho(h) && !monomial ? w.ubasis : nullptr;
    double2 *G = G_out ? G_out : w.G, *g = G_out ? g_out : w.g;
    if (dpd::launch_gram(precision, a, s) != cudaSuccess) return DPD_ERR_CUDA;
    const int D = dpd::gram_distinct(h->B, h->T);
    if (precision == dpd::kPrecFP32) {
        if (dpd::launch_gram_reduce(w.partials, nprob, cpp, D, w.S, s) != cudaSuccess ||
            dpd::launch_gram_assemble(w.S, nprob, h->K, h->Bp, h->B, h->T, G, g, w.tt, s) != cudaSuccess)
            return DPD_ERR_CUDA;
    } else if (dpd::launch_gram_lag_finish(w.partials, a.probs, a.one, a.ubasis, nprob, cpp, h->K, h->Bp, h->B, h->T,
                                           w.Clag, G, g, w.tt, s) != cudaSuccess) {
        return DPD_ERR_CUDA;
    }
    return DPD_OK;
}

// e = t - Psi(u) h for the current FP64 coefficients of problem p (FP32 filter);
// with `norms`, only ||e||^2 and ||t||^2 into w.norm_part + 2 kFwdNormSlots
// (e itself is not written).
dpd_status residual_of(dpd_handle h, int p, const float2 *u, const float2 *t, int64_t n, cudaStream_t s,
                       bool norms = false)
{
    EstimateWorkspace &w = h->est;
    dpd_status st = DPD_OK;
    const double2 *hm = monomial_h(h, p, 1, s, st);
    if (st != DPD_OK) return st;
    if (dpd::launch_wl_table_f64(hm, h->Bp, h->Bq, h->T, w.tab, s) != cudaSuccess) return DPD_ERR_CUDA;
    dpd::FwdArgs fa;
    fa.x = u;
    fa.y = w.y;
    fa.n = n;
    fa.tab = w.tab;
    fa.status = h->d_status;
    fa.vec_store = 1;
    fa.host_tab = nullptr;
    // Coefficients live on the device (shared-memory table): 6 samples per
    // thread, 16 warps in two groups of 8, 4 stages (measured best for these
    // shapes on GB300: 31.6 us per 2^22 samples at P = Q = 11, M = 7, against
    // about 42 at the single-stream default of 8 samples per thread).
    dpd::FwdLaunch L;
    L.mode = dpd::kModePackedFma;
    L.V = 6;
    L.warps = 16;
    L.group = 8;
    L.stages = 4;
    const bool aligned16 = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(t)) & 15u) == 0;
    if (aligned16) {
        // The filter writes e = t - Psi(u) h itself (no separate residual
        // pass), or only sums |e|^2 and |t|^2.
        L.mode = dpd::kModePackedFma | dpd::kModeSubtract | (norms ? dpd::kModeNorms : 0);
        fa.y = w.e;
        fa.sub = t;
        fa.norms = w.norm_part;
        return dpd::launch_fwd_any(h->B, h->T, fa, L, h->sm_count, s) == cudaSuccess ? DPD_OK : DPD_ERR_CUDA;
    }
    if ((reinterpret_cast<uintptr_t>(u) & 15u) != 0) {
        L.use_tma = 0;
        L.V = 4;
    }
    if (dpd::launch_fwd_any(h->B, h->T, fa, L, h->sm_count, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (norms)
        return dpd::launch_residual_norm(t, w.y, n, nullptr, w.norm_part, w.norm_part + 2 * dpd::kFwdNormSlots, s) ==
                       cudaSuccess
                   ? DPD_OK
                   : DPD_ERR_CUDA;
    if (dpd::launch_residual(t, w.y, n, w.e, s) != cudaSuccess) return DPD_ERR_CUDA;
    return DPD_OK;
}

// One refinement step of problem p:  h64[p] += G^{-1} Psi^H (t - Psi h).
dpd_status refine_once(dpd_handle h, int p, const float2 *u, const float2 *t, int64_t n, cudaStream_t s)
{
    EstimateWorkspace &w = h->est;
    const int K = h->K;
    dpd_status st = residual_of(h, p, u, t, n, s);
    if (st != DPD_OK) return st;
    dpd::AdjArgs aa;
    aa.x = u;
    aa.gy = w.e;
    aa.n = n;
    aa.gx = nullptr;
    aa.partials = h->d_partials;
    aa.adj_tab = h->d_adj_tab;
    aa.status = h->d_status;
    dpd::AdjLaunch al = h->adj;
    const int64_t need = (n + 1023) / 1024;
    if (al.gh_blocks > need) al.gh_blocks = (int)need;
    if (al.gh_blocks > h->rows_max) al.gh_blocks = h->rows_max;
    if (al.gh_blocks < 1) al.gh_blocks = 1;
    if (dpd::launch_adj_any(h->B, aa, al, h->T, h->Bp, h->Bq, K, h->sm_count, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (dpd::launch_adj_finalize64(h->d_partials, al.gh_blocks, K, w.delta, s) != cudaSuccess) return DPD_ERR_CUDA;
    const double2 *rhs = w.delta;   // Psi^H (t - Psi h) in the monomial basis
    if (ortho(h)) {                 // W^T of it, the right-hand side in the working basis
        if (dpd::launch_basis_transform(w.delta, w.hm64 + (size_t)p * K, w.ubasis64 + (size_t)p * dpd::kUSize, 1,
                                        K, h->Bp, h->Bq, h->T, 0, s) != cudaSuccess)
            return DPD_ERR_CUDA;
        rhs = w.hm64 + (size_t)p * K;
    }
    if (w.use_inverse && p == 0) {
        if (dpd::launch_solve_inverse(w.Linv, w.d, w.info, rhs, K, w.tmpv, w.h64, 1, s) != cudaSuccess)
            return DPD_ERR_CUDA;
    } else if (dpd::launch_chol_solve(w.L + (size_t)p * K * K, w.d + (size_t)p * K, w.info + p, rhs, 1, K,
                                      w.h64 + (size_t)p * K, 1, s) != cudaSuccess) {
        return DPD_ERR_CUDA;
    }
    return DPD_OK;
}

// Refinement of all problems of a batch together, each step one launch per
// kernel: the per-problem forward tables, the batched forward filter (6
// samples per thread, 16 warps in groups of 8, 4 stages) into the residual
// buffers, e = t - Psi h in place, the coefficient gradients of all problems
// (one CTA per problem and tap group), their FP64 sums, the basis transform
// (orthogonal basis) and the batched Cholesky solve.  Needs 16-byte aligned
// inputs u (the bulk-copy pipelines); the caller checks that.
dpd_status refine_batched(dpd_handle h, const std::vector<dpd::GramProblem> &probs, int64_t nmax, int iters,
                          cudaStream_t s)
{
    EstimateWorkspace &w = h->est;
    const int K = h->K, count = (int)probs.size();
    const int64_t stride = (nmax + 1) & ~int64_t(1);   // keeps every e_p 16-byte aligned
    const int tfl = dpd::wl_table_floats(h->B, h->T), tstride = (tfl + 3) & ~3;
    constexpr int V = 6, warps = 16, group = 8, stages = 4;
    const int S = warps * 32 * V;
    std::vector<dpd::BatchStream> st((size_t)count);
    std::vector<dpd::BatchItem> items;
    std::vector<dpd::AdjArgs> adj((size_t)count);
    for (int p = 0; p < count; ++p) {
        float2 *ep = w.e + (size_t)p * stride;
        st[p] = {probs[p].u, ep, probs[p].n, h->B, h->T, p * tstride, tstride * 4, probs[p].t};   // e = t - Psi h
        for (int64_t t = 0; t * S < probs[p].n; ++t) items.push_back({p, (int)t});
        dpd::AdjArgs &a = adj[p];
        a.x = probs[p].u;
        a.gy = ep;
        a.n = probs[p].n;
        a.gx = nullptr;
        a.adj_tab = nullptr;
        a.host_adj_tab = nullptr;
        a.status = h->d_status;
    }
    if ((size_t)count > w.bprob_cap) {
        cudaDeviceSynchronize();
        cudaFree(w.bstreams);
        cudaFree(w.badj);
        cudaFree(w.bpart);
        cudaFree(w.tabb);
        w.bstreams = w.badj = nullptr;
        w.bpart = nullptr;
        w.tabb = nullptr;
        w.bprob_cap = 0;
        if (cudaMalloc(&w.bstreams, sizeof(dpd::BatchStream) * count) != cudaSuccess ||
            cudaMalloc(&w.badj, sizeof(dpd::AdjArgs) * count) != cudaSuccess ||
            cudaMalloc(&w.bpart, sizeof(float2) * (size_t)count * K) != cudaSuccess ||
            cudaMalloc(&w.tabb, sizeof(float) * (size_t)count * tstride) != cudaSuccess)
            return DPD_ERR_ALLOC;
        w.bprob_cap = (size_t)count;
    }
    if (items.size() > w.bitems_cap) {
        cudaDeviceSynchronize();
        cudaFree(w.bitems);
        w.bitems = nullptr;
        w.bitems_cap = 0;
        if (cudaMalloc(&w.bitems, sizeof(dpd::BatchItem) * items.size()) != cudaSuccess) return DPD_ERR_ALLOC;
        w.bitems_cap = items.size();
    }
    for (int p = 0; p < count; ++p) adj[p].partials = w.bpart + (size_t)p * K;   // one row per problem
    // Stream-ordered uploads from pageable memory: the runtime stages the host
    // data before each call returns (no device synchronisation), so the vectors
    // may go out of scope and the host goes on enqueuing the launches.
    if (cudaMemcpyAsync(w.bstreams, st.data(), sizeof(dpd::BatchStream) * count, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.bitems, items.data(), sizeof(dpd::BatchItem) * items.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.badj, adj.data(), sizeof(dpd::AdjArgs) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    dpd::BatchArgs ba;
    ba.streams = static_cast<const dpd::BatchStream *>(w.bstreams);
    ba.items = static_cast<const dpd::BatchItem *>(w.bitems);
    ba.nitems = (int)items.size();
    ba.nstreams = count;
    ba.tabs = w.tabb;
    ba.tab_floats = (int64_t)count * tstride;
    ba.status = h->d_status;
    ba.gw = group;
    const bool small = h->B <= 5 && h->T <= 7;
    dpd_status stt = DPD_OK;
    for (int it = 0; it < iters; ++it) {
        const double2 *hm = monomial_h(h, 0, count, s, stt);
        if (stt != DPD_OK) return stt;
        if (dpd::launch_wl_table_f64_many(hm, count, K, h->Bp, h->Bq, h->T, w.tabb, tstride, s) != cudaSuccess)
            return DPD_ERR_CUDA;
        const cudaError_t fe = small ? dpd::launch_batched_57(ba, V, warps, stages, 0, h->sm_count, s)
                                     : dpd::launch_batched_68(ba, V, warps, stages, 0, h->sm_count, s);
        if (fe != cudaSuccess) return DPD_ERR_CUDA;   // the filter wrote e_p = t_p - Psi h_p
        if (dpd::launch_adj_gh_many_any(h->B, static_cast<const dpd::AdjArgs *>(w.badj), count, 1, h->adj.tap_group,
                                        h->T, h->Bp, h->Bq, K, s) != cudaSuccess)
            return DPD_ERR_CUDA;
        if (dpd::launch_adj_finalize64_many(w.bpart, 1, K, count, w.delta, s) != cudaSuccess) return DPD_ERR_CUDA;
        const double2 *rhs = w.delta;   // Psi^H (t - Psi h) in the monomial basis
        if (ortho(h)) {                 // W^T of it, the right-hand sides in the working basis
            if (dpd::launch_basis_transform(w.delta, w.hm64, w.ubasis64, count, K, h->Bp, h->Bq, h->T, 0, s) !=
                cudaSuccess)
                return DPD_ERR_CUDA;
            rhs = w.hm64;
        }
        if (dpd::launch_chol_solve(w.L, w.d, w.info, rhs, count, K, w.h64, 1, s) != cudaSuccess) return DPD_ERR_CUDA;
    }
    return DPD_OK;
}

// Condition number of A = D G D = L L^H (the equilibrated Gram matrix, D =
// diag(G)^{-1/2}) in the 2-norm: the largest eigenvalue of A (products with A
// itself, formed from G) times the largest eigenvalue of A^{-1} = L^{-H} L^{-1}
// (products with the explicit inverse of L that the solves use), FP64 on the
// host.  Complex vectors and matrices are kept as separate real and imaginary
// arrays, padded to an even length N with zeros, and processed two elements
// at a time with GCC vector types (portable across x86-64 and AArch64): every
// inner product is split over several vector partial sums, so no loop is one
// long chain of dependent additions.
namespace cond {

typedef double v2d __attribute__((vector_size(16)));

inline v2d ld2(const double *p) { return *reinterpret_cast<const v2d *>(p); }   // 16-byte aligned
inline void st2(double *p, v2d v) { *reinterpret_cast<v2d *>(p) = v; }
inline double hsum(v2d v) { return v[0] + v[1]; }

// Padded split storage: rows of N (even) doubles; the heap blocks of
// std::vector are 16-byte aligned (the allocator's fundamental alignment on
// x86-64 and AArch64), so every row starts on a 16-byte boundary.
struct Split {
    int N = 0;
    std::vector<double> re, im;
    Split(int rows, int n) : N(n), re((size_t)rows * n, 0.0), im((size_t)rows * n, 0.0) {}
    double *r(int row) { return re.data() + (size_t)row * N; }
    double *i(int row) { return im.data() + (size_t)row * N; }
    const double *r(int row) const { return re.data() + (size_t)row * N; }
    const double *i(int row) const { return im.data() + (size_t)row * N; }
};

// y = M x for the first `rows` rows of M (row-major, padded width N); with
// `lower`, row i reads columns < i + 1 rounded up to the block (M is zero above
// its diagonal).  Four rows at a time, so every x element is loaded once per
// four rows.
void matvec(const Split &M, int rows, bool lower, const double *xr, const double *xi, double *yr, double *yi)
{
    const int N = M.N;
    int i = 0;
    for (; i + 4 <= rows; i += 4) {
        const int kend = lower ? std::min(N, (i + 4 + 1) & ~1) : N;
        v2d sr[4] = {}, si[4] = {};
        for (int k = 0; k < kend; k += 2) {
            const v2d a = ld2(xr + k), b = ld2(xi + k);
            for (int q = 0; q < 4; ++q) {
                const v2d mr = ld2(M.r(i + q) + k), mi = ld2(M.i(i + q) + k);
                sr[q] += mr * a - mi * b;
                si[q] += mr * b + mi * a;
            }
        }
        for (int q = 0; q < 4; ++q) {
            yr[i + q] = hsum(sr[q]);
            yi[i + q] = hsum(si[q]);
        }
    }
    for (; i < rows; ++i) {
        const int kend = lower ? std::min(N, (i + 1 + 1) & ~1) : N;
        v2d sr = {0, 0}, si = {0, 0};
        for (int k = 0; k < kend; k += 2) {
            const v2d a = ld2(xr + k), b = ld2(xi + k), mr = ld2(M.r(i) + k), mi = ld2(M.i(i) + k);
            sr += mr * a - mi * b;
            si += mr * b + mi * a;
        }
        yr[i] = hsum(sr);
        yi[i] = hsum(si);
    }
}

// y = M^H z for a lower-triangular M (row-major, padded width N): row by row,
// y[0 .. i] += conj(M_i,0..i) z_i (independent over the columns).
void matvec_h_lower(const Split &M, int rows, const double *zr, const double *zi, double *yr, double *yi)
{
    const int N = M.N;
    for (int k = 0; k < N; k += 2) {
        st2(yr + k, v2d{0, 0});
        st2(yi + k, v2d{0, 0});
    }
    for (int i = 0; i < rows; ++i) {
        const v2d a = v2d{zr[i], zr[i]}, b = v2d{zi[i], zi[i]};
        const int kend = std::min(N, (i + 1 + 1) & ~1);
        for (int k = 0; k < kend; k += 2) {
            const v2d mr = ld2(M.r(i) + k), mi = ld2(M.i(i) + k);
            st2(yr + k, ld2(yr + k) + mr * a + mi * b);
            st2(yi + k, ld2(yi + k) + mr * b - mi * a);
        }
    }
}

double2 dotc(int N, const double *a_r, const double *a_i, const double *b_r, const double *b_i)   // a^H b
{
    v2d sr[2] = {}, si[2] = {};
    int k = 0;
    for (; k + 4 <= N; k += 4)
        for (int h = 0; h < 2; ++h) {
            const v2d ar = ld2(a_r + k + 2 * h), ai = ld2(a_i + k + 2 * h), br = ld2(b_r + k + 2 * h),
                      bi = ld2(b_i + k + 2 * h);
            sr[h] += ar * br + ai * bi;
            si[h] += ar * bi - ai * br;
        }
    for (; k < N; k += 2) {
        const v2d ar = ld2(a_r + k), ai = ld2(a_i + k), br = ld2(b_r + k), bi = ld2(b_i + k);
        sr[0] += ar * br + ai * bi;
        si[0] += ar * bi - ai * br;
    }
    return make_double2(hsum(sr[0] + sr[1]), hsum(si[0] + si[1]));
}

// Largest root of the Lanczos tridiagonal by Sturm-sequence bisection,
// starting from `floor_` (the Ritz values only grow with the step count).
double ritz_max(const std::vector<double> &al, const std::vector<double> &be, double floor_)
{
    const int n = (int)al.size();
    double lo = al[0], hi = al[0];
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(be[i]) : 0.0);
        lo = std::min(lo, al[i] - r);
        hi = std::max(hi, al[i] + r);
    }
    if (floor_ > lo && floor_ < hi) lo = floor_;
    auto below = [&](double x) {   // eigenvalues of the tridiagonal below x
        int c = 0;
        double dd = 1.0;
        for (int i = 0; i < n; ++i) {
            dd = al[i] - x - (i > 0 ? be[i - 1] * be[i - 1] / dd : 0.0);
            if (dd == 0.0) dd = -1e-300;
            if (dd < 0.0) ++c;
        }
        return c;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::fabs(hi); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) >= n)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Largest eigenvalue of the Hermitian positive definite operator `op` (w = op
// v on padded split vectors of length N, K of them significant) by Lanczos
// with full reorthogonalisation (classical Gram-Schmidt, repeated once when
// the first pass cancels more than half of the squared norm: without it, a
// vector formed after the Krylov space has converged keeps rounding-level
// components along the earlier ones, and the Ritz values of the next steps
// overshoot the spectrum), stopped once the largest Ritz value changes by
// less than 1e-12 relative over five steps (checked at steps 10, 15, ..., at
// most 40).  On these clustered spectra plain power iterations stay
// percent-level low after 100 steps; this converges to about 1e-11 in 15-40.
template <class Op>
double largest(int K, int N, Op op)
{
    const int m = std::min(K, 40);
    Split Q(m + 1, N), W(1, N);
    std::vector<double> cr(m + 1), ci(m + 1), al, be;
    double *wr = W.r(0), *wi = W.i(0);
    double nv = 0;
    for (int i = 0; i < K; ++i) {
        Q.r(0)[i] = 1.0 + 0.01 * i;
        Q.i(0)[i] = 0.003 * i;
        nv += Q.r(0)[i] * Q.r(0)[i] + Q.i(0)[i] * Q.i(0)[i];
    }
    nv = std::sqrt(nv);
    for (int i = 0; i < K; ++i) {
        Q.r(0)[i] /= nv;
        Q.i(0)[i] /= nv;
    }
    double prev = -1.0, lam = 0.0;
    for (int j = 0; j < m; ++j) {
        op(Q.r(j), Q.i(j), wr, wi);
        al.push_back(dotc(N, Q.r(j), Q.i(j), wr, wi).x);
        double before = dotc(N, wr, wi, wr, wi).x;
        for (int pass = 0; pass < 2; ++pass) {
            // c = Q^H w over the j + 1 vectors so far (the rows of Q), then w -= Q^T c.
            for (int i = 0; i <= j; ++i) {
                const double2 c = dotc(N, Q.r(i), Q.i(i), wr, wi);
                cr[i] = c.x;
                ci[i] = c.y;
            }
            for (int i = 0; i <= j; ++i) {
                const v2d a = v2d{cr[i], cr[i]}, b = v2d{ci[i], ci[i]};
                const double *ur = Q.r(i), *ui = Q.i(i);
                for (int k = 0; k < N; k += 2) {
                    const v2d qr2 = ld2(ur + k), qi2 = ld2(ui + k);
                    st2(wr + k, ld2(wr + k) - (a * qr2 - b * qi2));
                    st2(wi + k, ld2(wi + k) - (a * qi2 + b * qr2));
                }
            }
            const double after = dotc(N, wr, wi, wr, wi).x;
            if (after >= 0.5 * before) break;
            before = after;
        }
        const bool check = j >= 10 && (j % 5 == 0 || j == m - 1);
        if (check || j == m - 1) {
            lam = ritz_max(al, be, prev);
            if (check && prev > 0 && std::fabs(lam - prev) <= 1e-12 * lam) break;
            prev = lam * (1.0 - 1e-15);   // bisection floor for the next check
        }
        const double bn = std::sqrt(dotc(N, wr, wi, wr, wi).x);
        if (!(bn > 1e-14 * std::fabs(al.back()))) {   // invariant subspace: its Ritz values are exact
            lam = ritz_max(al, be, prev);
            break;
        }
        be.push_back(bn);
        for (int k = 0; k < N; ++k) {
            Q.r(j + 1)[k] = wr[k] / bn;
            Q.i(j + 1)[k] = wi[k] / bn;
        }
    }
    return lam;
}

// Largest eigenvalue of D G D (D = diag(G)^{-1/2}, as the factorisation forms it).
double largest_dgd(const double2 *G, int K)
{
    const int N = (K + 1) & ~1;
    std::vector<double> d(K);
    for (int i = 0; i < K; ++i) {
        const double gii = G[(size_t)i * K + i].x;
        d[i] = gii > 0.0 ? 1.0 / std::sqrt(gii) : 0.0;
    }
    Split A(K, N);
    for (int i = 0; i < K; ++i)
        for (int k = 0; k < K; ++k) {
            A.r(i)[k] = G[(size_t)i * K + k].x * d[i] * d[k];
            A.i(i)[k] = G[(size_t)i * K + k].y * d[i] * d[k];
        }
    return largest(K, N, [&](const double *vr, const double *vi, double *wr, double *wi) {
        matvec(A, K, false, vr, vi, wr, wi);
    });
}

// Largest eigenvalue of (L L^H)^{-1} = L^{-H} L^{-1}, from L^{-1} (lower triangle).
double largest_inverse(const double2 *Linv, int K)
{
    const int N = (K + 1) & ~1;
    Split Li(K, N), T(1, N);
    for (int i = 0; i < K; ++i)
        for (int k = 0; k <= i; ++k) {
            Li.r(i)[k] = Linv[(size_t)i * K + k].x;
            Li.i(i)[k] = Linv[(size_t)i * K + k].y;
        }
    return largest(K, N, [&](const double *vr, const double *vi, double *wr, double *wi) {
        matvec(Li, K, true, vr, vi, T.r(0), T.i(0));
        matvec_h_lower(Li, K, T.r(0), T.i(0), wr, wi);
    });
}

}  // namespace cond

// Statistics of a problem: ||t - Psi h||^2 and ||t||^2 of the final
// coefficients (FP32 residual summed in FP64 on the device), queued on s and
// read back into the pinned w.h_norm.
dpd_status queue_norms(dpd_handle h, int p, const float2 *u, const float2 *t, int64_t n, cudaStream_t s)
{
    EstimateWorkspace &w = h->est;
    dpd_status st = residual_of(h, p, u, t, n, s, true);
    if (st != DPD_OK) return st;
    if (cudaMemcpyAsync(w.h_norm, w.norm_part + 2 * dpd::kFwdNormSlots, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                        s) !=
        cudaSuccess)
        return DPD_ERR_CUDA;
    return DPD_OK;
}

dpd_status check_inputs(dpd_handle h, const void *u, const void *t, int64_t n, int precision)
{
    if (!h || n < 1 || !u || !aligned8(u) || (t && !aligned8(t))) return DPD_ERR_INVALID_ARGUMENT;
    if (!valid_precision(precision)) return DPD_ERR_INVALID_ARGUMENT;
    if (n > ((int64_t)1 << 40)) return DPD_ERR_UNSUPPORTED;
    if (dpd::gram_distinct(h->B, h->T) > dpd::kGramS) return DPD_ERR_UNSUPPORTED;
    return DPD_OK;
}

}  // namespace

void free_estimate_workspace(EstimateWorkspace &w)
{
    cudaFree(w.probs);
    cudaFree(w.partials);
    cudaFree(w.Clag);
    cudaFree(w.S);
    cudaFree(w.G);
    cudaFree(w.g);
    cudaFree(w.L);
    cudaFree(w.h64);
    cudaFree(w.delta);
    cudaFree(w.d);
    cudaFree(w.tt);
    cudaFree(w.info);
    cudaFree(w.hf);
    cudaFree(w.tab);
    cudaFree(w.y);
    cudaFree(w.e);
    cudaFree(w.norm_part);
    cudaFree(w.ubasis);
    cudaFree(w.ubasis64);
    cudaFree(w.mom);
    cudaFree(w.mom_part);
    cudaFree(w.hm64);
    cudaFree(w.Linv);
    cudaFree(w.tmpv);
    cudaFree(w.tabb);
    cudaFree(w.bstreams);
    cudaFree(w.bitems);
    cudaFree(w.badj);
    cudaFree(w.bpart);
    cudaFreeHost(w.h_G);
    cudaFreeHost(w.h_Linv);
    cudaFreeHost(w.h_info);
    cudaFreeHost(w.h_norm);
    if (w.ev_L) cudaEventDestroy(w.ev_L);
    if (w.ev_G) cudaEventDestroy(w.ev_G);
    w = EstimateWorkspace();
}

extern "C" {

dpd_status dpd_set_estimate_basis(dpd_handle h, int basis)
{
    if (!h || (basis != DPD_BASIS_MONOMIAL && basis != DPD_BASIS_ORTHOGONAL)) return DPD_ERR_INVALID_ARGUMENT;
    h->est_basis = basis;
    return DPD_OK;
}

dpd_status dpd_gram(dpd_handle h, const void *u, const void *t, int64_t n, int precision, void *G, void *g,
                    double *tt, void *stream)
{
    dpd_status st = check_inputs(h, u, t, n, precision);
    if (st != DPD_OK) return st;
    if (!G || !aligned8(G) || (g && (!t || !aligned8(g)))) return DPD_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int cpp = gram_cpp(h, 1, n, precision);
    if ((st = reserve(h, 1, cpp, 0)) != DPD_OK) return st;
    // Psi of Eq. 2 (the monomial basis, whatever the handle's estimate basis);
    // the problem travels by value in the kernel arguments.
    const dpd::GramProblem pr{static_cast<const float2 *>(u), static_cast<const float2 *>(t), n};
    if ((st = run_gram(h, 1, cpp, precision, s, &pr, static_cast<double2 *>(G), static_cast<double2 *>(g), true)) !=
        DPD_OK)
        return st;
    if (tt && t && (cudaMemcpyAsync(tt, h->est.tt, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess))
        return DPD_ERR_CUDA;
    return DPD_OK;
}

dpd_status dpd_estimate(dpd_handle h, const void *u, const void *t, int64_t n, int precision, int refine_iters,
                        void *h_out, double *stats, void *stream)
{
    dpd_status st = check_inputs(h, u, t, n, precision);
    if (st != DPD_OK) return st;
    if (!t || !h_out || !aligned8(h_out) || refine_iters < 0 || refine_iters > 100) return DPD_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int cpp = gram_cpp(h, 1, n, precision);
    if ((st = reserve(h, 1, cpp, (refine_iters > 0 || stats) ? n : 0)) != DPD_OK) return st;
    EstimateWorkspace &w = h->est;
    const dpd::GramProblem pr{static_cast<const float2 *>(u), static_cast<const float2 *>(t), n};
    if (ortho(h)) {
        if (cudaMemcpyAsync(w.probs, &pr, sizeof(pr), cudaMemcpyHostToDevice, s) != cudaSuccess) return DPD_ERR_CUDA;
        if ((st = compute_basis(h, std::vector<int64_t>{n}, s)) != DPD_OK) return st;
    }
    if ((st = run_gram(h, 1, cpp, precision, s, ortho(h) ? nullptr : &pr)) != DPD_OK) return st;
    // For the statistics, G and (after the factorisation) the inverse factor go
    // to pinned host memory while the device carries on, and so does the pivot
    // status: the host condition estimate (Lanczos on D G D from G, and on its
    // inverse) runs during the factorisation and the refinement instead of
    // after them, and the solves skip a failed factorisation on the device.
    const int K = h->K;
    if (stats && (cudaMemcpyAsync(w.h_G, w.G, sizeof(double2) * K * K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                  cudaEventRecord(w.ev_G, s) != cudaSuccess))
        return DPD_ERR_CUDA;
    if (dpd::launch_chol(w.G, 1, h->K, w.L, w.d, w.info, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (cudaMemcpyAsync(w.h_info, w.info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    // The solves go through the explicit inverse of L: two parallel
    // matrix-vector products instead of two K-step sequential chains each.
    if (dpd::launch_chol_invert(w.L, w.info, K, w.Linv, s) != cudaSuccess) return DPD_ERR_CUDA;
    if ((stats && cudaMemcpyAsync(w.h_Linv, w.Linv, sizeof(double2) * K * K, cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess) ||
        cudaEventRecord(w.ev_L, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    w.use_inverse = true;
    if (dpd::launch_solve_inverse(w.Linv, w.d, w.info, w.g, K, w.tmpv, w.h64, 0, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    for (int i = 0; i < refine_iters; ++i)
        if ((st = refine_once(h, 0, pr.u, pr.t, n, s)) != DPD_OK) return st;
    const double2 *hm = monomial_h(h, 0, 1, s, st);
    if (st != DPD_OK) return st;
    if (dpd::launch_h_to_f32(hm, K, static_cast<float2 *>(h_out), s) != cudaSuccess) return DPD_ERR_CUDA;
    if (stats && (st = queue_norms(h, 0, pr.u, pr.t, n, s)) != DPD_OK) return st;
    // The two Lanczos runs overlap the queued device work: the one on D G D
    // (a second host thread) as soon as G has landed, the one on the inverse
    // once the inverse factor has.
    double lmax = 0.0, linv = 0.0;
    std::thread dgd_run;
    bool threaded = false;
    if (stats) {
        if (cudaEventSynchronize(w.ev_G) != cudaSuccess) return DPD_ERR_CUDA;
        try {
            dgd_run = std::thread([&] { lmax = cond::largest_dgd(w.h_G, K); });
            threaded = true;
        } catch (const std::system_error &) {   // no thread available: on this one, below
        }
    }
    const bool synced = cudaEventSynchronize(w.ev_L) == cudaSuccess;
    const int info = synced ? *w.h_info : 0;
    if (synced && stats && info == 0) linv = cond::largest_inverse(w.h_Linv, K);
    if (threaded) dgd_run.join();
    if (!synced) return DPD_ERR_CUDA;
    if (stats && !threaded) lmax = cond::largest_dgd(w.h_G, K);
    const double cond = lmax * linv;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DPD_ERR_CUDA;
    if (info != 0) return DPD_ERR_NOT_SPD;
    if (stats) {
        stats[0] = cond;
        stats[1] = w.h_norm[1] > 0 ? w.h_norm[0] / w.h_norm[1] : 0.0;
    }
    return DPD_OK;
}

dpd_status dpd_estimate_batched(dpd_handle h, const void *const *u, const void *const *t, const int64_t *n,
                                int count, int precision, int refine_iters, void *h_out, int *info_out, void *stream)
{
    if (!h || count < 1 || !u || !t || !n || !h_out || !aligned8(h_out)) return DPD_ERR_INVALID_ARGUMENT;
    if (refine_iters < 0 || refine_iters > 100 || !valid_precision(precision)) return DPD_ERR_INVALID_ARGUMENT;
    if (dpd::gram_distinct(h->B, h->T) > dpd::kGramS) return DPD_ERR_UNSUPPORTED;
    std::vector<dpd::GramProblem> probs((size_t)count);
    int64_t nmax = 1;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || !u[i] || !t[i] || !aligned8(u[i]) || !aligned8(t[i])) return DPD_ERR_INVALID_ARGUMENT;
        probs[i] = {static_cast<const float2 *>(u[i]), static_cast<const float2 *>(t[i]), n[i]};
        nmax = std::max(nmax, n[i]);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int cpp = gram_cpp(h, count, nmax, precision);
    // Refinement of all problems together needs 16-byte aligned inputs and one
    // residual buffer per problem; otherwise the problems are refined one by one.
    bool together = refine_iters > 0 && count > 1;
    for (int i = 0; i < count && together; ++i) together = (reinterpret_cast<uintptr_t>(u[i]) & 15u) == 0;
    const int64_t nsamp = refine_iters > 0 ? (together ? ((nmax + 1) & ~int64_t(1)) * count : nmax) : 0;
    dpd_status st = reserve(h, count, cpp, nsamp);
    if (st != DPD_OK) return st;
    EstimateWorkspace &w = h->est;
    if (cudaMemcpyAsync(w.probs, probs.data(), sizeof(dpd::GramProblem) * count, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return DPD_ERR_CUDA;
    if (ortho(h) && (st = compute_basis(h, std::vector<int64_t>(n, n + count), s)) != DPD_OK) return st;
    if ((st = run_gram(h, count, cpp, precision, s)) != DPD_OK) return st;
    if (dpd::launch_chol(w.G, count, h->K, w.L, w.d, w.info, s) != cudaSuccess) return DPD_ERR_CUDA;
    w.use_inverse = false;
    if (dpd::launch_chol_solve(w.L, w.d, w.info, w.g, count, h->K, w.h64, 0, s) != cudaSuccess) return DPD_ERR_CUDA;
    // The pivot status comes back here only for the refinement problem by
    // problem, which skips problems that did not factor; refined together, the
    // launches are queued behind the solve without a host round trip and the
    // status is read at the end.
    std::vector<int> info((size_t)count);
    if (!together && (cudaMemcpyAsync(info.data(), w.info, sizeof(int) * count, cudaMemcpyDeviceToHost, s) !=
                          cudaSuccess ||
                      cudaStreamSynchronize(s) != cudaSuccess))
        return DPD_ERR_CUDA;
    if (together) {   // problems that did not factor keep unspecified coefficients
        if ((st = refine_batched(h, probs, nmax, refine_iters, s)) != DPD_OK) return st;
    } else {
        for (int it = 0; it < refine_iters; ++it)
            for (int p = 0; p < count; ++p)
                if (info[p] == 0 && (st = refine_once(h, p, probs[p].u, probs[p].t, probs[p].n, s)) != DPD_OK)
                    return st;
    }
    const double2 *hm = monomial_h(h, 0, count, s, st);
    if (st != DPD_OK) return st;
    if (dpd::launch_h_to_f32(hm, count * h->K, static_cast<float2 *>(h_out), s) != cudaSuccess) return DPD_ERR_CUDA;
    if (together &&
        cudaMemcpyAsync(info.data(), w.info, sizeof(int) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DPD_ERR_CUDA;
    bool any_bad = false;
    for (int i = 0; i < count; ++i) any_bad |= info[i] != 0;
    if (info_out) std::copy(info.begin(), info.end(), info_out);
    return any_bad ? DPD_ERR_NOT_SPD : DPD_OK;
}

}  // extern "C"
