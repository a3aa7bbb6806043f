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
        ok = ok && grow(w.S, 0, np * dpd::kGramS * dpd::kGramPartCols);
        ok = ok && grow(w.G, 0, np * K * K) && grow(w.L, 0, np * K * K);
        ok = ok && grow(w.g, 0, np * K) && grow(w.h64, 0, np * K) && grow(w.delta, 0, np * K);
        ok = ok && grow(w.d, 0, np * K) && grow(w.tt, 0, np) && grow(w.info, 0, np);
        ok = ok && grow(w.hf, 0, (size_t)K) && grow(w.tab, 0, (size_t)dpd::wl_table_floats(h->B, h->T));
        ok = ok && grow(w.norm_part, 0, (size_t)2 * 1024 + 2);
        ok = ok && grow(w.ubasis, 0, np * dpd::kUSize) && grow(w.ubasis64, 0, np * dpd::kUSize);
        ok = ok && grow(w.mom, 0, np * dpd::kMomK) && grow(w.mom_part, 0, np * dpd::kMomBlocks * dpd::kMomK);
        ok = ok && grow(w.hm64, 0, np * K);
        ok = ok && grow(w.Linv, 0, (size_t)K * K) && grow(w.tmpv, 0, (size_t)K);
        if (!ok) return DPD_ERR_ALLOC;
        w.nprob = nprob;
        w.cpp = cpp;
    }
    if (w.hK != K || !w.h_L) {
        cudaFreeHost(w.h_L);
        cudaFreeHost(w.h_info);
        cudaFreeHost(w.h_norm);
        w.h_L = nullptr;
        w.h_info = nullptr;
        w.h_norm = nullptr;
        w.hK = 0;
        if (cudaMallocHost(&w.h_L, sizeof(double2) * K * K) != cudaSuccess ||
            cudaMallocHost(&w.h_info, sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&w.h_norm, 2 * sizeof(double)) != cudaSuccess)
            return DPD_ERR_ALLOC;
        w.hK = K;
    }
    if (!w.ev_L && cudaEventCreateWithFlags(&w.ev_L, cudaEventDisableTiming) != cudaSuccess) return DPD_ERR_CUDA;
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

// Gram (+ reduction + assembly) of nprob problems already described in w.probs.
dpd_status run_gram(dpd_handle h, int nprob, int cpp, int precision, cudaStream_t s)
{
    EstimateWorkspace &w = h->est;
    dpd::GramArgs a;
    a.probs = static_cast<const dpd::GramProblem *>(w.probs);
    a.nprob = nprob;
    a.cpp = cpp;
    a.Bp = h->Bp;
    a.Bq = h->Bq;
    a.T = h->T;
    a.K = h->K;
    a.partials = w.partials;
    a.status = h->d_status;
    a.ubasis = ortho(h) ? w.ubasis : nullptr;
    if (dpd::launch_gram(precision, a, s) != cudaSuccess) return DPD_ERR_CUDA;
    const int D = dpd::gram_distinct(h->B, h->T);
    if (dpd::launch_gram_reduce(w.partials, nprob, cpp, D, w.S, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (dpd::launch_gram_assemble(w.S, nprob, h->K, h->Bp, h->B, h->T, w.G, w.g, w.tt, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    return DPD_OK;
}

// e = t - Psi(u) h for the current FP64 coefficients of problem p (FP32 filter);
// with `norms`, also ||e||^2 and ||t||^2 into w.norm_part + 2048.
dpd_status residual_of(dpd_handle h, int p, const float2 *u, const float2 *t, int64_t n, cudaStream_t s,
                       bool norms = false)
{
    EstimateWorkspace &w = h->est;
    dpd_status st = DPD_OK;
    const double2 *hm = monomial_h(h, p, 1, s, st);
    if (st != DPD_OK) return st;
    if (dpd::launch_h_to_f32(hm, h->K, w.hf, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (dpd::launch_wl_table(w.hf, h->Bp, h->Bq, h->T, w.tab, nullptr, s) != cudaSuccess) return DPD_ERR_CUDA;
    dpd::FwdArgs fa;
    fa.x = u;
    fa.y = w.y;
    fa.n = n;
    fa.tab = w.tab;
    fa.status = h->d_status;
    fa.vec_store = 1;
    fa.host_tab = nullptr;
    dpd::FwdLaunch L = h->fwd;
    L.mode = dpd::kModePackedFma;   // coefficients live on the device
    if ((reinterpret_cast<uintptr_t>(u) & 15u) != 0) {
        L.use_tma = 0;
        L.V = 4;
    }
    if (dpd::launch_fwd_any(h->B, h->T, fa, L, h->sm_count, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (norms)
        return dpd::launch_residual_norm(t, w.y, n, w.e, w.norm_part, w.norm_part + 2 * 1024, s) == cudaSuccess
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

// 2-norm condition number of A = L L^H (the equilibrated Gram matrix): the
// largest eigenvalues of A and of A^{-1} (two triangular solves per product),
// FP64 on the host.
double cond_estimate(const double2 *L, int K)
{
    auto mulL = [&](const std::vector<double2> &x, bool herm) {   // L x or L^H x
        std::vector<double2> y((size_t)K, make_double2(0, 0));
        for (int i = 0; i < K; ++i)
            for (int k = 0; k <= i; ++k) {
                const double2 l = L[(size_t)i * K + k];
                if (!herm) {
                    y[i].x += l.x * x[k].x - l.y * x[k].y;
                    y[i].y += l.x * x[k].y + l.y * x[k].x;
                } else {
                    y[k].x += l.x * x[i].x + l.y * x[i].y;
                    y[k].y += l.x * x[i].y - l.y * x[i].x;
                }
            }
        return y;
    };
    auto solveL = [&](std::vector<double2> b, bool herm) {   // L^{-1} b or L^{-H} b
        if (!herm) {
            for (int i = 0; i < K; ++i) {
                double2 s = b[i];
                for (int k = 0; k < i; ++k) {
                    const double2 l = L[(size_t)i * K + k];
                    s.x -= l.x * b[k].x - l.y * b[k].y;
                    s.y -= l.x * b[k].y + l.y * b[k].x;
                }
                const double d = L[(size_t)i * K + i].x;
                b[i] = make_double2(s.x / d, s.y / d);
            }
        } else {
            for (int i = K - 1; i >= 0; --i) {
                double2 s = b[i];
                for (int k = i + 1; k < K; ++k) {
                    const double2 l = L[(size_t)k * K + i];
                    s.x -= l.x * b[k].x + l.y * b[k].y;
                    s.y -= l.x * b[k].y - l.y * b[k].x;
                }
                const double d = L[(size_t)i * K + i].x;
                b[i] = make_double2(s.x / d, s.y / d);
            }
        }
        return b;
    };
    // Largest eigenvalue of the Hermitian positive definite operator by Lanczos
    // with full reorthogonalisation (one Gram-Schmidt pass per step), stopped
    // once the largest Ritz value -- the largest root of the Lanczos
    // tridiagonal, found by Sturm-sequence bisection -- changes by less than
    // 1e-12 relative over five steps (checked at steps 10, 15, ..., at most
    // 40).  On these clustered spectra plain power iterations stay
    // percent-level low after 100 steps; this converges to about 1e-11 in
    // 15-30.  The largest Ritz value only grows with the step count, so each
    // bisection starts from the previous one.
    auto dotc = [&](const std::vector<double2> &a, const std::vector<double2> &b) {   // a^H b
        double2 r = make_double2(0, 0);
        for (int i = 0; i < K; ++i) {
            r.x += a[i].x * b[i].x + a[i].y * b[i].y;
            r.y += a[i].x * b[i].y - a[i].y * b[i].x;
        }
        return r;
    };
    auto ritz_max = [](const std::vector<double> &al, const std::vector<double> &be, double floor_) {
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
            double d = 1.0;
            for (int i = 0; i < n; ++i) {
                d = al[i] - x - (i > 0 ? be[i - 1] * be[i - 1] / d : 0.0);
                if (d == 0.0) d = -1e-300;
                if (d < 0.0) ++c;
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
    };
    auto largest = [&](bool inverse) {
        const int m = std::min(K, 40);
        std::vector<std::vector<double2>> q;
        std::vector<double> al, be;
        std::vector<double2> v((size_t)K);
        double nv = 0;
        for (int i = 0; i < K; ++i) {
            v[i] = make_double2(1.0 + 0.01 * i, 0.003 * i);
            nv += v[i].x * v[i].x + v[i].y * v[i].y;
        }
        nv = std::sqrt(nv);
        for (auto &e : v) e = make_double2(e.x / nv, e.y / nv);
        q.push_back(v);
        double prev = -1.0, lam = 0.0;
        for (int j = 0; j < m; ++j) {
            std::vector<double2> w =
                inverse ? solveL(solveL(q[j], false), true) : mulL(mulL(q[j], true), false);
            al.push_back(dotc(q[j], w).x);
            for (int i = 0; i <= j; ++i) {
                const double2 c = dotc(q[i], w);
                for (int k = 0; k < K; ++k) {
                    w[k].x -= c.x * q[i][k].x - c.y * q[i][k].y;
                    w[k].y -= c.x * q[i][k].y + c.y * q[i][k].x;
                }
            }
            const bool check = j >= 10 && (j % 5 == 0 || j == m - 1);
            if (check || j == m - 1) {
                lam = ritz_max(al, be, prev);
                if (check && prev > 0 && std::fabs(lam - prev) <= 1e-12 * lam) break;
                prev = lam * (1.0 - 1e-15);   // bisection floor for the next check
            }
            double bn = 0;
            for (const auto &e : w) bn += e.x * e.x + e.y * e.y;
            bn = std::sqrt(bn);
            if (!(bn > 1e-14 * std::fabs(al.back()))) {   // invariant subspace: its Ritz values are exact
                lam = ritz_max(al, be, prev);
                break;
            }
            be.push_back(bn);
            for (auto &e : w) e = make_double2(e.x / bn, e.y / bn);
            q.push_back(w);
        }
        return lam;
    };
    // The two runs are independent: the inverse one on a second host thread.
    double linv = 0.0;
    try {
        std::thread inv_run([&] { linv = largest(true); });
        const double lmax = largest(false);
        inv_run.join();
        return lmax * linv;
    } catch (const std::system_error &) {   // no thread available: one after the other
        return largest(false) * largest(true);
    }
}

// Statistics of a problem: ||t - Psi h||^2 and ||t||^2 of the final
// coefficients (FP32 residual summed in FP64 on the device), queued on s and
// read back into the pinned w.h_norm.
dpd_status queue_norms(dpd_handle h, int p, const float2 *u, const float2 *t, int64_t n, cudaStream_t s)
{
    EstimateWorkspace &w = h->est;
    dpd_status st = residual_of(h, p, u, t, n, s, true);
    if (st != DPD_OK) return st;
    if (cudaMemcpyAsync(w.h_norm, w.norm_part + 2 * 1024, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
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
    cudaFreeHost(w.h_L);
    cudaFreeHost(w.h_info);
    cudaFreeHost(w.h_norm);
    if (w.ev_L) cudaEventDestroy(w.ev_L);
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
    const dpd::GramProblem pr{static_cast<const float2 *>(u), static_cast<const float2 *>(t), n};
    if (cudaMemcpyAsync(h->est.probs, &pr, sizeof(pr), cudaMemcpyHostToDevice, s) != cudaSuccess) return DPD_ERR_CUDA;
    if ((st = run_gram(h, 1, cpp, precision, s)) != DPD_OK) return st;
    const size_t KK = (size_t)h->K * h->K;
    if (cudaMemcpyAsync(G, h->est.G, sizeof(double2) * KK, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    if (g && cudaMemcpyAsync(g, h->est.g, sizeof(double2) * h->K, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return DPD_ERR_CUDA;
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
    if (cudaMemcpyAsync(w.probs, &pr, sizeof(pr), cudaMemcpyHostToDevice, s) != cudaSuccess) return DPD_ERR_CUDA;
    if (ortho(h) && (st = compute_basis(h, std::vector<int64_t>{n}, s)) != DPD_OK) return st;
    if ((st = run_gram(h, 1, cpp, precision, s)) != DPD_OK) return st;
    if (dpd::launch_chol(w.G, 1, h->K, w.L, w.d, w.info, s) != cudaSuccess) return DPD_ERR_CUDA;
    // The factor and its pivot status go to pinned host memory while the
    // device carries on: the solves skip a failed factorisation on the device,
    // and the host condition estimate (Lanczos on L) runs during the
    // refinement instead of after it.
    const int K = h->K;
    if (cudaMemcpyAsync(w.h_info, w.info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (stats && cudaMemcpyAsync(w.h_L, w.L, sizeof(double2) * K * K, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaEventRecord(w.ev_L, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    // The solves go through the explicit inverse of L: two parallel
    // matrix-vector products instead of two K-step sequential chains each.
    if (dpd::launch_chol_invert(w.L, w.info, K, w.Linv, s) != cudaSuccess) return DPD_ERR_CUDA;
    w.use_inverse = true;
    if (dpd::launch_solve_inverse(w.Linv, w.d, w.info, w.g, K, w.tmpv, w.h64, 0, s) != cudaSuccess)
        return DPD_ERR_CUDA;
    for (int i = 0; i < refine_iters; ++i)
        if ((st = refine_once(h, 0, pr.u, pr.t, n, s)) != DPD_OK) return st;
    const double2 *hm = monomial_h(h, 0, 1, s, st);
    if (st != DPD_OK) return st;
    if (dpd::launch_h_to_f32(hm, K, static_cast<float2 *>(h_out), s) != cudaSuccess) return DPD_ERR_CUDA;
    if (stats && (st = queue_norms(h, 0, pr.u, pr.t, n, s)) != DPD_OK) return st;
    double cond = 0.0;
    if (cudaEventSynchronize(w.ev_L) != cudaSuccess) return DPD_ERR_CUDA;
    const int info = *w.h_info;
    if (stats && info == 0) cond = cond_estimate(w.h_L, K);   // overlaps the queued device work
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
    dpd_status st = reserve(h, count, cpp, refine_iters > 0 ? nmax : 0);
    if (st != DPD_OK) return st;
    EstimateWorkspace &w = h->est;
    if (cudaMemcpy(w.probs, probs.data(), sizeof(dpd::GramProblem) * count, cudaMemcpyHostToDevice) != cudaSuccess)
        return DPD_ERR_CUDA;
    if (ortho(h) && (st = compute_basis(h, std::vector<int64_t>(n, n + count), s)) != DPD_OK) return st;
    if ((st = run_gram(h, count, cpp, precision, s)) != DPD_OK) return st;
    if (dpd::launch_chol(w.G, count, h->K, w.L, w.d, w.info, s) != cudaSuccess) return DPD_ERR_CUDA;
    w.use_inverse = false;
    if (dpd::launch_chol_solve(w.L, w.d, w.info, w.g, count, h->K, w.h64, 0, s) != cudaSuccess) return DPD_ERR_CUDA;
    std::vector<int> info((size_t)count);
    if (cudaMemcpyAsync(info.data(), w.info, sizeof(int) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DPD_ERR_CUDA;
    bool any_bad = false;
    for (int i = 0; i < count; ++i) any_bad |= info[i] != 0;
    for (int it = 0; it < refine_iters; ++it)
        for (int p = 0; p < count; ++p)
            if (info[p] == 0 && (st = refine_once(h, p, probs[p].u, probs[p].t, probs[p].n, s)) != DPD_OK) return st;
    const double2 *hm = monomial_h(h, 0, count, s, st);
    if (st != DPD_OK) return st;
    if (dpd::launch_h_to_f32(hm, count * h->K, static_cast<float2 *>(h_out), s) != cudaSuccess) return DPD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DPD_ERR_CUDA;
    if (info_out) std::copy(info.begin(), info.end(), info_out);
    return any_bad ? DPD_ERR_NOT_SPD : DPD_OK;
}

}  // extern "C"
