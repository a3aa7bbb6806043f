// FP64 side of the least-squares estimate (see dpd_gram.cuh): fixed-order
// reduction of the Gram partials, assembly of G = Psi^H Psi and g = Psi^H t,
// equilibrated Cholesky factorisation and triangular solves, and the small
// kernels of the iterative refinement.
#include <cooperative_groups.h>

#include "dpd_gram.cuh"

namespace dpd {

// Column sums over the problem's CTAs of the partial P and Q blocks (rows and
// columns < D), in FP64 and a fixed order: SPQ[i][c] for c < 2 kGramS.
constexpr int kReduceGroups = 8;   // partial groups per column, summed by separate warps

__global__ void __launch_bounds__(32 * kReduceGroups) gram_reduce_kernel(const float *__restrict__ partials, int cpp,
                                                                         int D, double *__restrict__ SPQ)
{
    // Lane l of warp g sums partials g, g + 8, g + 16, ... of entry idx in
    // FP64 (four interleaved sums), then warp 0 adds the eight group sums in
    // group order: a fixed order, with up to 19 loads in flight per thread
    // instead of one chain over all partials.
    __shared__ double grp[kReduceGroups][32];
    const int p = blockIdx.y;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int idx = blockIdx.x * 32 + lane;   // i * kGramPartCols + c
    const bool in = idx < kGramS * kGramPartCols;
    const int i = idx / kGramPartCols, c = idx % kGramPartCols, j = c % kGramS;
    double s = 0.0;
    if (in && i < D && j < D) {
        const size_t part = (size_t)kGramRows * kGramPartCols;
        const float *base = partials + (size_t)p * cpp * part + (size_t)i * kGramPartCols + c;
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        int k = g, q = 0;
        for (; k < cpp; k += kReduceGroups, q = (q + 1) & 3) s4[q] += (double)base[(size_t)k * part];
        s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    grp[g][lane] = s;
    __syncthreads();
    if (g == 0 && in) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kReduceGroups; ++q) t += grp[q][lane];
        SPQ[(size_t)p * kGramS * kGramPartCols + idx] = t;
    }
}

cudaError_t launch_gram_reduce(const float *partials, int nprob, int cpp, int D, double *S, cudaStream_t s)
{
    dim3 grid((kGramS * kGramPartCols + 31) / 32, nprob);
    gram_reduce_kernel<<<grid, 32 * kReduceGroups, 0, s>>>(partials, cpp, D, S);
    count_launch();
    return cudaGetLastError();
}

// Each thread sums its powers as FP32 pairs (sum, rounding error) with an
// exact two-sum per addition: FP32 arithmetic, about 2^-48 relative accuracy,
// where FP64 additions (about two per clock per SM on GB300) bound the kernel.
// The pairs become FP64 for the block's fixed-order tree.
__global__ void moments_kernel(const GramProblem *__restrict__ probs, double *__restrict__ part)
{
    const GramProblem pr = probs[blockIdx.y];
    float hi[kMomK], lo[kMomK];
#pragma unroll
    for (int k = 0; k < kMomK; ++k) {
        hi[k] = 0.f;
        lo[k] = 0.f;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pr.n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = pr.u[i];
        const float r = fmaf(x.x, x.x, x.y * x.y);
        float p = r;
#pragma unroll
        for (int k = 0; k < kMomK; ++k) {
            const float t = hi[k] + p, z = t - hi[k];
            lo[k] += (hi[k] - (t - z)) + (p - z);
            hi[k] = t;
            p *= r;
        }
    }
    __shared__ double red[kMomK][256];
#pragma unroll
    for (int k = 0; k < kMomK; ++k) red[k][threadIdx.x] = (double)hi[k] + (double)lo[k];
    __syncthreads();
    for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
#pragma unroll
            for (int k = 0; k < kMomK; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x < kMomK)
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kMomK + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void moments_sum_kernel(const double *__restrict__ part, int blocks, double *__restrict__ mom)
{
    const int p = blockIdx.x, k = threadIdx.x;
    if (k >= kMomK) return;
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += part[((size_t)p * blocks + b) * kMomK + k];
    mom[(size_t)p * kMomK + k] = s;
}

cudaError_t launch_moments(const GramProblem *probs, int nprob, double *part, double *mom, cudaStream_t s)
{
    moments_kernel<<<dim3(kMomBlocks, nprob), 256, 0, s>>>(probs, part);
    count_launch();
    moments_sum_kernel<<<nprob, 32, 0, s>>>(part, kMomBlocks, mom);
    count_launch();
    return cudaGetLastError();
}

__global__ void basis_transform_kernel(const double2 *__restrict__ in, double2 *__restrict__ out,
                                       const double *__restrict__ Uall, int K, int Bp, int Bq, int T, int to_monomial)
{
    const int p = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const double2 *x = in + (size_t)p * K;
    const double *U = Uall + (size_t)p * kUSize;
    double2 v;
    if (j == K - 1) {
        v = x[j];
    } else {
        const bool conj = j >= Bp * T;
        const int base = conj ? Bp * T : 0, nb = conj ? Bq : Bp, jj = j - base, a = jj / T, k = jj % T;
        v = make_double2(0.0, 0.0);
        if (to_monomial) {   // h[(a, k)] = sum_{b >= a} U[a][b] h_U[(b, k)]
            for (int b = a; b < nb; ++b) {
                const double u = U[a * kMaxB + b];
                v.x += u * x[base + b * T + k].x;
                v.y += u * x[base + b * T + k].y;
            }
        } else {             // g_U[(a, k)] = sum_{c <= a} U[c][a] g[(c, k)]
            for (int c = 0; c <= a; ++c) {
                const double u = U[c * kMaxB + a];
                v.x += u * x[base + c * T + k].x;
                v.y += u * x[base + c * T + k].y;
            }
        }
    }
    out[(size_t)p * K + j] = v;
}

cudaError_t launch_basis_transform(const double2 *in, double2 *out, const double *U, int nprob, int K, int Bp,
                                   int Bq, int T, int to_monomial, cudaStream_t s)
{
    basis_transform_kernel<<<dim3((K + 127) / 128, nprob), 128, 0, s>>>(in, out, U, K, Bp, Bq, T, to_monomial);
    count_launch();
    return cudaGetLastError();
}

// <x, y> for two signed distinct-column references: S = P + Q + Q^T from the
// summed blocks (P upper triangle in columns [0, kGramS), Q in [kGramS, 2 kGramS)).
__device__ __forceinline__ double dot(const double *SPQ, ColRef x, ColRef y)
{
    if (x.sign == 0 || y.sign == 0) return 0.0;
    const int i = x.d < y.d ? x.d : y.d, j = x.d < y.d ? y.d : x.d;
    const double v = SPQ[(size_t)i * kGramPartCols + j] + SPQ[(size_t)i * kGramPartCols + kGramS + j] +
                     SPQ[(size_t)j * kGramPartCols + kGramS + i];
    return x.sign * y.sign > 0 ? v : -v;
}

__global__ void gram_assemble_kernel(const double *__restrict__ Sall, int K, int Bp, int B, int T,
                                     double2 *__restrict__ G, double2 *__restrict__ g, double *__restrict__ tt)
{
    const int p = blockIdx.y;
    const double *S = Sall + (size_t)p * kGramS * kGramPartCols;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const ColRef tre{2 * B * T + 1, 1}, tim{2 * B * T + 2, 1};
    if (idx < K * K) {
        const int a = idx / K, b = idx % K;
        ColRef ar, ai, br, bi;
        psi_column_refs(a, K, Bp, B, T, ar, ai);
        psi_column_refs(b, K, Bp, B, T, br, bi);
        G[(size_t)p * K * K + idx] = make_double2(dot(S, ar, br) + dot(S, ai, bi), dot(S, ar, bi) - dot(S, ai, br));
    } else if (idx < K * K + K) {
        const int a = idx - K * K;
        ColRef ar, ai;
        psi_column_refs(a, K, Bp, B, T, ar, ai);
        if (g) g[(size_t)p * K + a] = make_double2(dot(S, ar, tre) + dot(S, ai, tim), dot(S, ar, tim) - dot(S, ai, tre));
    } else if (idx == K * K + K) {
        if (tt) tt[p] = dot(S, tre, tre) + dot(S, tim, tim);
    }
}

cudaError_t launch_gram_assemble(const double *S, int nprob, int K, int Bp, int B, int T, double2 *G, double2 *g,
                                 double *tt, cudaStream_t s)
{
    dim3 grid((K * K + K + 1 + 255) / 256, nprob);
    gram_assemble_kernel<<<grid, 256, 0, s>>>(S, K, Bp, B, T, G, g, tt);
    count_launch();
    return cudaGetLastError();
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b)   // a * conj(b)
{
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// 1/sqrt(x) for a pivot x in (1e-30, 1e30): the FP32 hardware estimate refined
// by two Newton-Raphson steps y <- y (3 - x y^2) / 2 in FP64 (each step squares
// the relative error: about 2^-22 -> 2^-44 -> FP64 rounding).  Six FP64
// operations on the factorisation's sequential path instead of a full FP64
// square root and division.
__device__ __forceinline__ double rsqrt_newton(double x)
{
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double p = hx * y;
        const double e = fma(-p, y, 0.5);   // 1/2 - x y^2 / 2
        y = fma(y, e, y);
    }
    return y;
}

// Offset of row i in a lower triangle packed by rows (row i holds columns
// 0 .. i).  The batch kernels keep only that triangle in shared memory: 76 KB
// at K = 97 instead of 150 KB for the full matrix, so that two CTAs share an SM
// and a batch of more problems than SMs runs in one wave.
__device__ __forceinline__ int tri_row(int i) { return i * (i + 1) / 2; }

// One CTA per problem: A = D G D in shared memory (packed lower triangle),
// factored in place (right looking), written to L; d = diag(G)^{-1/2}.  On this GPU FP64
// runs at a small fraction of the FP32 rate (about two FMAs per clock per SM),
// so the K^3/6 complex updates of one problem (K = 97: 0.6 M FP64 FMAs) and the
// K sequential pivot steps bound the kernel: each complex update is four fused
// multiply-adds, and the pivot's reciprocal root comes from rsqrt_newton.  Step
// j: thread 0 takes the pivot; the threads scale column j; the trailing update
// of rows i > j, columns j < k <= i is split into equal contiguous runs of the
// triangle, one per thread.
__global__ void __launch_bounds__(256) chol_kernel(const double2 *__restrict__ Gall, int K,
                                                   double2 *__restrict__ Lall, double *__restrict__ dall,
                                                   int *__restrict__ info)
{
    extern __shared__ double2 A[];   // lower triangle of K x K, packed by rows (tri_row)
    __shared__ double dsh[kMaxT * 12 + 1];
    __shared__ double rinv;
    __shared__ int bad;
    const int p = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 15, ty = tid >> 4, nty = nt >> 4;
    const double2 *G = Gall + (size_t)p * K * K;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int i = tid; i < K; i += nt) {
        const double gii = G[(size_t)i * K + i].x;
        dsh[i] = gii > 0.0 ? 1.0 / sqrt(gii) : 0.0;
        if (!(gii > 0.0)) atomicMax(&bad, i + 1);
    }
    __syncthreads();
    for (int i = ty; i < K; i += nty)
        for (int k = tx; k <= i; k += 16) {
            const double2 v = G[(size_t)i * K + k];
            const double sc = dsh[i] * dsh[k];
            A[tri_row(i) + k] = make_double2(v.x * sc, v.y * sc);
        }
    __syncthreads();
    for (int j = 0; j < K && !bad; ++j) {
        if (tid == 0) {
            const double piv = A[tri_row(j) + j].x;
            if (!(piv > 1e-30 && piv < 1e30)) {   // not positive definite (or numerically singular)
                bad = j + 1;
            } else {
                const double ri = rsqrt_newton(piv);
                A[tri_row(j) + j] = make_double2(piv * ri, 0.0);
                rinv = ri;
            }
        }
        __syncthreads();
        if (bad) break;
        const double ri = rinv;
        for (int i = j + 1 + tid; i < K; i += nt) {
            const double2 v = A[tri_row(i) + j];
            A[tri_row(i) + j] = make_double2(v.x * ri, v.y * ri);
        }
        __syncthreads();
        // A[i][k] -= L[i][j] conj(L[k][j]) over the m (m + 1) / 2 elements of the
        // trailing lower triangle, row-major, each thread a contiguous run of
        // them: every lane of a warp stays busy (an FP64 warp instruction costs
        // the FP64 unit the same time however many lanes it has).
        {
            const int m = K - j - 1;
            const int tot = m * (m + 1) / 2;
            const int per = (tot + nt - 1) / nt;
            int e = tid * per;
            if (e < tot) {
                // row r of the triangle holding element e: r (r + 1) / 2 <= e < (r + 1) (r + 2) / 2
                int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while ((r + 1) * (r + 2) / 2 <= e) ++r;
                while (r * (r + 1) / 2 > e) --r;
                int c = e - r * (r + 1) / 2;
                const int end = min(e + per, tot);
                int i = j + 1 + r, k = j + 1 + c;
                int ib = tri_row(i), kb = tri_row(k);   // packed offsets of rows i and k
                double2 a = A[ib + j];
                for (; e < end; ++e) {
                    const double2 b = A[kb + j];
                    double2 &cc = A[ib + k];
                    cc.x = fma(-a.x, b.x, fma(-a.y, b.y, cc.x));
                    cc.y = fma(-a.y, b.x, fma(a.x, b.y, cc.y));
                    if (++c > r) {   // next row of the triangle
                        c = 0;
                        ++r;
                        ++i;
                        ib += i;   // tri_row(i) = tri_row(i - 1) + i
                        k = j + 1;
                        kb = tri_row(k);
                        if (i < K) a = A[ib + j];
                    } else {
                        ++k;
                        kb += k;
                    }
                }
            }
        }
        __syncthreads();
    }
    double2 *L = Lall + (size_t)p * K * K;
    for (int e = tid; e < K * K; e += nt) {
        const int i = e / K, k = e % K;
        L[e] = k <= i ? A[tri_row(i) + k] : make_double2(0.0, 0.0);
    }
    for (int i = tid; i < K; i += nt) dall[(size_t)p * K + i] = dsh[i];
    if (tid == 0) info[p] = bad;
}

// The same factorisation spread over a cluster of kCholCluster CTAs (one SM
// each), for few problems: one CTA per problem leaves all but a few SMs idle
// and is bound by one SM's FP64 rate.  Columns are dealt out cyclically (CTA r
// owns columns k = r, r + C, ...; its rows i >= k in shared memory).  Step j:
// every CTA updates its own columns k > j with column j, which its owner
// wrote, with the pivot status, into every CTA's shared buffer pc[j % 3]
// (distributed shared memory) before the cluster barrier that ended step
// j - 1.  Look-ahead: the owner of column j + 1 first updates that column
// alone, takes its pivot, scales it and sends it into pc[(j + 1) % 3], then
// arrives on the barrier and only then updates its other columns, so the next
// step waits for the column's pivot chain, not for its owner's other updates.
// The barrier is split (arrive, work, wait); the owner's later reads of
// pc[j % 3] end before it arrives in step j + 1, and that buffer is written
// again (column j + 3) only after the barrier of step j + 1: three buffers
// make the deferral safe.  Every CTA reads the same pivot status after the
// same barrier, so all of them leave the loop at the same step and pass the
// same number of barriers.
// (Measured on GB300, K = 97: 3,750 cycles per column with one barrier per
// step after all updates; the owner's chain was the critical path.)
// Split cluster barrier: every thread of every CTA arrives (release: its
// earlier shared-memory writes, local and remote, are visible to the cluster
// once the phase completes), then waits (acquire).
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

constexpr int kCholCluster = 8;
constexpr int kCholClusterThreads = 256;
constexpr int kCholMaxK = 2 * kMaxB * kMaxT + 1;   // 97: P = Q = 11, M = 7

__global__ void __launch_bounds__(kCholClusterThreads) chol_cluster_kernel(const double2 *__restrict__ Gall, int K,
                                                                            double2 *__restrict__ Lall,
                                                                            double *__restrict__ dall,
                                                                            int *__restrict__ info)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int C = kCholCluster;
    extern __shared__ double2 A[];            // [K][ncl]: this CTA's columns
    __shared__ double2 pc[3][kCholMaxK];      // broadcast pivot columns
    __shared__ int pbad[3];                   // their pivot status (0 or failing column + 1)
    __shared__ double dsh[kCholMaxK];
    __shared__ double rinv;
    const int rank = (int)cluster.block_rank();
    const int p = blockIdx.x / C, tid = threadIdx.x, nt = blockDim.x;
    const int ncl = (K + C - 1) / C;          // local columns (the last may be short)
    const double2 *G = Gall + (size_t)p * K * K;
    // Equilibration, computed by every CTA (the same values everywhere).
    int bad0 = 0;
    for (int i = 0; i < K; ++i) {
        const double gii = G[(size_t)i * K + i].x;
        if (!(gii > 0.0) && bad0 == 0) bad0 = i + 1;
    }
    for (int i = tid; i < K; i += nt) {
        const double gii = G[(size_t)i * K + i].x;
        dsh[i] = gii > 0.0 ? 1.0 / sqrt(gii) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < K * ncl; e += nt) {
        const int i = e / ncl, lc = e % ncl, k = rank + lc * C;
        double2 v = make_double2(0.0, 0.0);
        if (k < K && i >= k) {
            const double2 g = G[(size_t)i * K + k];
            const double sc = dsh[i] * dsh[k];
            v = make_double2(g.x * sc, g.y * sc);
        }
        A[(size_t)i * ncl + lc] = v;
    }
    __syncthreads();

    // Pivot of local column lc (global k), by thread 0: the scaled diagonal,
    // 1/sqrt(pivot) in rinv and the status in sbad (shared).
    __shared__ int sbad;
    auto pivot = [&](int k, int lc) {
        const double piv = A[(size_t)k * ncl + lc].x;
        if (!(piv > 1e-30 && piv < 1e30)) {
            sbad = k + 1;
            rinv = 0.0;
        } else {
            const double ri = rsqrt_newton(piv);
            A[(size_t)k * ncl + lc] = make_double2(piv * ri, 0.0);
            rinv = ri;
            sbad = 0;
        }
    };
    // After the pivot and a CTA barrier: status and column (rows below the
    // pivot scaled, in one pass) into every CTA's buffer b.
    auto send = [&](int k, int lc, int b) {
        if (tid < C) *cluster.map_shared_rank(&pbad[b], tid) = sbad;
        const double ri = rinv;
        for (int i = k + tid; i < K; i += nt) {
            double2 v = A[(size_t)i * ncl + lc];
            if (i > k) {
                v = make_double2(v.x * ri, v.y * ri);
                A[(size_t)i * ncl + lc] = v;
            }
#pragma unroll
            for (int r = 0; r < C; ++r) *cluster.map_shared_rank(&pc[b][i], r) = v;
        }
    };
    // A[i][k] -= pc[i] conj(pc[k]) for rows i >= k of one local column.
    auto update_col = [&](const double2 *col, int k, int lc, int first_row, int stride) {
        const double2 b = col[k];
        for (int i = k + first_row; i < K; i += stride) {
            const double2 a = col[i];
            double2 &cc = A[(size_t)i * ncl + lc];
            cc.x = fma(-a.x, b.x, fma(-a.y, b.y, cc.x));
            cc.y = fma(-a.y, b.x, fma(a.x, b.y, cc.y));
        }
    };

    int bad = bad0;
    if (bad == 0 && rank == 0) {
        if (tid == 0) pivot(0, 0);
        __syncthreads();
        send(0, 0, 0);
    }
    cluster.sync();
    for (int j = 0; j < K && bad == 0; ++j) {
        const int b = j % 3;
        if (pbad[b]) {   // the same value in every CTA after the same barrier
            bad = pbad[b];
            break;
        }
        const double2 *col = pc[b];
        const int next = j + 1;
        const bool own_next = next < K && next % C == rank;
        if (own_next) {   // look-ahead: column j + 1 first, then its pivot and broadcast
            update_col(col, next, next / C, tid, nt);   // thread 0 takes the diagonal row
            if (tid == 0) pivot(next, next / C);        // while the other rows are updated
            __syncthreads();
            send(next, next / C, next % 3);
            cluster_arrive();   // column j + 1 is out
        }
        // The rest of this CTA's columns k > j: (local column, row) pairs dealt
        // to the threads, columns in order.
        const int lc0 = (j + 1 - rank + C - 1) / C + (own_next ? 1 : 0);   // first local column with k > j (after next)
        for (int lc = lc0 + tid / 32; lc < ncl; lc += nt / 32) {
            const int k = rank + lc * C;
            if (k < K) update_col(col, k, lc, tid % 32, 32);
        }
        if (!own_next) cluster_arrive();
        cluster_wait();
    }
    cluster.sync();   // no CTA leaves while another may still write into its buffers

    double2 *L = Lall + (size_t)p * K * K;
    for (int e = tid; e < K * ncl; e += nt) {
        const int i = e / ncl, lc = e % ncl, k = rank + lc * C;
        if (k < K) L[(size_t)i * K + k] = i >= k ? A[(size_t)i * ncl + lc] : make_double2(0.0, 0.0);
    }
    if (rank == 0) {
        for (int i = tid; i < K; i += nt) dall[(size_t)p * K + i] = dsh[i];
        if (tid == 0) info[p] = bad;
    }
}

cudaError_t launch_chol(const double2 *G, int nprob, int K, double2 *L, double *d, int *info, cudaStream_t s)
{
    const size_t smem = sizeof(double2) * (size_t)K * (K + 1) / 2;   // packed lower triangle
    if (nprob * kCholCluster <= 64 && K <= kCholMaxK) {
        // Few problems: a cluster of CTAs per problem (see chol_cluster_kernel).
        const size_t csmem = sizeof(double2) * (size_t)K * ((K + kCholCluster - 1) / kCholCluster);
        static SmemAttr csmem_rec;
        cudaError_t e = ensure_smem(csmem_rec, (const void *)chol_cluster_kernel, csmem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nprob * kCholCluster));
        cfg.blockDim = dim3(kCholClusterThreads);
        cfg.dynamicSmemBytes = csmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kCholCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, chol_cluster_kernel, G, K, L, d, info);
        count_launch();
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    static SmemAttr smem_rec;
    const cudaError_t e = ensure_smem(smem_rec, (const void *)chol_kernel, smem);
    if (e != cudaSuccess) return e;
    chol_kernel<<<nprob, 256, smem, s>>>(G, K, L, d, info);
    count_launch();
    return cudaGetLastError();
}

// One CTA per problem: G x = rhs with G = D^{-1} L L^H D^{-1}:
// x = D (L^H)^{-1} L^{-1} D rhs.  With L = U Lambda (U unit lower triangular,
// Lambda = diag(L)): y = U^{-1} (D rhs), z = Lambda^{-2} y, v = U^{-H} z, x = D v,
// so the sequential steps carry no division or scaling.  The CTA stages U
// (the columns of L divided by their diagonal) in shared memory and solves in
// blocks of 32 rows: a diagonal block is one warp's sequential part (element
// b0 + l on lane l; each step broadcasts one finished element and the later
// lanes take a complex FMA -- two dependent FP64 FMAs, the latency that bounds
// the solve on this GPU, where a dependent FP64 FMA takes 64 cycles); the
// update of the remaining rows is a block matrix-vector product spread over the
// CTA (8 threads per row).
constexpr int kSolveNB = 32;

__global__ void __launch_bounds__(256) chol_solve_kernel(const double2 *__restrict__ Lall,
                                                         const double *__restrict__ dall,
                                                         const int *__restrict__ info,
                                                         const double2 *__restrict__ rhs, int K,
                                                         double2 *__restrict__ h, int accumulate)
{
    extern __shared__ double2 Us[];   // U = L Lambda^{-1}, lower triangle packed by rows (tri_row)
    __shared__ double inv[12 * kMaxT + 1];
    __shared__ double2 wv[12 * kMaxT + 1];
    const int p = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int sub = tid & 7, grp = tid >> 3, ngrp = nt >> 3;   // 8 threads per row in the updates
    if (info[p] != 0) return;   // uniform over the CTA
    const double2 *L = Lall + (size_t)p * K * K;
    const double *d = dall + (size_t)p * K;
    const double2 *b = rhs + (size_t)p * K;
    for (int i = tid; i < K; i += nt) {
        inv[i] = 1.0 / L[(size_t)i * K + i].x;
        wv[i] = make_double2(b[i].x * d[i], b[i].y * d[i]);
    }
    __syncthreads();
    for (int i = warp; i < K; i += nt / 32)
        for (int k = lane; k <= i; k += 32) {
            const double2 l = L[(size_t)i * K + k];
            Us[tri_row(i) + k] = k < i ? make_double2(l.x * inv[k], l.y * inv[k]) : make_double2(0.0, 0.0);
        }
    __syncthreads();

    // forward: U y = D b
    for (int b0 = 0; b0 < K; b0 += kSolveNB) {
        const int nb = min(kSolveNB, K - b0);
        if (warp == 0) {
            double2 v = lane < nb ? wv[b0 + lane] : make_double2(0.0, 0.0);
            for (int i = 0; i < nb; ++i) {
                const double2 vi = make_double2(__shfl_sync(0xffffffffu, v.x, i), __shfl_sync(0xffffffffu, v.y, i));
                if (lane > i && lane < nb) {   // v -= U[b0+lane][b0+i] vi
                    const double2 u = Us[tri_row(b0 + lane) + b0 + i];
                    v.x = fma(-u.x, vi.x, fma(u.y, vi.y, v.x));
                    v.y = fma(-u.x, vi.y, fma(-u.y, vi.x, v.y));
                }
            }
            if (lane < nb) wv[b0 + lane] = v;
        }
        __syncthreads();
        for (int r0 = b0 + nb; r0 < K; r0 += ngrp) {   // rows below: y_r -= U[r][block] y[block]
            const int r = r0 + grp;
            double2 acc = make_double2(0.0, 0.0);
            if (r < K)
                for (int c = sub; c < nb; c += 8) {
                    const double2 u = Us[tri_row(r) + b0 + c], v = wv[b0 + c];
                    acc.x = fma(u.x, v.x, fma(-u.y, v.y, acc.x));
                    acc.y = fma(u.x, v.y, fma(u.y, v.x, acc.y));
                }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (r < K && sub == 0) wv[r] = make_double2(wv[r].x - acc.x, wv[r].y - acc.y);
        }
        __syncthreads();
    }
    for (int i = tid; i < K; i += nt) {   // z = Lambda^{-2} y
        const double s = inv[i] * inv[i];
        wv[i] = make_double2(wv[i].x * s, wv[i].y * s);
    }
    __syncthreads();
    // backward: U^H v = z
    for (int b0 = ((K - 1) / kSolveNB) * kSolveNB; b0 >= 0; b0 -= kSolveNB) {
        const int nb = min(kSolveNB, K - b0);
        if (warp == 0) {
            double2 v = lane < nb ? wv[b0 + lane] : make_double2(0.0, 0.0);
            for (int i = nb - 1; i >= 0; --i) {
                const double2 vi = make_double2(__shfl_sync(0xffffffffu, v.x, i), __shfl_sync(0xffffffffu, v.y, i));
                if (lane < i) {   // v -= conj(U[b0+i][b0+lane]) vi
                    const double2 u = Us[tri_row(b0 + i) + b0 + lane];
                    v.x = fma(-u.x, vi.x, fma(-u.y, vi.y, v.x));
                    v.y = fma(-u.x, vi.y, fma(u.y, vi.x, v.y));
                }
            }
            if (lane < nb) wv[b0 + lane] = v;
        }
        __syncthreads();
        for (int r0 = 0; r0 < b0; r0 += ngrp) {   // rows above: v_r -= sum_c conj(U[b0+c][r]) v[b0+c]
            const int r = r0 + grp;
            double2 acc = make_double2(0.0, 0.0);
            if (r < b0)
                for (int c = sub; c < nb; c += 8) {
                    const double2 u = Us[tri_row(b0 + c) + r], v = wv[b0 + c];
                    acc.x = fma(u.x, v.x, fma(u.y, v.y, acc.x));
                    acc.y = fma(u.x, v.y, fma(-u.y, v.x, acc.y));
                }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (r < b0 && sub == 0) wv[r] = make_double2(wv[r].x - acc.x, wv[r].y - acc.y);
        }
        __syncthreads();
    }
    double2 *out = h + (size_t)p * K;
    for (int k = tid; k < K; k += nt) {
        const double2 x = make_double2(wv[k].x * d[k], wv[k].y * d[k]);
        if (accumulate)
            out[k] = make_double2(out[k].x + x.x, out[k].y + x.y);
        else
            out[k] = x;
    }
}

cudaError_t launch_chol_solve(const double2 *L, const double *d, const int *info, const double2 *rhs, int nprob,
                              int K, double2 *h, int accumulate, cudaStream_t s)
{
    const size_t smem = sizeof(double2) * (size_t)K * (K + 1) / 2;   // packed lower triangle
    static SmemAttr smem_rec;
    const cudaError_t e = ensure_smem(smem_rec, (const void *)chol_solve_kernel, smem);
    if (e != cudaSuccess) return e;
    chol_solve_kernel<<<nprob, 256, smem, s>>>(L, d, info, rhs, K, h, accumulate);
    count_launch();
    return cudaGetLastError();
}

// Column j of L^{-1} per CTA: L x = e_j by column-oriented forward
// substitution.  The CTA first stages the strictly lower triangle of the
// trailing block L[j:, j:] in shared memory (packed by rows); thread t then
// owns row j + t.  Step k: the thread of row k finishes x_k = r_k / L_kk and
// publishes it, and after one barrier every thread of a row i > k subtracts
// L_ik x_k.  The rows are spread over four warps, so the FP64 updates of a
// step (about 2 fused multiply-adds per clock per SM on this GPU, i.e. one
// warp instruction per 64 clocks in each SM sub-partition) run on all four
// sub-partitions instead of one.  The columns are independent, so the K CTAs
// spread the inverse (K^3/6 complex updates) over as many SMs; column 0, the
// longest, bounds the kernel.
constexpr int kInvThreads = 128;   // one row per thread: K <= 128

__global__ void __launch_bounds__(kInvThreads) chol_invert_kernel(const double2 *__restrict__ L,
                                                                  const int *__restrict__ info, int K,
                                                                  double2 *__restrict__ Linv)
{
    extern __shared__ double2 tri[];   // row i' (i' = i - j) of L[j:, j:] at i'(i'-1)/2, i' entries; then x
    if (info[0] != 0) return;
    const int j = blockIdx.x, tid = threadIdx.x;
    const int m_ = K - j;
    double2 *xs = tri + (size_t)m_ * (m_ - 1) / 2;   // x_k, published at step k
    for (int e = tid; e < m_ * (m_ - 1) / 2; e += kInvThreads) {
        int ip = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);   // row of packed element e
        while (ip * (ip - 1) / 2 > e) --ip;
        while ((ip + 1) * ip / 2 <= e) ++ip;
        const int kp = e - ip * (ip - 1) / 2;
        tri[e] = L[(size_t)(j + ip) * K + j + kp];
    }
    const bool mine = tid < m_;
    double2 r = make_double2(tid == 0 ? 1.0 : 0.0, 0.0);
    const double inv_own = mine ? 1.0 / L[(size_t)(j + tid) * K + j + tid].x : 0.0;
    const double2 *lrow = tri + (size_t)tid * (tid - 1) / 2;   // row tid of the staged triangle
    __syncthreads();
    for (int kp = 0; kp < m_; ++kp) {
        if (tid == kp) {   // row k is final: x_k = r_k / L_kk (real diagonal)
            r = make_double2(r.x * inv_own, r.y * inv_own);
            xs[kp] = r;
        }
        __syncthreads();
        if (mine && tid > kp) {
            const double2 l = lrow[kp], xk = xs[kp];
            r.x = fma(-l.x, xk.x, fma(l.y, xk.y, r.x));
            r.y = fma(-l.x, xk.y, fma(-l.y, xk.x, r.y));
        }
    }
    if (mine) Linv[(size_t)(j + tid) * K + j] = r;   // column j, rows >= j
    for (int i = tid; i < j; i += kInvThreads) Linv[(size_t)i * K + j] = make_double2(0.0, 0.0);
}

// One warp per output element: tmp_i = sum_{k <= i} Linv[i][k] d_k rhs_k
// (lower) or h_k (+)= d_k sum_{i >= k} conj(Linv[i][k]) tmp_i (upper).
__global__ void __launch_bounds__(128) inv_matvec_kernel(const double2 *__restrict__ Linv,
                                                         const double *__restrict__ d, const int *__restrict__ info,
                                                         const double2 *__restrict__ v, int K, int upper,
                                                         double2 *__restrict__ out, int accumulate)
{
    if (info[0] != 0) return;
    const int row = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= K) return;
    double2 acc = make_double2(0.0, 0.0);
    if (!upper) {
        for (int k = lane; k <= row; k += 32) {
            const double2 l = Linv[(size_t)row * K + k];
            const double2 b = make_double2(v[k].x * d[k], v[k].y * d[k]);
            acc.x = fma(l.x, b.x, fma(-l.y, b.y, acc.x));
            acc.y = fma(l.x, b.y, fma(l.y, b.x, acc.y));
        }
    } else {
        for (int i = row + lane; i < K; i += 32) {
            const double2 l = Linv[(size_t)i * K + row];
            const double2 b = v[i];
            acc.x = fma(l.x, b.x, fma(l.y, b.y, acc.x));
            acc.y = fma(l.x, b.y, fma(-l.y, b.x, acc.y));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
        if (upper) {
            acc = make_double2(acc.x * d[row], acc.y * d[row]);
            if (accumulate) acc = make_double2(out[row].x + acc.x, out[row].y + acc.y);
        }
        out[row] = acc;
    }
}

// Both products of a solve in one launch: a cluster of kSolveCluster CTAs,
// warp w of the cluster taking rows w, w + 64, ...  Phase 1: tmp_i =
// sum_{k <= i} Linv[i][k] d_k rhs_k, each finished element written into every
// CTA's copy of tmp (distributed shared memory); after the cluster barrier,
// phase 2: h_k (+)= d_k sum_{i >= k} conj(Linv[i][k]) tmp_i.  The same
// arithmetic and summation order per element as inv_matvec_kernel.
constexpr int kSolveCluster = 8;
constexpr int kSolveThreads = 256;

__global__ void __launch_bounds__(kSolveThreads) solve_inverse_cluster_kernel(const double2 *__restrict__ Linv,
                                                                              const double *__restrict__ d,
                                                                              const int *__restrict__ info,
                                                                              const double2 *__restrict__ rhs, int K,
                                                                              double2 *__restrict__ h, int accumulate)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ double2 tmp[kCholMaxK];
    if (info[0] != 0) return;   // the same value for every CTA of the cluster: none reaches the barrier
    const int lane = threadIdx.x & 31;
    const int gw = (int)cluster.block_rank() * (kSolveThreads / 32) + (threadIdx.x >> 5);
    constexpr int NW = kSolveCluster * (kSolveThreads / 32);
    for (int row = gw; row < K; row += NW) {
        double2 acc = make_double2(0.0, 0.0);
        for (int k = lane; k <= row; k += 32) {
            const double2 l = Linv[(size_t)row * K + k];
            const double2 b = make_double2(rhs[k].x * d[k], rhs[k].y * d[k]);
            acc.x = fma(l.x, b.x, fma(-l.y, b.y, acc.x));
            acc.y = fma(l.x, b.y, fma(l.y, b.x, acc.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane < kSolveCluster) *cluster.map_shared_rank(&tmp[row], lane) = acc;
    }
    cluster.sync();
    for (int row = gw; row < K; row += NW) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = row + lane; i < K; i += 32) {
            const double2 l = Linv[(size_t)i * K + row];
            const double2 b = tmp[i];
            acc.x = fma(l.x, b.x, fma(l.y, b.y, acc.x));
            acc.y = fma(l.x, b.y, fma(-l.y, b.x, acc.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            acc = make_double2(acc.x * d[row], acc.y * d[row]);
            if (accumulate) acc = make_double2(h[row].x + acc.x, h[row].y + acc.y);
            h[row] = acc;
        }
    }
}

cudaError_t launch_chol_invert(const double2 *L, const int *info, int K, double2 *Linv, cudaStream_t s)
{
    if (K > kInvThreads) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double2) * ((size_t)K * (K - 1) / 2 + (size_t)K);
    static SmemAttr smem_rec;
    const cudaError_t e = ensure_smem(smem_rec, (const void *)chol_invert_kernel, smem > 0 ? smem : 16);
    if (e != cudaSuccess) return e;
    chol_invert_kernel<<<K, kInvThreads, smem > 0 ? smem : 16, s>>>(L, info, K, Linv);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_solve_inverse(const double2 *Linv, const double *d, const int *info, const double2 *rhs, int K,
                                 double2 *tmp, double2 *h, int accumulate, cudaStream_t s)
{
    const int grid = (K + 3) / 4;
    if (K <= kCholMaxK) {   // one cluster launch (see solve_inverse_cluster_kernel)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kSolveCluster);
        cfg.blockDim = dim3(kSolveThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kSolveCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, solve_inverse_cluster_kernel, Linv, d, info, rhs, K, h,
                                                 accumulate);
        count_launch();
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    inv_matvec_kernel<<<grid, 128, 0, s>>>(Linv, d, info, rhs, K, 0, tmp, 0);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    inv_matvec_kernel<<<grid, 128, 0, s>>>(Linv, d, info, tmp, K, 1, h, accumulate);
    count_launch();
    return cudaGetLastError();
}

__global__ void h_to_f32_kernel(const double2 *__restrict__ h, int n, float2 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)h[i].x, (float)h[i].y);
}

cudaError_t launch_h_to_f32(const double2 *h, int n, float2 *out, cudaStream_t s)
{
    h_to_f32_kernel<<<(n + 127) / 128, 128, 0, s>>>(h, n, out);
    count_launch();
    return cudaGetLastError();
}

__global__ void residual_kernel(const float2 *__restrict__ t, const float2 *__restrict__ y, int64_t n,
                                float2 *__restrict__ e)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = t[i], b = y[i];
        e[i] = make_float2(a.x - b.x, a.y - b.y);
    }
}

cudaError_t launch_residual(const float2 *t, const float2 *y, int64_t n, float2 *e, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) return cudaSuccess;
    residual_kernel<<<(unsigned)blocks, 256, 0, s>>>(t, y, n, e);
    count_launch();
    return cudaGetLastError();
}

constexpr int kNormBlocks = 1024;
static_assert(kNormBlocks <= kFwdNormSlots, "partial pairs of the statistics pass");

__global__ void sum_pairs_kernel(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    __shared__ double sa[256], sb[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sa[threadIdx.x] += sa[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sa[0];
        out[1] = sb[0];
    }
}

// Residual and both sums of squares in one pass: e = t - y (when e is not
// null), and per block sum |e|^2 and sum |t|^2, then one fixed-order final sum
// (sum_pairs_kernel).  The squares of the FP32 samples are formed and summed
// in FP32 over the four samples of a pass, and the passes are added in FP64
// (FP64 arithmetic on this GPU is a small fraction of the FP32 rate).
__global__ void residual_norm_kernel(const float2 *__restrict__ t, const float2 *__restrict__ y, int64_t n,
                                     float2 *__restrict__ e, double *__restrict__ part)
{
    // Four samples per thread and pass (all loads issued before any use);
    // e is written only when requested.
    __shared__ double se[256], st[256];
    double a = 0.0, b = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        float2 tv[4], yv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q * stride;
            tv[q] = i < n ? t[i] : make_float2(0.f, 0.f);
            yv[q] = i < n ? y[i] : make_float2(0.f, 0.f);
        }
        float a32 = 0.f, b32 = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 ev = make_float2(tv[q].x - yv[q].x, tv[q].y - yv[q].y);
            const int64_t i = i0 + q * stride;
            if (e && i < n) e[i] = ev;
            a32 = fmaf(ev.x, ev.x, fmaf(ev.y, ev.y, a32));
            b32 = fmaf(tv[q].x, tv[q].x, fmaf(tv[q].y, tv[q].y, b32));
        }
        a += (double)a32;
        b += (double)b32;
    }
    se[threadIdx.x] = a;
    st[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            se[threadIdx.x] += se[threadIdx.x + o];
            st[threadIdx.x] += st[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = se[0];
        part[2 * blockIdx.x + 1] = st[0];
    }
}

cudaError_t launch_residual_norm(const float2 *t, const float2 *y, int64_t n, float2 *e, double *part, double *out,
                                 cudaStream_t s)
{
    residual_norm_kernel<<<kNormBlocks, 256, 0, s>>>(t, y, n, e, part);
    count_launch();
    sum_pairs_kernel<<<1, 256, 0, s>>>(part, kNormBlocks, out);
    count_launch();
    return cudaGetLastError();
}


}  // namespace dpd
