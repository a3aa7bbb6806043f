// Internal declarations of libdpd shared by the host API and the kernel
// translation units.  Not part of the public C ABI (include/dpd.h).
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

namespace dpd {

// Bits of the per-handle device error word.
enum : int {
    kFlagTimeout = 1,   // a barrier wait inside a kernel exceeded its time limit
    kFlagBadWork = 2,   // a work descriptor failed a device-side range check
};

constexpr int kMaxB = 6;       // (P+1)/2 for P <= 11
constexpr int kMaxT = 8;       // M + 1 <= 8
constexpr int kHalo = 8;       // samples of history staged in front of a tile (>= kMaxT - 1, 16-byte multiple)

// Size in floats of the widely-linear coefficient table consumed by the
// forward kernels.  Four real polynomials in r = |x|^2 per tap k,
//   P0 = Re(A+C), P1 = -Im(A-C), P2 = Im(A+C), P3 = Re(A-C),
// where A_k(r) = sum_b h_{2b+1,k} r^b and C_k(r) = sum_b hbar_{2b+1,k} r^b, so that
// A_k(r) x + C_k(r) conj(x) = (P0 a + P1 b) + j (P2 a + P3 b) for x = a + j b.
// Layout: tab[(k*B + m)*4 + {0,1,2,3}] = {P0, P2, P1, P3} coefficient of r^m
// (so {P0,P2} and {P1,P3} are adjacent pairs), then Re c, Im c at 4*B*T.
__host__ __device__ constexpr int wl_table_floats(int B, int T) { return 4 * B * T + 2; }
__host__ __device__ constexpr int wl_index(int B, int k, int m, int poly)
{
    return (k * B + m) * 4 + (poly == 0 ? 0 : poly == 2 ? 1 : poly == 1 ? 2 : 3);
}

// Largest table that is passed by value as a kernel parameter (B = 6, T = 8).
constexpr int kMaxTabFloats = 4 * 6 * 8 + 2;
struct HostTab {
    float v[kMaxTabFloats];
};

// Forward compute modes (template bits): coefficients read from the kernel
// parameter bank instead of shared memory; packed f32x2 fused multiply-adds.
// kModeSubtract (internal, least-squares refinement only): the kernel writes
// sub[n] - y[n] instead of y[n].  kModeNorms (with kModeSubtract, internal:
// the statistics of an estimate) writes nothing per sample: it sums
// |sub - y|^2 and |sub|^2 instead (FwdArgs::norms).
enum : int { kModeParamCoef = 1, kModePackedFma = 2, kModeSubtract = 4, kModeNorms = 8 };

// Partial-sum slots of kModeNorms: one pair per CTA of the grid.
constexpr int kFwdNormSlots = 4096;

// Forward launch shape.
constexpr int kFwdMaxWarps = 16;   // consumer warps per CTA of the TMA kernel (register budget)

struct FwdLaunch {
    int mode = kModeParamCoef | kModePackedFma;   // compute mode bits
    int V = 8;            // samples per consumer thread (2, 4, 6 or 8)
    int warps = 16;       // consumer warps per CTA (tile = warps * 32 * V samples)
    int stages = 4;       // shared-memory ring depth per group (bulk-copy pipeline)
    int ctas_per_sm = 0;  // 0: as many as fit
    int use_tma = 1;      // 0: plain global loads (also used for 8-byte aligned buffers)
    int group = 4;        // warps per group (own ring and barriers); 0: one group of all warps
};

struct FwdArgs {
    const float2 *x;
    float2 *y;
    int64_t n;
    const float *tab;     // device widely-linear table, wl_table_floats(B, T) floats
    int *status;          // device error word
    int vec_store;        // y is 16-byte aligned
    const HostTab *host_tab;   // host copy of the table (param-bank modes), or null
    const float2 *sub = nullptr;   // kModeSubtract: minuend, n samples, 16-byte aligned
    // kModeNorms: kFwdNormSlots partial sums (one float4 per CTA: the FP32
    // (hi, lo) pairs of both sums, the size of two doubles), then the two
    // results in FP64 (sum |sub - y|^2, sum |sub|^2), then a completion counter
    // (an unsigned in the next double; zero between launches).  The last CTA to
    // finish adds the partials in a fixed order, writes the results and clears
    // the counter.
    double *norms = nullptr;
};

// Floats of the adjoint table: per tap, four polynomials of B coefficients
// (Q0..Q3 for conj(E) g + H conj(g)) and four of B-1 (S0..S3 for
// conj(G) g + F conj(g)), stored power-major as quadruples {Q0, Q3, Q1, Q2}
// then {S0, S3, S1, S2}; see dpd_adj.cuh.
__host__ __device__ constexpr int adj_table_floats(int B, int T) { return (4 * B + 4 * (B - 1)) * T; }
constexpr int kMaxAdjTabFloats = adj_table_floats(6, 8);   // 352

struct AdjArgs {
    const float2 *x;
    const float2 *gy;
    int64_t n;
    float2 *gx;             // nullable: input gradient (n)
    float2 *partials;       // nullable: per-CTA coefficient-gradient rows (rows x K)
    const float *adj_tab;   // device adjoint table
    int *status;
    // Host copy of the adjoint table (coefficients set from host memory), or
    // null: when present the input-gradient kernel takes its coefficients from
    // the kernel parameter bank.
    const float *host_adj_tab = nullptr;
};

struct AdjLaunch {
    int gh_blocks = 0;      // CTAs per tap group for the coefficient gradient (rows of partials)
    int tap_group = 2;      // taps per group: 1 .. 5
};

template <int B>
cudaError_t launch_adj(const AdjArgs &a, const AdjLaunch &L, int T, int Bp, int Bq, int K, int sm_count,
                       cudaStream_t s);
// Coefficient gradients of `count` independent problems in one launch (staged
// kernel; args[z] on the device, 16-byte aligned x and gy, one partials row
// per CTA of each problem).
template <int B>
cudaError_t launch_adj_gh_many(const AdjArgs *args, int count, int blocks, int tap_group, int T, int Bp, int Bq,
                               int K, cudaStream_t s);
cudaError_t launch_adj_gh_many_any(int B, const AdjArgs *args, int count, int blocks, int tap_group, int T, int Bp,
                                   int Bq, int K, cudaStream_t s);
cudaError_t launch_adj_any(int B, const AdjArgs &a, const AdjLaunch &L, int T, int Bp, int Bq, int K,
                           int sm_count, cudaStream_t s);
// gh[i] = sum over `rows` rows of partials[row * K + i], accumulated in FP64 in row order.
cudaError_t launch_adj_finalize(const float2 *partials, int rows, int K, float2 *gh, cudaStream_t s);

// Launch the forward filter for max branch count B and T taps (host side;
// defined per B in fwd_b<B>.cu).  Returns the launch error.
template <int B>
cudaError_t launch_fwd(int T, const FwdArgs &a, const FwdLaunch &L, int sm_count, cudaStream_t s);

cudaError_t launch_fwd_any(int B, int T, const FwdArgs &a, const FwdLaunch &L, int sm_count,
                           cudaStream_t s);

// Build the forward widely-linear table and the adjoint table from the stacked
// coefficient vector h (K complex); adj_tab may be null.
// The forward table straight from FP64 coefficients (rounded to FP32 first);
// _many: `count` problems, coefficients hstride and tables tstride apart.
cudaError_t launch_wl_table_f64(const double2 *h, int Bp, int Bq, int T, float *tab, cudaStream_t s);
cudaError_t launch_wl_table_f64_many(const double2 *h, int count, int hstride, int Bp, int Bq, int T, float *tab,
                                     int tstride, cudaStream_t s);
cudaError_t launch_wl_table(const float2 *h, int Bp, int Bq, int T, float *tab, float *adj_tab,
                            cudaStream_t s);

void count_launch(int n = 1);

// A kernel's dynamic shared-memory limit and its occupancy belong to each
// device, so the launchers keep them per device ordinal (one record per kernel
// instantiation); ordinals past kMaxDevices are served without a cache.
constexpr int kMaxDevices = 64;

struct SmemAttr {
    std::atomic<size_t> set[kMaxDevices] = {};
    std::mutex mu;
};

// Raise `kern`'s dynamic shared-memory limit on the current device to at least
// `bytes` (never lowers it).
inline cudaError_t ensure_smem(SmemAttr &rec, const void *kern, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (rec.set[dev].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
    std::lock_guard<std::mutex> lock(rec.mu);
    const size_t cur = rec.set[dev].load(std::memory_order_relaxed);
    if (cur >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) rec.set[dev].store(bytes, std::memory_order_release);
    return e;
}

// Resident CTAs per SM of `kern` at (threads, smem) on the current device,
// remembered per device for the last shape asked.
struct OccCache {
    struct Entry {
        int threads = -1;
        size_t smem = 0;
        int occ = 0;
    };
    Entry e[kMaxDevices];
    std::mutex mu;
};

inline cudaError_t occupancy(OccCache &c, const void *kern, int threads, size_t smem, int *occ)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, threads, smem);
    std::lock_guard<std::mutex> lock(c.mu);
    OccCache::Entry &en = c.e[dev];
    if (en.threads != threads || en.smem != smem) {
        int o = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem);
        if (err != cudaSuccess) return err;
        en.threads = threads;
        en.smem = smem;
        en.occ = o;
    }
    *occ = en.occ;
    return cudaSuccess;
}

}  // namespace dpd
