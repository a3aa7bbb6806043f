// Gram contraction S = X^T X of the distinct real columns of the basis (see
// dpd_gram.cuh): tcgen05 tensor-core kernel with split BF16 / TF32 operands,
// and the plain FP32 CUDA-core form it is compared against.
#include <cuda_bf16.h>

#include "dpd_gram.cuh"
#include "dpd_tc.cuh"

namespace dpd {

namespace {

// ------------------------------------------------------------------ the basis
// Every distinct column is one of 15 "series" -- Re / Im of psi_b(u_j) for
// b < 6, Re / Im of t, or the constant 1 -- read at stage row rr from element
// w = rr + off, off = T-1-k for a tap-k column and T-1 for the others.
// Element w of a stage is sample n0 - (T-1) + w.
constexpr int kSeries = 15;
constexpr int kSerT = 12;      // Re t = 12, Im t = 13
constexpr int kSerOne = 14;
constexpr int kSerLen = 72;    // elements per series (>= 64 + kMaxT - 1, even)
// Per series: BF16: hi, hi shifted by one, lo, lo shifted by one (16-bit each);
// TF32: hi, lo (32-bit each).  Both 4 * kSerLen * 2 bytes.
constexpr int kSerBytes = 4 * kSerLen * 2;
constexpr int kStagingBytes = kSeries * kSerBytes;
constexpr int kPsiStride = 64 + kMaxT - 1;

__device__ __forceinline__ void distinct_source(int d, int B, int T, int &series, int &off)
{
    const int BT = B * T;
    if (d < 2 * BT) {
        const int im = d >= BT ? 1 : 0, dd = im ? d - BT : d;
        series = 2 * (dd / T) + im;
        off = T - 1 - dd % T;
    } else {
        series = d == 2 * BT ? kSerOne : kSerT + (d - 2 * BT - 1);
        off = T - 1;
    }
}

// Series work of a stage is spread over the 512 threads: threads
// 0 .. 6 kSerLen - 1 own element w = tid % kSerLen of the psi series of order
// b = tid / kSerLen (Re and Im); threads 6 kSerLen .. 511 own target row
// rr = tid - 6 kSerLen (Re t, Im t and the constant).
constexpr int kPsiThreads = kMaxB * kSerLen;   // 432
static_assert(512 - kPsiThreads >= 64, "a target row per remaining thread");

// The raw samples of a stage (kSerLen basis samples from n0 - (T-1), then up
// to 64 target samples from n0) are fetched kAhead stages in advance with
// asynchronous 8-byte copies into a ring of shared-memory slots (zero-filled
// outside the problem), one copy group per stage and thread.
constexpr int kAhead = 3;
constexpr int kRawSlots = kAhead + 1;
constexpr int kRawLen = kSerLen + 64;

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// This thread's copies of the stage starting at row n0 into `slot`; `active`
// false commits an empty group (keeps the per-thread group count uniform).
template <int R>
__device__ __forceinline__ void fetch_stage(float2 *slot, const GramProblem &pr, int64_t n0, int T, bool active)
{
    const int tid = threadIdx.x;
    if (active) {
        if (tid < kSerLen) {
            const int64_t j = n0 - (T - 1) + tid;
            const bool v = tid < R + T - 1 && j >= 0 && j < pr.n;
            cp_async8(smem_addr(slot + tid), v ? pr.u + j : pr.u, v ? 8u : 0u);
        } else if (tid >= kPsiThreads && tid - kPsiThreads < R) {
            const int r = tid - kPsiThreads;
            const int64_t j = n0 + r;
            const bool v = pr.t != nullptr && j < pr.n;
            cp_async8(smem_addr(slot + kSerLen + r), v ? pr.t + j : pr.u, v ? 8u : 0u);
        }
    }
    cp_async_commit();
}

template <int FMT>
__device__ __forceinline__ void put_series(unsigned char *stg, int series, int w, float v)
{
    unsigned char *base = stg + series * kSerBytes;
    if constexpr (FMT == kFmtBF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        uint16_t *hi0 = reinterpret_cast<uint16_t *>(base);   // element i at i
        uint16_t *hi1 = hi0 + kSerLen;                         // element i at i - 1
        uint16_t *lo0 = hi0 + 2 * kSerLen;
        uint16_t *lo1 = hi0 + 3 * kSerLen;
        const uint16_t hb = *reinterpret_cast<const uint16_t *>(&h), lb = *reinterpret_cast<const uint16_t *>(&l);
        hi0[w] = hb;
        lo0[w] = lb;
        if (w >= 1) {
            hi1[w - 1] = hb;
            lo1[w - 1] = lb;
        }
    } else {
        uint32_t *hi = reinterpret_cast<uint32_t *>(base);
        uint32_t *lo = hi + kSerLen;
        const float h = to_tf32(v);
        hi[w] = __float_as_uint(h);
        lo[w] = __float_as_uint(to_tf32(v - h));
    }
}

// Convert the raw samples of a stage (rows from n0) into the series arrays.
template <int FMT, int R>
__device__ __forceinline__ void stage_series(unsigned char *stg, const float2 *slot, int64_t n0, int64_t n, int B,
                                             int T, const float *su)
{
    const int tid = threadIdx.x;
    if (tid < kPsiThreads) {
        const int w = tid % kSerLen, b = tid / kSerLen;
        if (b < B) {
            const float2 u = slot[w];   // zero outside the problem
            const float r = fmaf(u.x, u.x, u.y * u.y);
            float p = 1.f;
            if (su) {   // sum_{a <= b} U[a][b] r^a by Horner's rule
                p = su[b * kMaxB + b];
                for (int a = b - 1; a >= 0; --a) p = fmaf(p, r, su[a * kMaxB + b]);
            } else {
                for (int e = 0; e < b; ++e) p *= r;   // r^b, low order first as in the filter
            }
            put_series<FMT>(stg, 2 * b, w, p * u.x);   // psi_b = |u|^{2b} u (or its combination)
            put_series<FMT>(stg, 2 * b + 1, w, p * u.y);
        }
    } else {
        const int rr = tid - kPsiThreads;
        if (rr < R) {
            const int w = rr + T - 1;
            const float2 t = slot[kSerLen + rr];
            put_series<FMT>(stg, kSerT, w, t.x);
            put_series<FMT>(stg, kSerT + 1, w, t.y);
            put_series<FMT>(stg, kSerOne, w, n0 + rr < n ? 1.f : 0.f);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ tensor cores
// Operand generation.  Each stage converts every basis value to its hi / lo
// pair once, into a series array in shared memory; an operand chunk (8 BF16 or
// 4 TF32 rows of one distinct column) is then four 32-bit shared loads per
// half and two 16-byte stores.  BF16 series are kept twice, as 16-bit arrays
// starting at element 0 and at element 1, so a chunk at any offset reads whole
// aligned words.  Every generator thread owns up to four fixed chunks (the
// addresses are computed once); the global loads of the next stage are issued
// before the current stage is generated.
//
// Products.  X = hi + lo; the split product hi^T hi + hi^T lo + lo^T hi is
// P + Q + Q^T with P = hi^T hi, Q = hi^T lo.  The hi and lo tiles of a stage
// are adjacent in shared memory, so one MMA with A = hi (128 operand rows) and
// B = [hi; lo] (256 rows) produces [P | Q] in a 128 x 256 accumulator: one
// MMA per K step (a tcgen05 MMA with M = 128 takes the same time for any N up
// to 256, so the full width is used).
//
// Accumulation.  The tensor core's FP32 accumulator drops low-order bits on
// every MMA step, a bias that grows with the number of steps summed into one
// accumulator.  So each accumulation covers a chunk of kChunk stages only and
// is then added, with round-to-nearest, into FP32 running sums in registers:
// every thread owns one tensor-memory lane (a distinct column) and one piece
// of its columns -- P [0, 64), P [64, 112), Q [128, 192) or Q [192, 240) --
// read as 64 columns with one wait (the 48-column pieces read 16 unused ones).  Two accumulators in tensor memory
// (2 x 256 columns) alternate between chunks, so the MMAs of one chunk run
// while the previous one is drained.
//
// Roles.  All sixteen warps generate operands and drain accumulators; thread 0
// also issues the MMAs of a stage once the barrier at the top of the next
// iteration has shown that every thread has written it.  Sixteen warps (four
// per SM sub-partition) at 128 registers each fill the register file.
constexpr int kThreads = 512;
constexpr int kOpTile = 16384;            // 128 operand rows x 128 bytes
constexpr int kStageBytes = 2 * kOpTile;  // hi tile, then lo tile
constexpr int kStages = 4;
constexpr int kChunk = 8;
// A chunk is drained kStages stages after its last one was generated, and its
// accumulator is reused by the chunk two later, whose first stage is issued
// kChunk + 1 stages after that last one.
static_assert(kStages <= kChunk + 1, "drain must precede the reuse of an accumulator");
constexpr int kAccN = 256;                // accumulator columns: P in [0, 128), Q in [128, 256)
constexpr int kAccPer = 64;               // sums per thread (a piece of 64 or 48 columns)
constexpr int kTasks = 2;                 // operand chunks per thread (8 D <= 792 <= 2 x 512)
constexpr int kTmemCols = 2 * kAccN;

// Barriers: empty[s] (MMA commit: stage s consumed), acc_full[b] (MMA commit:
// a chunk's sum is complete in accumulator b), fin (MMA commit: everything
// issued has completed, before tensor memory is released).
template <int FMT>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramArgs a)
{
    constexpr int R = (FMT == kFmtBF16) ? 64 : 32;   // rows per stage: 128 bytes per operand row
    constexpr int NK = 4;                            // MMAs along K per stage (K = 16 bf16 / 8 tf32)
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stages = smem;
    unsigned char *staging = smem + kStages * kStageBytes;   // 2 x kStagingBytes
    float2 *raw = reinterpret_cast<float2 *>(staging + 2 * kStagingBytes);   // kRawSlots x kRawLen
    uint64_t *empty = reinterpret_cast<uint64_t *>(raw + kRawSlots * kRawLen);
    uint64_t *acc_full = empty + kStages;
    uint64_t *fin = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    float *su_buf = reinterpret_cast<float *>(tmem_slot + 4);   // basis coefficients U (kUSize)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int prob = blockIdx.x / a.cpp, chunk = blockIdx.x % a.cpp;
    const GramProblem pr = a.probs[prob];
    const int T = a.T, B = a.Bp > a.Bq ? a.Bp : a.Bq;
    const int D = gram_distinct(B, T);
    const int64_t nblk = (pr.n + R - 1) / R;
    const int64_t b0 = nblk * chunk / a.cpp, b1 = nblk * (chunk + 1) / a.cpp;
    const int nits = (int)(b1 - b0);
    const int nchunks = (nits + kChunk - 1) / kChunk;

    const float *su = nullptr;
    if (a.ubasis) {
        if (tid < kUSize) su_buf[tid] = a.ubasis[(size_t)prob * kUSize + tid];
        su = su_buf;
    }
    // Operand rows >= D are never written and stay zero.
    for (int i = tid; i < kStages * kStageBytes / 16; i += kThreads)
        reinterpret_cast<uint4 *>(stages)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&empty[s]), 1);
        for (int b = 0; b < 2; ++b) mbar_init(smem_addr(&acc_full[b]), 1);
        mbar_init(smem_addr(fin), 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), kTmemCols);
        tmem_relinquish();
    }
#pragma unroll
    for (int j = 0; j <= kAhead; ++j) fetch_stage<R>(raw + j * kRawLen, pr, (b0 + j) * R, T, j < nits);
    cp_async_wait<kAhead>();   // stage 0 has landed (this thread's copies)
    __syncthreads();
    if (nits > 0) stage_series<FMT, R>(staging, raw, b0 * R, pr.n, B, T, su);
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int quarter = warp & 3, piece = warp >> 2;
    const int row = 32 * quarter + lane;   // tensor-memory lane = distinct column
    // piece 0: P [0, 64), 1: P [64, 112), 2: Q [128, 192), 3: Q [192, 240)
    const int pcol = (piece >> 1) * 128 + (piece & 1) * 64;
    const bool wide = (piece & 1) == 0;   // 64 columns, else 48
    const uint32_t lane_taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)pcol;
    float acc[kAccPer];
#pragma unroll
    for (int i = 0; i < kAccPer; ++i) acc[i] = 0.f;

    // This thread's operand chunks: task tid + 256 q = (column << 3) | chunk.
    int src[kTasks], dst[kTasks], chk[kTasks];
#pragma unroll
    for (int q = 0; q < kTasks; ++q) {
        const int task = tid + kThreads * q;
        src[q] = -1;
        dst[q] = 0;
        chk[q] = 0;
        if (task < 8 * D) {
            const int d = task >> 3, ch = task & 7;
            int series, off;
            distinct_source(d, B, T, series, off);
            int word;
            if constexpr (FMT == kFmtBF16) {
                const int o = ch * 8 + off;
                word = (o & 1) ? kSerLen / 2 + (o - 1) / 2 : o / 2;
            } else {
                word = ch * 4 + off;
            }
            src[q] = series * (kSerBytes / 4) + word;
            dst[q] = (int)sw128_offset(d, ch);
            chk[q] = ch;
        }
    }

    // MMAs of stage j (thread 0, after a barrier that followed every thread's
    // writes of that stage and every drain of the accumulator it reuses).
    const uint32_t idesc = umma_idesc(FMT, 128, kAccN);   // M = 128, N = 256
    int issued = 0;
    auto issue = [&](int j) {
        const int s = j % kStages, c = j / kChunk, buf = c & 1;
        tc_fence_after_sync();
        const uint32_t hb = smem_addr(stages + s * kStageBytes);   // hi rows 0-127, lo rows 128-255
        const uint32_t dacc = tmem + (uint32_t)(buf * kAccN);
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) {
            const uint64_t desc = umma_desc_sw128(hb + kk * 32);
            const uint32_t accumulate = (j % kChunk == 0 && kk == 0) ? 0u : 1u;
            if constexpr (FMT == kFmtBF16)
                umma_bf16(dacc, desc, desc, idesc, accumulate);
            else
                umma_tf32(dacc, desc, desc, idesc, accumulate);
        }
        ++issued;
        umma_commit(smem_addr(&empty[s]));
        if ((j + 1) % kChunk == 0 || j + 1 == nits) umma_commit(smem_addr(&acc_full[buf]));
    };

    auto drain = [&](int c) -> bool {
        const int buf = c & 1;
        const bool ok = mbar_wait(smem_addr(&acc_full[buf]), (uint32_t)((c >> 1) & 1), a.status);
        tc_fence_after_sync();
        if (ok) {
            float v[64];
            tmem_ld64(lane_taddr + (uint32_t)(buf * kAccN), v);
#pragma unroll
            for (int i = 0; i < 64; ++i) acc[i] += v[i];
        }
        tc_fence_before_sync();
        return ok;
    };

    bool failed = false;
    int next_drain = 0;
    bool drained_ok = true;   // drains of the previous iteration
    for (int it = 0; it < nits; ++it) {
        const int s = it % kStages;
        bool ok = drained_ok;
        if (it >= kStages)
            ok = mbar_wait(smem_addr(&empty[s]), (uint32_t)(((it / kStages) - 1) & 1), a.status) && ok;
        cp_async_wait<kAhead - 1>();   // this thread's copies of stage it + 1 have landed
        // every thread has written stage it - 1, drained what it had to, and
        // its copies of stage it + 1 are visible
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0 && it > 0) issue(it - 1);
        const int64_t n0 = (b0 + it) * R;
        // the slot of stage it (read in the previous iteration) receives stage it + kAhead + 1
        fetch_stage<R>(raw + (it % kRawSlots) * kRawLen, pr, n0 + (int64_t)(kAhead + 1) * R, T,
                       it + kAhead + 1 < nits);
        const uint32_t *stw = reinterpret_cast<const uint32_t *>(staging + (it & 1) * kStagingBytes);
        unsigned char *hi = stages + s * kStageBytes;
        unsigned char *lo = hi + kOpTile;
        const int64_t rem = pr.n - n0;
        const int nvalid = rem < R ? (int)rem : R;
#pragma unroll
        for (int q = 0; q < kTasks; ++q) {
            if (src[q] < 0) continue;
            const uint32_t *hw = stw + src[q];
            const uint32_t *lw = hw + kSerLen;   // lo arrays follow the hi arrays
            uint32_t h[4], l[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                h[k] = hw[k];
                l[k] = lw[k];
            }
            if (nvalid < R) {   // last stage of the problem: rows past the end are zero
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t m;
                    if constexpr (FMT == kFmtBF16) {
                        const int r0 = chk[q] * 8 + 2 * k;
                        m = (r0 < nvalid ? 0x0000FFFFu : 0u) | (r0 + 1 < nvalid ? 0xFFFF0000u : 0u);
                    } else {
                        m = chk[q] * 4 + k < nvalid ? 0xFFFFFFFFu : 0u;
                    }
                    h[k] &= m;
                    l[k] &= m;
                }
            }
            *reinterpret_cast<uint4 *>(hi + dst[q]) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(lo + dst[q]) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        if (it + 1 < nits)
            stage_series<FMT, R>(staging + ((it + 1) & 1) * kStagingBytes, raw + ((it + 1) % kRawSlots) * kRawLen,
                                 n0 + R, pr.n, B, T, su);
        fence_async_shared();
        // Drain every chunk whose last stage was consumed kStages stages ago:
        // its MMAs are complete (this stage's empty wait saw them).  A failed
        // drain is voted on at the top of the next iteration.
        while (next_drain < nchunks) {
            const int last = min((next_drain + 1) * kChunk, nits) - 1;
            if (last + kStages > it) break;
            drained_ok = drain(next_drain++) && drained_ok;
        }
    }
    if (!failed && nits > 0) {
        if (__syncthreads_or(!drained_ok)) {
            failed = true;
        } else {
            if (tid == 0) issue(nits - 1);
            while (next_drain < nchunks) drained_ok = drain(next_drain++) && drained_ok;
            failed = __syncthreads_or(!drained_ok);
        }
    }
    cp_async_wait<0>();   // no copy into this CTA's shared memory outlives it
    // Every MMA issued must be complete before tensor memory is released.
    if (tid == 0 && issued > 0) {
        umma_commit(smem_addr(fin));
        mbar_wait(smem_addr(fin), 0u, a.status);
    }

    float *part = a.partials + (size_t)blockIdx.x * kGramRows * kGramPartCols;
    const bool zero = failed || nits == 0;
#pragma unroll
    for (int i = 0; i < kAccPer; ++i)   // P -> partial columns [0, 112), Q -> [112, 224)
        if (wide || i < 48) part[(size_t)row * kGramPartCols + (piece >> 1) * kGramS + (piece & 1) * 64 + i] = zero ? 0.f : acc[i];

    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

size_t gram_tc_smem()
{
    return 1024 + (size_t)kStages * kStageBytes + 2 * (size_t)kStagingBytes + (size_t)kRawSlots * kRawLen * 8 +
           (kStages + 3) * 8 + 16 + kUSize * 4;
}

// ------------------------------------------------------------------ FP32 CUDA cores
// Each CTA stages 64 rows of the distinct columns (row-major, padded to 104,
// FP32) in shared memory; thread t owns one 8 x 8 block (I, J), I <= J, of the
// upper triangle of S and accumulates it over the rows.
constexpr int kF32Rows = 64;
constexpr int kF32Stride = 104;   // D <= 99, padded to whole 8-column blocks
constexpr int kF32Threads = 96;   // >= 13 * 14 / 2 = 91 diagonal-and-upper 8 x 8 blocks

// Fill psi[b][w] = |u|^{2b} u for samples n0 - (T-1) + w (zero outside [0, n)) and tv[rr] = t.
template <int R>
__device__ __forceinline__ void stage_basis(const GramProblem &pr, int64_t n0, int T, int B, float2 *psi, float2 *tv,
                                            const float *su)
{
    const int W = R + T - 1;
    for (int i = threadIdx.x; i < W * B; i += blockDim.x) {
        const int bb = i / W, w = i % W;
        const int64_t j = n0 - (T - 1) + w;
        float2 v = make_float2(0.f, 0.f);
        if (j >= 0 && j < pr.n) {
            const float2 x = pr.u[j];
            const float r = fmaf(x.x, x.x, x.y * x.y);
            float p = 1.f;
            if (su) {   // sum_{a <= bb} U[a][bb] r^a by Horner's rule
                p = su[bb * kMaxB + bb];
                for (int a2 = bb - 1; a2 >= 0; --a2) p = fmaf(p, r, su[a2 * kMaxB + bb]);
            } else {
                for (int e = 0; e < bb; ++e) p *= r;
            }
            v = make_float2(p * x.x, p * x.y);
        }
        psi[bb * kPsiStride + w] = v;
    }
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (pr.t && n0 + i < pr.n) v = pr.t[n0 + i];
        tv[i] = v;
    }
}

// Value of distinct column d at stage row rr (sample n0 + rr).
__device__ __forceinline__ float distinct_value(int d, int B, int T, const float2 *psi, const float2 *tv, int rr,
                                                bool valid)
{
    const int BT = B * T;
    if (!valid || d >= 2 * BT + 3) return 0.f;
    if (d < 2 * BT) {
        const int im = d >= BT, dd = im ? d - BT : d;
        const float2 p = psi[(dd / T) * kPsiStride + rr + (T - 1) - dd % T];
        return im ? p.y : p.x;
    }
    if (d == 2 * BT) return 1.f;
    return d == 2 * BT + 1 ? tv[rr].x : tv[rr].y;
}

__global__ void __launch_bounds__(kF32Threads) gram_fp32_kernel(GramArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_f[];
    float *Atile = reinterpret_cast<float *>(smem_f);                           // [kF32Rows][kF32Stride]
    float2 *psi = reinterpret_cast<float2 *>(Atile + kF32Rows * kF32Stride);  // [kMaxB][kPsiStride]
    float2 *tv = psi + kMaxB * kPsiStride;
    float *su_buf = reinterpret_cast<float *>(tv + 64);   // basis coefficients U (kUSize)

    const int tid = threadIdx.x;
    const int prob = blockIdx.x / a.cpp, chunk = blockIdx.x % a.cpp;
    const GramProblem pr = a.probs[prob];
    const int T = a.T, B = a.Bp > a.Bq ? a.Bp : a.Bq;
    const int D = gram_distinct(B, T);
    const int nb8 = (D + 7) / 8;
    const float *su = nullptr;
    if (a.ubasis) {
        for (int i = tid; i < kUSize; i += kF32Threads) su_buf[i] = a.ubasis[(size_t)prob * kUSize + i];
        su = su_buf;   // read after the first __syncthreads of the row loop
    }
    // block (I, J) of this thread: enumerate the upper triangle row by row
    int I = -1, J = -1;
    {
        int idx = tid;
        for (int i = 0; i < nb8 && I < 0; ++i) {
            const int cnt = nb8 - i;
            if (idx < cnt) {
                I = i;
                J = i + idx;
            } else {
                idx -= cnt;
            }
        }
    }
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int64_t nblk = (pr.n + kF32Rows - 1) / kF32Rows;
    const int64_t b0 = nblk * chunk / a.cpp, b1 = nblk * (chunk + 1) / a.cpp;
    for (int64_t blk = b0; blk < b1; ++blk) {
        const int64_t n0 = blk * kF32Rows;
        __syncthreads();
        stage_basis<kF32Rows>(pr, n0, T, B, psi, tv, su);
        __syncthreads();
        for (int e = tid; e < kF32Rows * kF32Stride; e += kF32Threads) {
            const int rr = e / kF32Stride, d = e % kF32Stride;
            Atile[e] = distinct_value(d, B, T, psi, tv, rr, n0 + rr < pr.n);
        }
        __syncthreads();
        if (I >= 0) {
            for (int rr = 0; rr < kF32Rows; ++rr) {
                const float4 *rowp = reinterpret_cast<const float4 *>(Atile + rr * kF32Stride);
                const float4 a0 = rowp[2 * I], a1 = rowp[2 * I + 1], b0v = rowp[2 * J], b1v = rowp[2 * J + 1];
                const float ai[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bj[8] = {b0v.x, b0v.y, b0v.z, b0v.w, b1v.x, b1v.y, b1v.z, b1v.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(ai[i], bj[j], acc[i][j]);
            }
        }
    }
    // P = the sums (upper blocks; the rest of P is never read), Q = 0.
    float *part = a.partials + (size_t)blockIdx.x * kGramRows * kGramPartCols;
    for (int e = tid; e < kGramRows * kGramS; e += kF32Threads)
        part[(size_t)(e / kGramS) * kGramPartCols + kGramS + e % kGramS] = 0.f;
    if (I >= 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = 8 * I + i, c = 8 * J + j;
                if (r < kGramS && c < kGramS) part[(size_t)r * kGramPartCols + c] = acc[i][j];
            }
    }
}

size_t gram_fp32_smem() { return (size_t)kF32Rows * kF32Stride * 4 + (kMaxB * kPsiStride + 64) * 8 + kUSize * 4; }

int gram_ctas_per_problem(int precision, int sm_count, int nprob, int64_t n)
{
    // tensor kernel: one CTA per SM in total; FP32 kernel: four (small CTAs);
    // at least one per problem, no more than row blocks
    const int total = precision == kPrecFP32 ? 4 * sm_count : sm_count;
    int cpp = total / (nprob > 0 ? nprob : 1);
    if (cpp < 1) cpp = 1;
    const int64_t blocks = (n + 63) / 64;
    if (cpp > blocks) cpp = (int)(blocks > 1 ? blocks : 1);
    return cpp;
}

cudaError_t launch_gram(int precision, const GramArgs &a, cudaStream_t s)
{
    const int grid = a.nprob * a.cpp;
    if (grid <= 0) return cudaSuccess;
    if (precision == kPrecFP32) {
        static SmemAttr smem_rec;
        const cudaError_t e = ensure_smem(smem_rec, (const void *)gram_fp32_kernel, gram_fp32_smem());
        if (e != cudaSuccess) return e;
        gram_fp32_kernel<<<grid, kF32Threads, gram_fp32_smem(), s>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    auto kern = precision == kPrecBF16x3 ? gram_tc_kernel<kFmtBF16> : gram_tc_kernel<kFmtTF32>;
    static SmemAttr smem_rec[2];
    const int ai = precision == kPrecBF16x3 ? 0 : 1;
    const cudaError_t e = ensure_smem(smem_rec[ai], (const void *)kern, gram_tc_smem());
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, gram_tc_smem(), s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
