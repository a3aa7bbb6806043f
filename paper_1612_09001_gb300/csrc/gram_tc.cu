// Gram contraction S = X^T X of the distinct real columns of the basis (see
// dpd_gram.cuh): the tcgen05 tensor-core kernel (lagged correlations of the
// basis and target signals, split BF16 / TF32 operands) with the kernels that
// turn its sums into S, and the plain FP32 CUDA-core form it is compared
// against.
#include <cuda_bf16.h>

#include "dpd_gram.cuh"
#include "dpd_tc.cuh"

namespace dpd {

namespace {

constexpr int kPsiStride = 64 + kMaxT - 1;   // basis samples staged per FP32 tile (64 rows + taps)

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace

constexpr int kThreads = 512;

// ------------------------------------------------------------------ lag-correlation form
// Every distinct column is a signal read at a delay: tap k of signal s is
// x_s(n - k), zero before the record starts.  An entry of S that pairs taps
// m >= m' of signals a and b is therefore a lagged correlation of the two
// signals, less the products that fall off the end of the record:
//   S[(a, m), (b, m')] = C_ab(d) - sum_{k = N-m}^{N-1-d} x_a(k) x_b(k + d),  d = m - m',
//   C_ab(d) = sum_{k >= 0} x_a(k) x_b(k + d)   (x = 0 outside [0, N)).
// The tensor kernel below computes C for the 15 signals (Re / Im psi_b, b < 6;
// Re / Im t; the constant) against the 14 non-constant ones at lags 0 .. 7;
// the finishing kernels subtract the end products (at most T - 1 per entry,
// from the last samples of the record) and fill S.  The operands hold each
// signal once per sample instead of once per tap.
//
// Polyphase contraction.  With n = 8 q + r (phase r < 8),
//   D[(a, r), (b, j)] = sum_q x_a(8 q + r) x_b(8 q + j),   j < 16,
// and C_ab(d) = sum_r D[(a, r), (b, r + d)].  Rows (a, r) form the A operand
// (15 signals x 8 phases, padded to M = 128), rows (b, j) the B operand
// (14 signals x 16 = N = 224), q is the contraction index.  In the K-major
// layout without swizzle a core matrix is 8 rows x 16 bytes, so the 8 rows of
// one signal's phases r form one core-matrix row group; row (b, j + 8) is row
// (b, j) advanced by one q and is written as a second group right behind it.
// A signal's slot in a stage is [phases 0-7 | phases 8-15], 1 KB each (8 rows
// x 128 bytes: 8 core matrices along K); the A descriptor steps over slots
// (2 KB per 8 rows: first halves only, slot 15 stays zero), the B descriptor
// over halves (1 KB).
//
// Products.  X = hi + lo (BF16 or TF32) and hi hi + hi lo + lo hi are summed
// into one FP32 accumulator: three MMAs per K step, four K steps per stage.
//
// Generation.  One task per thread and stage: a core-matrix row (c, r) of one
// signal pair (Re / Im psi_b, or Re / Im t), i.e. E + 1 raw samples 8 apart
// (E = 8 BF16 / 4 TF32 values per 16-byte row, and the one that follows for
// the advanced row), or a row of the constant.  The raw ring is padded by 8
// samples per 8 E so that the 16 lanes of a half warp (two core matrices c)
// load from distinct banks.
constexpr int kLagSigA = 15;                 // A side: 12 basis, 2 target, the constant
constexpr int kLagSigB = 14;                 // B side: all but the constant
constexpr int kLagSerT = 12, kLagSerOne = 14;
constexpr int kLagHalfBytes = 1024;          // 8 rows x 128 bytes (8 core matrices along K)
constexpr int kLagSlotBytes = 2 * kLagHalfBytes;
constexpr int kLagPart = 16 * kLagSlotBytes; // hi (then lo) part of a stage
constexpr int kLagStageBytes = 2 * kLagPart;
constexpr int kLagStages = 3;
constexpr int kLagAhead = 2;                 // raw stages fetched ahead
constexpr int kLagRawSlots = kLagAhead + 1;
constexpr int kLagKSteps = 4;                // MMA K steps per stage (16 BF16 / 8 TF32 values each)
constexpr int kLagN = 16 * kLagSigB;         // 224 accumulator columns
constexpr int kLagAccCols = 256;             // column spacing of the two accumulators
constexpr int kLagChunk = 4;                 // stages per accumulation chunk
constexpr int kLagDStride = 257;             // row stride of the final D in shared memory (floats)
constexpr int kLagGenWarps = 15;             // operand generators; warp 15 issues the MMAs
constexpr int kLagGenThreads = 32 * kLagGenWarps;
static_assert(kLagStages <= kLagChunk + 1, "drain must precede the reuse of an accumulator");
static_assert(kLagN == 3 * 64 + 32, "drain pieces: three of 64 columns and one of 32");
static_assert(kLagEntries == kLagSigA * kLagSigB * kMaxT, "lag partial size");

template <int FMT>
struct LagGeom {
    static constexpr int E = FMT == kFmtBF16 ? 8 : 4;      // values per 16-byte core-matrix row
    static constexpr int R = 8 * 8 * E;                    // samples per stage: 8 phases x 8 core matrices x E
    __host__ __device__ static constexpr int pidx(int j) { return j + 8 * (j / (8 * E)); }
    static constexpr int RawSig = R + 8 + 8 * ((R + 7) / (8 * E));   // padded samples per raw signal
    static constexpr int Raw = 2 * RawSig;                 // float2 per raw slot: u, then t
};

// psi_b = w_b(|u|^2) u: w_b(r) = r^b, or sum_{a <= b} U[a][b] r^a (Horner).
__device__ __forceinline__ float psi_weight(int b, float r, const float *su)
{
    float p = 1.f;
    if (su) {
        p = su[b * kMaxB + b];
        for (int a = b - 1; a >= 0; --a) p = fmaf(p, r, su[a * kMaxB + b]);
    } else {
        for (int e = 0; e < b; ++e) p *= r;   // low order first, as in the filter
    }
    return p;
}

// Raw samples of a stage: u and t from n0, R + 8 of each (the last 8 feed the
// advanced rows), zero outside the problem.  One copy group per generator
// thread and stage.
template <int FMT>
__device__ __forceinline__ void lag_fetch(float2 *slot, const GramProblem &pr, int64_t n0, bool active)
{
    using G = LagGeom<FMT>;
    if (active) {
        for (int i = threadIdx.x; i < G::R + 8; i += kLagGenThreads) {
            const int64_t j = n0 + i;
            const bool vu = j < pr.n, vt = pr.t != nullptr && j < pr.n;
            const int o = G::pidx(i);
            cp_async8(smem_addr(slot + o), vu ? pr.u + j : pr.u, vu ? 8u : 0u);
            cp_async8(smem_addr(slot + G::RawSig + o), vt ? pr.t + j : pr.u, vt ? 8u : 0u);
        }
    }
    cp_async_commit();
}

// One core-matrix row (16 bytes) of a signal and its advanced copy, hi and lo:
// v[i] is the value at K index i of the row, v[E] the next one.
__device__ __forceinline__ uint32_t bf16x2_bits(float lo_elem, float hi_elem)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);   // lo_elem in the low half
    return *reinterpret_cast<const uint32_t *>(&h);
}

template <int FMT, int E>
__device__ __forceinline__ void lag_put(unsigned char *p, const float (&v)[E + 1])
{
    uint32_t h[4], hs[4], l[4], ls[4];
    if constexpr (FMT == kFmtBF16) {
        uint32_t H[5], L[5];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            H[k] = bf16x2_bits(v[2 * k], v[2 * k + 1]);
            L[k] = bf16x2_bits(v[2 * k] - __uint_as_float(H[k] << 16),
                               v[2 * k + 1] - __uint_as_float(H[k] & 0xFFFF0000u));
        }
        H[4] = bf16x2_bits(v[8], 0.f);
        L[4] = bf16x2_bits(v[8] - __uint_as_float(H[4] << 16), 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // advanced by one: elements 2k + 1, 2k + 2
            h[k] = H[k];
            l[k] = L[k];
            hs[k] = __byte_perm(H[k], H[k + 1], 0x5432);
            ls[k] = __byte_perm(L[k], L[k + 1], 0x5432);
        }
    } else {
        float hf[E + 1];
        uint32_t lw[E + 1];
#pragma unroll
        for (int i = 0; i <= E; ++i) {
            hf[i] = to_tf32(v[i]);
            lw[i] = __float_as_uint(to_tf32(v[i] - hf[i]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            h[k] = __float_as_uint(hf[k]);
            hs[k] = __float_as_uint(hf[k + 1]);
            l[k] = lw[k];
            ls[k] = lw[k + 1];
        }
    }
    *reinterpret_cast<uint4 *>(p) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(p + kLagHalfBytes) = make_uint4(hs[0], hs[1], hs[2], hs[3]);
    *reinterpret_cast<uint4 *>(p + kLagPart) = make_uint4(l[0], l[1], l[2], l[3]);
    *reinterpret_cast<uint4 *>(p + kLagPart + kLagHalfBytes) = make_uint4(ls[0], ls[1], ls[2], ls[3]);
}

// Operands of the stage starting at sample n0 from its raw slot.  Warp w:
// w < 12: Re / Im psi_{w/2}; 12, 13: Re / Im t, core matrices c = 4 (w & 1)
// .. + 3, lane (c, r); 14: the constant, all 64 rows.
template <int FMT>
__device__ __forceinline__ void lag_generate(unsigned char *st, const float2 *slot, int64_t n0, int64_t n,
                                             const float *su)
{
    using G = LagGeom<FMT>;
    constexpr int E = G::E;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == 14) {   // 1 inside the record (hi only; lo and the advanced rows stay zero)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int c = 4 * hh + (lane >> 3), r = lane & 7;
            uint32_t q[4];
            if constexpr (FMT == kFmtBF16) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t s0 = n0 + 8 * (E * c + 2 * k) + r;
                    q[k] = (s0 < n ? 0x3F80u : 0u) | (s0 + 8 < n ? 0x3F800000u : 0u);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) q[k] = n0 + 8 * (E * c + k) + r < n ? 0x3F800000u : 0u;
            }
            *reinterpret_cast<uint4 *>(st + kLagSerOne * kLagSlotBytes + c * 128 + r * 16) =
                make_uint4(q[0], q[1], q[2], q[3]);
        }
        return;
    }
    const int c = 4 * (w & 1) + (lane >> 3), r = lane & 7;
    const bool target = w >= 12;
    // sample 8 (E c + i) + r of the slot sits at pidx = (8 E + 8) c + 8 i + r for
    // i < E, and sample E (the next core matrix) 8 further
    const float2 *src = slot + (target ? G::RawSig : 0) + (8 * E + 8) * c + r;
    float re[E + 1], im[E + 1];
#pragma unroll
    for (int i = 0; i <= E; ++i) {
        const float2 x = src[i < E ? 8 * i : 8 * E + 8];
        re[i] = x.x;
        im[i] = x.y;
    }
    int sig = kLagSerT;
    if (!target) {
        const int b = w >> 1;
        sig = 2 * b;
        float rr[E + 1], pw[E + 1];
#pragma unroll
        for (int i = 0; i <= E; ++i) rr[i] = fmaf(re[i], re[i], im[i] * im[i]);
        // w_b(r) exactly as psi_weight evaluates it
        if (su) {
            const float top = su[b * kMaxB + b];
#pragma unroll
            for (int i = 0; i <= E; ++i) pw[i] = top;
            for (int a = b - 1; a >= 0; --a) {
                const float cf = su[a * kMaxB + b];
#pragma unroll
                for (int i = 0; i <= E; ++i) pw[i] = fmaf(pw[i], rr[i], cf);
            }
        } else {
#pragma unroll
            for (int i = 0; i <= E; ++i) pw[i] = 1.f;
            for (int e = 0; e < b; ++e)
#pragma unroll
                for (int i = 0; i <= E; ++i) pw[i] *= rr[i];
        }
#pragma unroll
        for (int i = 0; i <= E; ++i) {
            re[i] *= pw[i];
            im[i] *= pw[i];
        }
    }
    unsigned char *p = st + sig * kLagSlotBytes + c * 128 + r * 16;
    lag_put<FMT, E>(p, re);
    lag_put<FMT, E>(p + kLagSlotBytes, im);
}

// Named barrier over the generator warps, OR-reducing a flag.
__device__ __forceinline__ bool gen_barrier_or(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
        "barrier.cta.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kLagGenThreads)
        : "memory");
    return r != 0;
}

// Barriers: full[s] (the 15 generator warps have written stage buffer s),
// empty[s] (MMA commit: stage buffer s consumed), acc_full[b] (a chunk's sum is
// complete in accumulator b), fin (everything issued has completed).
// Roles: warps 0 .. 14 fetch and generate, warp 15 issues the MMAs (lane 0),
// all sixteen drain.  An MMA issue blocks while the tensor core's queue is
// full, so the issuing warp does nothing else on the way: the generators run
// up to kLagStages stages ahead of it, synchronised only among themselves
// (raw-slot reuse) and through full / empty.
template <int FMT>
__global__ void __launch_bounds__(kThreads, 1) gram_lag_kernel(GramArgs a)
{
    using G = LagGeom<FMT>;
    constexpr int R = G::R;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stages = smem;
    float2 *raw = reinterpret_cast<float2 *>(stages + kLagStages * kLagStageBytes);
    uint64_t *empty = reinterpret_cast<uint64_t *>(raw + kLagRawSlots * G::Raw);
    uint64_t *full = empty + kLagStages;
    uint64_t *acc_full = full + kLagStages;
    uint64_t *fin = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    float *su_buf = reinterpret_cast<float *>(tmem_slot + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int prob = blockIdx.x / a.cpp, chunk = blockIdx.x % a.cpp;
    const GramProblem pr = a.probs ? a.probs[prob] : a.one;
    const int64_t nblk = (pr.n + R - 1) / R;
    const int64_t b0 = nblk * chunk / a.cpp, b1 = nblk * (chunk + 1) / a.cpp;
    const int nits = (int)(b1 - b0);
    const int nchunks = (nits + kLagChunk - 1) / kLagChunk;

    const float *su = nullptr;
    if (a.ubasis) {
        if (tid < kUSize) su_buf[tid] = a.ubasis[(size_t)prob * kUSize + tid];
        su = su_buf;
    }
    // Slot 15, the constant's lo and advanced rows are never written and stay zero.
    for (int i = tid; i < kLagStages * kLagStageBytes / 16; i += kThreads)
        reinterpret_cast<uint4 *>(stages)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int s = 0; s < kLagStages; ++s) {
            mbar_init(smem_addr(&empty[s]), 1);
            mbar_init(smem_addr(&full[s]), kLagGenWarps);
        }
        for (int b = 0; b < 2; ++b) mbar_init(smem_addr(&acc_full[b]), 1);
        mbar_init(smem_addr(fin), 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), 2 * kLagAccCols);
        tmem_relinquish();
    }
    const bool generator = warp < kLagGenWarps;
    if (generator) {
#pragma unroll
        for (int j = 0; j < kLagAhead; ++j) lag_fetch<FMT>(raw + j * G::Raw, pr, (b0 + j) * R, j < nits);
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int quarter = warp & 3, piece = warp >> 2;
    const int row = 32 * quarter + lane;   // tensor-memory lane = A row (signal, phase)
    const uint32_t lane_taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(64 * piece);
    float acc[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0.f;

    const uint32_t idesc = umma_idesc(FMT, 128, kLagN);
    int issued = 0;
    auto issue = [&](int j) {
        const int s = j % kLagStages, c = j / kLagChunk, buf = c & 1;
        tc_fence_after_sync();
        const uint32_t hb = smem_addr(stages + s * kLagStageBytes), lb = hb + kLagPart;
        const uint32_t dacc = tmem + (uint32_t)(buf * kLagAccCols);
#pragma unroll
        for (int kk = 0; kk < kLagKSteps; ++kk) {
            const uint32_t o = (uint32_t)kk * 256u;   // two core matrices along K per step
            const uint64_t ah = umma_desc_kmajor(hb + o, 128u, kLagSlotBytes);
            const uint64_t al = umma_desc_kmajor(lb + o, 128u, kLagSlotBytes);
            const uint64_t bh = umma_desc_kmajor(hb + o, 128u, kLagHalfBytes);
            const uint64_t bl = umma_desc_kmajor(lb + o, 128u, kLagHalfBytes);
            const uint32_t first = (j % kLagChunk == 0 && kk == 0) ? 0u : 1u;
            if constexpr (FMT == kFmtBF16) {
                umma_bf16(dacc, ah, bh, idesc, first);
                umma_bf16(dacc, ah, bl, idesc, 1u);
                umma_bf16(dacc, al, bh, idesc, 1u);
            } else {
                umma_tf32(dacc, ah, bh, idesc, first);
                umma_tf32(dacc, ah, bl, idesc, 1u);
                umma_tf32(dacc, al, bh, idesc, 1u);
            }
        }
        ++issued;
        umma_commit(smem_addr(&empty[s]));
        if ((j + 1) % kLagChunk == 0 || j + 1 == nits) umma_commit(smem_addr(&acc_full[buf]));
    };

    auto drain = [&](int c) -> bool {
        const int buf = c & 1;
        const bool ok = mbar_wait(smem_addr(&acc_full[buf]), (uint32_t)((c >> 1) & 1), a.status);
        tc_fence_after_sync();
        if (ok) {
            if (piece == 3) {   // columns 192 .. 223: the last 32 of the 256 are unused (N = 224)
                float v[32];
                tmem_ld32(lane_taddr + (uint32_t)(buf * kLagAccCols), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[i] += v[i];
            } else {
                float v[64];
                tmem_ld64(lane_taddr + (uint32_t)(buf * kLagAccCols), v);
#pragma unroll
                for (int i = 0; i < 64; ++i) acc[i] += v[i];
            }
        }
        tc_fence_before_sync();
        return ok;
    };

    bool failed = false;
    int next_drain = 0;
    bool drained_ok = true;
    if (generator) {
        for (int it = 0; it < nits; ++it) {
            const int s = it % kLagStages;
            bool ok = drained_ok;
            if (it >= kLagStages)
                ok = mbar_wait(smem_addr(&empty[s]), (uint32_t)(((it / kLagStages) - 1) & 1), a.status) && ok;
            cp_async_wait<kLagAhead - 1>();   // this thread's copies of stage it have landed
            // every generator has finished stage it - 1 and its copies of stage it are visible
            if (gen_barrier_or(!ok)) {
                failed = true;
                break;
            }
            // the slot of stage it - 1 (read in the previous iteration) receives stage it + kLagAhead
            lag_fetch<FMT>(raw + ((it + kLagAhead) % kLagRawSlots) * G::Raw, pr, (b0 + it + kLagAhead) * R,
                           it + kLagAhead < nits);
            lag_generate<FMT>(stages + s * kLagStageBytes, raw + (it % kLagRawSlots) * G::Raw, (b0 + it) * R, pr.n,
                              su);
            fence_async_shared();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&full[s]));
            while (next_drain < nchunks) {
                const int last = min((next_drain + 1) * kLagChunk, nits) - 1;
                if (last + kLagStages > it) break;
                drained_ok = drain(next_drain++) && drained_ok;
            }
        }
        if (!failed)
            while (next_drain < nchunks) drained_ok = drain(next_drain++) && drained_ok;
    } else {
        // The issuer drains chunk c once the first stage after it is queued
        // (the tensor core stays busy while it waits).
        for (int j = 0; j < nits; ++j) {
            const int s = j % kLagStages;
            bool ok = mbar_wait(smem_addr(&full[s]), (uint32_t)((j / kLagStages) & 1), a.status);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                failed = true;
                break;
            }
            if (lane == 0) issue(j);
            __syncwarp();
            while (next_drain < nchunks && min((next_drain + 1) * kLagChunk, nits) <= j)
                drained_ok = drain(next_drain++) && drained_ok;
        }
        if (!failed)
            while (next_drain < nchunks) drained_ok = drain(next_drain++) && drained_ok;
    }
    failed = failed || !drained_ok;
    cp_async_wait<0>();
    if (warp == kLagGenWarps && lane == 0 && issued > 0) {
        umma_commit(smem_addr(fin));
        mbar_wait(smem_addr(fin), 0u, a.status);
    }
    tc_fence_before_sync();
    failed = __syncthreads_or(failed);   // every MMA has completed: the stage buffers are free

    // C[a][b][d] = sum_r D[(a, r), (b, r + d)] through shared memory: an FP32
    // sum with its rounding error carried exactly (two-sum), stored as the
    // pair (sum, error); the FP64 additions (slow on this GPU) are left to the
    // reduction over CTAs.
    float *Dsm = reinterpret_cast<float *>(stages);
    const bool zero = failed || nits == 0;
#pragma unroll
    for (int i = 0; i < 64; ++i)
        if (64 * piece + i < kLagN) Dsm[row * kLagDStride + 64 * piece + i] = zero ? 0.f : acc[i];
    __syncthreads();
    float2 *part = reinterpret_cast<float2 *>(a.partials) + (size_t)blockIdx.x * kLagEntries;
    for (int e = tid; e < kLagEntries; e += kThreads) {
        const int sa = e / (kLagSigB * kMaxT), sb = (e / kMaxT) % kLagSigB, d = e % kMaxT;
        const float *dp = Dsm + (8 * sa) * kLagDStride + 16 * sb + d;
        float sum = dp[0], err = 0.f;
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            const float x = dp[r * (kLagDStride + 1)];
            const float t = sum + x, z = t - sum;
            err += (sum - (t - z)) + (x - z);
            sum = t;
        }
        part[e] = make_float2(sum, err);
    }

    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 2 * kLagAccCols);
    }
}

size_t gram_lag_smem(int fmt)
{
    const int raw = fmt == kFmtBF16 ? LagGeom<kFmtBF16>::Raw : LagGeom<kFmtTF32>::Raw;
    const size_t body = (size_t)kLagStages * kLagStageBytes + (size_t)kLagRawSlots * raw * 8 +
                        (2 * kLagStages + 3) * 8 + 16 + kUSize * 4;
    const size_t dfinal = (size_t)128 * kLagDStride * 4;
    return 1024 + (body > dfinal ? body : dfinal);
}

// ---- finishing: partial lag sums -> S
// C[p][e] = sum over the problem's CTAs of the partial pairs, in a fixed order (FP32 pairs, then FP64).
__global__ void __launch_bounds__(256) gram_lag_reduce_kernel(const float2 *__restrict__ partials, int cpp,
                                                              double *__restrict__ C)
{
    __shared__ double grp[8][32];
    const int p = blockIdx.y, lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (e < kLagEntries) {
        // The partials are FP32 (sum, error) pairs; they are added as pairs in
        // FP32 (about 2^-48 relative) and each thread's total becomes FP64 once:
        // FP64 additions and conversions per partial (a small fraction of the
        // FP32 rate on this GPU) bound this kernel before.
        const float2 *base = partials + (size_t)p * cpp * kLagEntries + e;
        auto val = [&](int k) { return base[(size_t)k * kLagEntries]; };
        float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;   // partials g, g + 8, g + 16, g + 24, ...
        int k = g;
        for (; k + 24 < cpp; k += 32) {
            s0 = pair_add(s0, val(k));
            s1 = pair_add(s1, val(k + 8));
            s2 = pair_add(s2, val(k + 16));
            s3 = pair_add(s3, val(k + 24));
        }
        for (; k < cpp; k += 8) s0 = pair_add(s0, val(k));
        const float2 t = pair_add(pair_add(s0, s1), pair_add(s2, s3));
        s = (double)t.x + (double)t.y;
    }
    grp[g][lane] = s;
    __syncthreads();
    if (g == 0 && e < kLagEntries) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += grp[q][lane];
        C[(size_t)p * kLagEntries + e] = t;
    }
}

// Signal and tap of distinct column d (the order of dpd_gram.cuh).
__device__ __forceinline__ void lag_source(int d, int B, int T, int &sig, int &tap)
{
    const int BT = B * T;
    if (d < 2 * BT) {
        const int im = d >= BT ? 1 : 0, dd = im ? d - BT : d;
        sig = 2 * (dd / T) + im;
        tap = dd % T;
    } else {
        sig = d == 2 * BT ? kLagSerOne : kLagSerT + (d - 2 * BT - 1);
        tap = 0;
    }
}

// G, g and t^H t of each problem from its lag sums; grid (entries / 256,
// problems).  An entry of S is C less the end products, which come from the
// last T - 1 samples of every signal evaluated as the tensor kernel evaluates
// them; they are a few of the N products of an entry, so they are summed in
// FP32 and only the difference is formed in FP64.
__global__ void __launch_bounds__(256) gram_lag_assemble_kernel(const double *__restrict__ Call,
                                                                const GramProblem *__restrict__ probs,
                                                                GramProblem one, const float *__restrict__ ubasis,
                                                                int K, int Bp, int B, int T, double2 *__restrict__ G,
                                                                double2 *__restrict__ g, double *__restrict__ tt)
{
    __shared__ float xt[kLagSigA][kMaxT];   // x_s(N - 8 + i), zero before the record
    __shared__ float su_buf[kUSize];
    __shared__ int2 src[kGramS];             // (signal, tap) of each distinct column
    const int p = blockIdx.y, tid = threadIdx.x;
    const GramProblem pr = probs ? probs[p] : one;
    const int64_t N = pr.n;
    const int D = gram_distinct(B, T);
    const double *C = Call + (size_t)p * kLagEntries;
    const float *su = nullptr;
    if (ubasis) {
        if (tid < kUSize) su_buf[tid] = ubasis[(size_t)p * kUSize + tid];
        su = su_buf;
    }
    if (tid < D) {
        int sig, tap;
        lag_source(tid, B, T, sig, tap);
        src[tid] = make_int2(sig, tap);
    }
    __syncthreads();
    if (tid < kMaxT * 8) {
        const int i = tid / 8, gi = tid % 8;   // sample N - 8 + i; gi < 6 basis, 6 target, 7 constant
        const int64_t k = N - kMaxT + i;
        float v0 = 0.f, v1 = 0.f;
        if (k >= 0) {
            if (gi < 6) {
                const float2 x = pr.u[k];
                const float w = psi_weight(gi, fmaf(x.x, x.x, x.y * x.y), su);
                v0 = w * x.x;
                v1 = w * x.y;
            } else if (gi == 6) {
                if (pr.t) {
                    const float2 x = pr.t[k];
                    v0 = x.x;
                    v1 = x.y;
                }
            } else {
                v0 = 1.f;
            }
        }
        if (gi < 6) {
            xt[2 * gi][i] = v0;
            xt[2 * gi + 1][i] = v1;
        } else if (gi == 6) {
            xt[kLagSerT][i] = v0;
            xt[kLagSerT + 1][i] = v1;
        } else {
            xt[kLagSerOne][i] = v0;
        }
    }
    __syncthreads();
    // <x, y> for two signed distinct-column references, as the pair (lag sum,
    // end products): <x, y> = c - t.  The entries of G and g add two such
    // values; their lag sums are added in FP64 and their end products in FP32
    // (at most 2 (T - 1) products of the last samples), so that each component
    // costs one FP64 addition, one conversion and one FP64 subtraction (FP64 on
    // this GPU is a small fraction of the FP32 rate).
    struct Pair {
        double c;
        float t;
    };
    auto dot = [&](ColRef x, ColRef y) -> Pair {
        if (x.sign == 0 || y.sign == 0) return {0.0, 0.f};
        int sa = src[x.d].x, ma = src[x.d].y, sb = src[y.d].x, mb = src[y.d].y;
        // (sa, ma): the larger tap; at equal taps the constant on the A side
        if (mb > ma || (mb == ma && sb == kLagSerOne)) {
            const int s0 = sa, m0 = ma;
            sa = sb;
            ma = mb;
            sb = s0;
            mb = m0;
        }
        const int dl = ma - mb;
        double c = 0.0;
        float tl = 0.f;
        if ((int64_t)ma >= N) {
            // column (sa, ma) is zero on every row
        } else if (sb == kLagSerOne) {
            // against the constant at tap 0: sum_{k < N - ma} x_sa(k) = C[one][sa][0] less the last ma samples
            if (sa == kLagSerOne) {
                c = (double)N;
            } else {
                for (int k = 0; k < ma; ++k) tl += xt[sa][kMaxT - 1 - k];
                c = C[(kLagSerOne * kLagSigB + sa) * kMaxT];
            }
        } else {
            // samples N - ma .. N - 1 - dl: xt index k = sample - (N - 8)
            for (int k = kMaxT - ma; k <= kMaxT - 1 - dl; ++k) tl = fmaf(xt[sa][k], xt[sb][k + dl], tl);
            c = C[(sa * kLagSigB + sb) * kMaxT + dl];
        }
        return x.sign * y.sign > 0 ? Pair{c, tl} : Pair{-c, -tl};
    };
    // x + y and x - y of two such values
    auto sum = [](Pair x, Pair y) { return (x.c + y.c) - (double)(x.t + y.t); };
    auto diff = [](Pair x, Pair y) { return (x.c - y.c) - (double)(x.t - y.t); };
    const int idx = blockIdx.x * blockDim.x + tid;
    const ColRef tre{2 * B * T + 1, 1}, tim{2 * B * T + 2, 1};
    if (idx < K * K) {
        const int a = idx / K, b = idx % K;
        ColRef ar, ai, br, bi;
        psi_column_refs(a, K, Bp, B, T, ar, ai);
        psi_column_refs(b, K, Bp, B, T, br, bi);
        G[(size_t)p * K * K + idx] = make_double2(sum(dot(ar, br), dot(ai, bi)), diff(dot(ar, bi), dot(ai, br)));
    } else if (idx < K * K + K) {
        const int a = idx - K * K;
        ColRef ar, ai;
        psi_column_refs(a, K, Bp, B, T, ar, ai);
        if (g) g[(size_t)p * K + a] = make_double2(sum(dot(ar, tre), dot(ai, tim)), diff(dot(ar, tim), dot(ai, tre)));
    } else if (idx == K * K + K) {
        if (tt) tt[p] = sum(dot(tre, tre), dot(tim, tim));
    }
}

cudaError_t launch_gram_lag_finish(const float *partials, const GramProblem *probs, GramProblem one,
                                   const float *ubasis, int nprob, int cpp, int K, int Bp, int B, int T, double *C,
                                   double2 *G, double2 *g, double *tt, cudaStream_t s)
{
    gram_lag_reduce_kernel<<<dim3((kLagEntries + 31) / 32, nprob), 256, 0, s>>>(
        reinterpret_cast<const float2 *>(partials), cpp, C);
    count_launch();
    gram_lag_assemble_kernel<<<dim3((K * K + K + 1 + 255) / 256, nprob), 256, 0, s>>>(C, probs, one, ubasis, K, Bp,
                                                                                       B, T, G, g, tt);
    count_launch();
    return cudaGetLastError();
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
            const float p = psi_weight(bb, fmaf(x.x, x.x, x.y * x.y), su);
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
    const GramProblem pr = a.probs ? a.probs[prob] : a.one;
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
    const int rows = precision == kPrecFP32   ? kF32Rows
                     : precision == kPrecBF16x3 ? LagGeom<kFmtBF16>::R
                                                : LagGeom<kFmtTF32>::R;   // samples per stage
    const int64_t blocks = (n + rows - 1) / rows;
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
    const int fmt = precision == kPrecBF16x3 ? kFmtBF16 : kFmtTF32;
    auto kern = fmt == kFmtBF16 ? gram_lag_kernel<kFmtBF16> : gram_lag_kernel<kFmtTF32>;
    static SmemAttr smem_rec[2];
    const int ai = fmt == kFmtBF16 ? 0 : 1;
    const cudaError_t e = ensure_smem(smem_rec[ai], (const void *)kern, gram_lag_smem(fmt));
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, gram_lag_smem(fmt), s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
