// Gram contraction S = A^T A of the real-form basis (see dpd_gram.cuh):
// tcgen05 tensor-core kernel with split BF16 / TF32 operands, and the plain
// FP32 CUDA-core form it is compared against.
#include <cuda_bf16.h>

#include "dpd_gram.cuh"
#include "dpd_tc.cuh"

namespace dpd {

namespace {

constexpr int kGramThreads = 256;
constexpr int kTile = 16384;          // 128 operand rows x 128 bytes
constexpr int kBuf = 2 * kTile;       // 256 operand rows
constexpr int kStageBytes = 2 * kBuf; // hi + lo
constexpr int kStages = 2;
constexpr int kPsiStride = 64 + kMaxT - 1;

// Value of real-form column c at stage row rr (sample n0 + rr).
struct ColumnDecode {
    bool is_t, imag, conj, one;
    int b, k;
};

__device__ __forceinline__ ColumnDecode decode_column(int c, int K, int Bp, int T)
{
    ColumnDecode d{};
    int j;
    if (c < K) {
        j = c;
    } else if (c == K) {
        d.is_t = true;
        return d;
    } else if (c < 2 * K + 1) {
        d.imag = true;
        j = c - K - 1;
    } else {
        d.is_t = true;
        d.imag = true;
        return d;
    }
    if (j == K - 1) {
        d.one = true;
        return d;
    }
    if (j < Bp * T) {
        d.b = j / T;
        d.k = j % T;
    } else {
        d.conj = true;
        d.b = (j - Bp * T) / T;
        d.k = (j - Bp * T) % T;
    }
    return d;
}

__device__ __forceinline__ float column_value(const ColumnDecode &d, const float2 *psi, const float2 *tv, int rr,
                                              int T, bool valid)
{
    if (!valid) return 0.f;
    if (d.is_t) return d.imag ? tv[rr].y : tv[rr].x;
    if (d.one) return d.imag ? 0.f : 1.f;
    const float2 p = psi[d.b * kPsiStride + rr + (T - 1) - d.k];
    return d.imag ? (d.conj ? -p.y : p.y) : p.x;
}

// Fill psi[b][w] = |u|^{2b} u for samples n0 - (T-1) + w (zero outside [0, n)) and tv[rr] = t.
template <int R>
__device__ __forceinline__ void stage_basis(const GramProblem &pr, int64_t n0, int T, int B, float2 *psi, float2 *tv)
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
            for (int e = 0; e < bb; ++e) p *= r;
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

}  // namespace

// ------------------------------------------------------------------ tensor cores
// Operand generation.  Every real-form column of A is one of 15 "series" --
// Re / Im of psi_b(u_j) for b < 6, Re / Im of t, or the constant 1 -- read at
// row rr from element w = rr + off, off = T-1-k for the tap-k column and T-1
// for the unshifted ones (element w of a stage is sample n0 - (T-1) + w).  So
// each stage converts every basis value to its hi / lo pair once, into a
// series array in shared memory, and an operand chunk (8 BF16 or 4 TF32 rows
// of one column) is a few 32-bit shared loads and two 16-byte stores.  BF16
// series are kept twice, as 16-bit arrays starting at element 0 and at
// element 1, so a chunk at any offset reads whole aligned words.  The global
// loads of the next stage are issued before the current stage is generated.
//
// Accumulation.  The tensor core's FP32 accumulator drops low-order bits on
// every MMA step, a bias that grows with the number of steps summed into one
// accumulator.  So each accumulation covers a chunk of kChunk stages only:
// after a chunk, every thread adds its share of the tensor-memory
// accumulators (one lane quarter, 144 of the 288 columns) into FP32
// sums with round-to-nearest (D0 in registers, D1 in shared memory), and the
// next chunk starts from zero.
constexpr int kChunk = 4;
constexpr int kAccCols = 104;   // per generator thread: half of D0's 208 columns of its lane
constexpr int kD1Cols = 80;     // D1 running sums in shared memory: 128 lanes x 80 columns
constexpr int kD1Half = 40;
constexpr int kSeries = 15;     // 2 per basis order (6), 2 for t, 1 constant
constexpr int kSerLen = 72;     // elements per series (>= 64 + kMaxT - 1, even)
// Per series: BF16: hi, hi shifted by one, lo, lo shifted by one (16-bit each);
// TF32: hi, lo (32-bit each).  Both 4 * kSerLen * 2 bytes.
constexpr int kSerBytes = 4 * kSerLen * 2;
constexpr int kStagingBytes = kSeries * kSerBytes;

// Column map entry: series | off << 8 | flags << 16 (bit 0 negate, bit 1 zero column).
__device__ __forceinline__ int column_map(int c, int K, int Bp, int T)
{
    const ColumnDecode d = decode_column(c, K, Bp, T);
    int series, off = T - 1, flags = 0;
    if (d.is_t) {
        series = d.imag ? 13 : 12;
    } else if (d.one) {
        series = 14;
        if (d.imag) flags |= 2;
    } else {
        series = 2 * d.b + (d.imag ? 1 : 0);
        off = T - 1 - d.k;
        if (d.imag && d.conj) flags |= 1;
    }
    return series | (off << 8) | (flags << 16);
}

struct Prefetch {
    float2 u;     // basis sample, element w = tid (threads 0 .. kSerLen-1)
    float2 t;     // target of row tid - 128 (threads 128 .. 128 + R - 1)
    bool urow, trow;
};

template <int R>
__device__ __forceinline__ Prefetch prefetch_stage(const GramProblem &pr, int64_t n0, int T)
{
    Prefetch f{};
    const int tid = threadIdx.x;
    if (tid < kSerLen) {
        const int64_t j = n0 - (T - 1) + tid;
        f.urow = tid < R + T - 1 && j >= 0 && j < pr.n;
        if (f.urow) f.u = pr.u[j];
    }
    if (tid >= 128 && tid < 128 + R) {
        const int64_t j = n0 + (tid - 128);
        f.trow = j < pr.n;
        if (f.trow && pr.t) f.t = pr.t[j];
    }
    return f;
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

// Convert the prefetched samples of a stage into the series arrays.
template <int FMT, int R>
__device__ __forceinline__ void stage_series(unsigned char *stg, const Prefetch &f, int T, int B)
{
    const int tid = threadIdx.x;
    if (tid < kSerLen) {
        const float r = fmaf(f.u.x, f.u.x, f.u.y * f.u.y);
        float p = 1.f;
        for (int b = 0; b < B; ++b) {   // psi_b = |u|^{2b} u, low order first
            put_series<FMT>(stg, 2 * b, tid, f.urow ? p * f.u.x : 0.f);
            put_series<FMT>(stg, 2 * b + 1, tid, f.urow ? p * f.u.y : 0.f);
            p *= r;
        }
    }
    if (tid >= 128 && tid < 128 + R) {
        const int w = tid - 128 + (T - 1);
        put_series<FMT>(stg, 12, w, f.trow ? f.t.x : 0.f);
        put_series<FMT>(stg, 13, w, f.trow ? f.t.y : 0.f);
        put_series<FMT>(stg, 14, w, f.trow ? 1.f : 0.f);
    }
}

// One 16-byte chunk (rows ch*EPC .. +EPC) of real-form column c, hi and lo.
template <int FMT>
__device__ __forceinline__ void make_chunk(const unsigned char *stg, int cm, int ch, int nvalid, uint4 &H, uint4 &L)
{
    const int series = cm & 0xFF, off = (cm >> 8) & 0xFF, flags = cm >> 16;
    const unsigned char *base = stg + series * kSerBytes;
    uint32_t h[4], l[4];
    if constexpr (FMT == kFmtBF16) {
        const int o = ch * 8 + off;
        const uint32_t *hw = reinterpret_cast<const uint32_t *>(base) + ((o & 1) ? kSerLen / 2 + (o - 1) / 2 : o / 2);
        const uint32_t *lw = hw + kSerLen;   // lo arrays follow the two hi arrays
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = hw[q];
            l[q] = lw[q];
        }
        if (flags & 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] ^= 0x80008000u;
                l[q] ^= 0x80008000u;
            }
        }
        if (nvalid < 64) {   // last stage of the problem: rows past the end are zero
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r0 = ch * 8 + 2 * q;
                const uint32_t m = (r0 < nvalid ? 0x0000FFFFu : 0u) | (r0 + 1 < nvalid ? 0xFFFF0000u : 0u);
                h[q] &= m;
                l[q] &= m;
            }
        }
    } else {
        const int o = ch * 4 + off;
        const uint32_t *hw = reinterpret_cast<const uint32_t *>(base) + o;
        const uint32_t *lw = hw + kSerLen;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = hw[q];
            l[q] = lw[q];
        }
        if (flags & 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] ^= 0x80000000u;
                l[q] ^= 0x80000000u;
            }
        }
        if (nvalid < 32) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (ch * 4 + q >= nvalid) h[q] = l[q] = 0u;
        }
    }
    if (flags & 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = l[q] = 0u;
    }
    H = make_uint4(h[0], h[1], h[2], h[3]);
    L = make_uint4(l[0], l[1], l[2], l[3]);
}

// Named barrier 1 over the eight generator warps, with an OR vote of `pred`.
__device__ __forceinline__ bool gen_sync_or(bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
    return r != 0;
}

// Warp roles: warps 0-7 generate operands and own the FP32 running sums;
// warp 8 (lane 0) issues the MMAs.  Barriers: full[s] (8 generator arrivals:
// stage s written), empty[s] (MMA commit: stage s consumed), chunk_done (MMA
// commit after a chunk's last stage), tmem_free (8 generator arrivals: the
// chunk has been drained from tensor memory).
template <int FMT>
__global__ void __launch_bounds__(kGramThreads + 32, 1) gram_tc_kernel(GramArgs a)
{
    constexpr int R = (FMT == kFmtBF16) ? 64 : 32;    // rows per stage: 128 bytes per operand row
    constexpr int NK = 4;                             // MMAs along K per stage (K = 16 bf16 / 8 tf32)
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stages = smem;
    unsigned char *staging = smem + kStages * kStageBytes;              // 2 x kStagingBytes
    int *colmap = reinterpret_cast<int *>(staging + 2 * kStagingBytes);  // [256]
    float *d1sum = reinterpret_cast<float *>(colmap + 256);               // [128][kD1Cols]
    uint64_t *full = reinterpret_cast<uint64_t *>(d1sum + 128 * kD1Cols);
    uint64_t *empty = full + kStages;
    uint64_t *chunk_done = empty + kStages;
    uint64_t *tmem_free = chunk_done + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_free + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int prob = blockIdx.x / a.cpp, chunk = blockIdx.x % a.cpp;
    const GramProblem pr = a.probs[prob];
    const int K = a.K, C = 2 * K + 2, T = a.T, B = a.Bp > a.Bq ? a.Bp : a.Bq;
    const bool two = C > 128;
    const int N0 = ((C + 15) / 16) * 16;
    const int N1 = two ? N0 - 128 : 0;
    const int64_t nblk = (pr.n + R - 1) / R;
    const int64_t b0 = nblk * chunk / a.cpp, b1 = nblk * (chunk + 1) / a.cpp;
    const int nits = (int)(b1 - b0);
    const int nchunks = (nits + kChunk - 1) / kChunk;

    for (int i = tid; i < kStages * kStageBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(stages)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int c = tid; c < 256; c += blockDim.x) colmap[c] = c < C ? column_map(c, K, a.Bp, T) : 0;
    for (int i = tid; i < 128 * kD1Cols; i += blockDim.x) d1sum[i] = 0.f;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(&full[s]), 8);
            mbar_init(smem_addr(&empty[s]), 1);
        }
        mbar_init(smem_addr(chunk_done), 1);
        mbar_init(smem_addr(tmem_free), 8);
        fence_barrier_init();
    }
    if (warp == 8) {
        tmem_alloc(smem_addr(tmem_slot), 512);
        tmem_relinquish();
    }
    if (nits > 0 && warp < 8) stage_series<FMT, R>(staging, prefetch_stage<R>(pr, b0 * R, T), T, B);
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool failed = false;
    if (warp == 8) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc0 = umma_idesc(FMT, 128, N0);
            const uint32_t idesc1 = two ? umma_idesc(FMT, 128, N1) : 0u;
            int commits = 0;
            bool issued_all = true;
            for (int it = 0; it < nits; ++it) {
                const int s = it % kStages;
                if (!mbar_wait(smem_addr(&full[s]), (uint32_t)((it / kStages) & 1), a.status)) {
                    issued_all = false;
                    break;
                }
                if (it > 0 && it % kChunk == 0 &&
                    !mbar_wait(smem_addr(tmem_free), (uint32_t)((it / kChunk - 1) & 1), a.status)) {
                    issued_all = false;
                    break;
                }
                tc_fence_after_sync();
                const uint32_t hb = smem_addr(stages + s * kStageBytes), lb = hb + kBuf;
                const uint32_t pa[3] = {hb, hb, lb}, pb[3] = {hb, lb, hb};   // hi*hi + hi*lo + lo*hi
                uint32_t accumulate = (it % kChunk == 0) ? 0u : 1u;
#pragma unroll
                for (int kk = 0; kk < NK; ++kk) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const uint32_t ka = pa[q] + kk * 32, kb = pb[q] + kk * 32;
                        if constexpr (FMT == kFmtBF16) {
                            umma_bf16(tmem, umma_desc_sw128(ka), umma_desc_sw128(kb), idesc0, accumulate);
                            if (two)
                                umma_bf16(tmem + (uint32_t)N0, umma_desc_sw128(ka + kTile),
                                          umma_desc_sw128(kb + kTile), idesc1, accumulate);
                        } else {
                            umma_tf32(tmem, umma_desc_sw128(ka), umma_desc_sw128(kb), idesc0, accumulate);
                            if (two)
                                umma_tf32(tmem + (uint32_t)N0, umma_desc_sw128(ka + kTile),
                                          umma_desc_sw128(kb + kTile), idesc1, accumulate);
                        }
                        accumulate = 1;
                    }
                }
                umma_commit(smem_addr(&empty[s]));
                if ((it + 1) % kChunk == 0 || it + 1 == nits) {
                    umma_commit(smem_addr(chunk_done));
                    ++commits;
                }
            }
            // Every MMA issued must be complete before tensor memory is released.
            // Normally the last chunk's commit covers them all (the generators
            // wait on that same phase).  After a failure, commit once more and
            // wait for that phase.
            if (issued_all) {
                if (nits > 0) mbar_wait(smem_addr(chunk_done), (uint32_t)((commits - 1) & 1), a.status);
            } else {
                umma_commit(smem_addr(chunk_done));
                mbar_wait(smem_addr(chunk_done), (uint32_t)(commits & 1), a.status);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ generators
        const int quarter = warp & 3, half = warp >> 2;
        const int row = 32 * quarter + lane;   // tensor-memory lane
        const uint32_t lane_taddr = tmem + ((uint32_t)(32 * quarter) << 16);
        float acc[kAccCols];
#pragma unroll
        for (int i = 0; i < kAccCols; ++i) acc[i] = 0.f;

        auto drain = [&](int c) -> bool {
            const bool ok = mbar_wait(smem_addr(chunk_done), (uint32_t)(c & 1), a.status);
            tc_fence_after_sync();
            if (ok) {
#pragma unroll
                for (int cc = 0; cc < kAccCols / 8; ++cc) {
                    if (half * kAccCols + cc * 8 < N0) {
                        float v[8];
                        tmem_ld8(lane_taddr + (uint32_t)(half * kAccCols + cc * 8), v);
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc[cc * 8 + q] += v[q];
                    }
                }
                if (two) {
                    float *d1row = d1sum + row * kD1Cols + half * kD1Half;
#pragma unroll
                    for (int cc = 0; cc < kD1Half / 8; ++cc) {
                        if (half * kD1Half + cc * 8 < N1) {
                            float v[8];
                            tmem_ld8(lane_taddr + (uint32_t)(N0 + half * kD1Half + cc * 8), v);
#pragma unroll
                            for (int q = 0; q < 8; ++q) d1row[cc * 8 + q] += v[q];
                        }
                    }
                }
            }
            tc_fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(tmem_free));
            return ok;
        };

        for (int it = 0; it < nits; ++it) {
            const int s = it % kStages;
            bool ok = true;
            if (it >= kStages) ok = mbar_wait(smem_addr(&empty[s]), (uint32_t)(((it / kStages) - 1) & 1), a.status);
            if (gen_sync_or(!ok)) {   // also: every generator finished the previous stage
                failed = true;
                break;
            }
            const int64_t n0 = (b0 + it) * R;
            Prefetch nxt{};
            if (it + 1 < nits) nxt = prefetch_stage<R>(pr, n0 + R, T);   // in flight during generation
            const unsigned char *stg = staging + (it & 1) * kStagingBytes;
            unsigned char *hi = stages + s * kStageBytes;
            unsigned char *lo = hi + kBuf;
            const int64_t rem = pr.n - n0;
            const int nvalid = rem < R ? (int)rem : R;
            for (int task = tid; task < C * 8; task += kGramThreads) {
                const int c = task >> 3, ch = task & 7;
                uint4 H, L;
                make_chunk<FMT>(stg, colmap[c], ch, nvalid, H, L);
                const uint32_t off = sw128_offset(c, ch);
                *reinterpret_cast<uint4 *>(hi + off) = H;
                *reinterpret_cast<uint4 *>(lo + off) = L;
            }
            if (it + 1 < nits) stage_series<FMT, R>(staging + ((it + 1) & 1) * kStagingBytes, nxt, T, B);
            fence_async_shared();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&full[s]));
            if (it > 0 && it % kChunk == 0) {   // drain the previous chunk while this stage is queued
                const bool okd = drain(it / kChunk - 1);
                if (gen_sync_or(!okd)) {
                    failed = true;
                    break;
                }
            }
        }
        if (!failed && nits > 0) failed = gen_sync_or(!drain(nchunks - 1));

        float *part = a.partials + (size_t)blockIdx.x * kGramRows * kGramCols;
        const bool zero = failed || nits == 0;
#pragma unroll
        for (int i = 0; i < kAccCols; ++i) {
            const int c = half * kAccCols + i;   // column of D0
            if (c < N0) part[(size_t)row * kGramCols + c] = zero ? 0.f : acc[i];
        }
        for (int i = 0; i < kD1Half; ++i) {
            const int c = half * kD1Half + i;   // column of D1 (real-form column 128 + c)
            if (c < N1) part[(size_t)(128 + row) * kGramCols + 128 + c] = zero ? 0.f : d1sum[row * kD1Cols + c];
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

size_t gram_tc_smem()
{
    return 1024 + (size_t)kStages * kStageBytes + 2 * (size_t)kStagingBytes + 256 * 4 + 128 * kD1Cols * 4 + 128;
}

// ------------------------------------------------------------------ FP32 CUDA cores
// Each CTA stages 64 rows of A (row-major, 256 padded columns, FP32) in shared
// memory; thread t owns one 8 x 8 block (I, J), I <= J, of the upper triangle
// of S and accumulates it over the rows.
constexpr int kF32Rows = 64;
constexpr int kF32Threads = 352;   // >= 25 * 26 / 2 = 325 diagonal-and-upper 8 x 8 blocks

__global__ void __launch_bounds__(kF32Threads, 1) gram_fp32_kernel(GramArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_f[];
    float *Atile = reinterpret_cast<float *>(smem_f);                    // [kF32Rows][256]
    float2 *psi = reinterpret_cast<float2 *>(Atile + kF32Rows * 256);  // [kMaxB][kPsiStride]
    float2 *tv = psi + kMaxB * kPsiStride;

    const int tid = threadIdx.x;
    const int prob = blockIdx.x / a.cpp, chunk = blockIdx.x % a.cpp;
    const GramProblem pr = a.probs[prob];
    const int K = a.K, C = 2 * K + 2, T = a.T, B = a.Bp > a.Bq ? a.Bp : a.Bq;
    const int nb8 = (C + 7) / 8;
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
        stage_basis<kF32Rows>(pr, n0, T, B, psi, tv);
        __syncthreads();
        for (int e = tid; e < kF32Rows * 256; e += kF32Threads) {
            const int rr = e >> 8, c = e & 255;
            float v = 0.f;
            if (c < C) v = column_value(decode_column(c, K, a.Bp, T), psi, tv, rr, T, n0 + rr < pr.n);
            Atile[e] = v;
        }
        __syncthreads();
        if (I >= 0) {
            for (int rr = 0; rr < kF32Rows; ++rr) {
                const float4 *row = reinterpret_cast<const float4 *>(Atile + rr * 256);
                const float4 a0 = row[2 * I], a1 = row[2 * I + 1], b0v = row[2 * J], b1v = row[2 * J + 1];
                const float ai[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bj[8] = {b0v.x, b0v.y, b0v.z, b0v.w, b1v.x, b1v.y, b1v.z, b1v.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(ai[i], bj[j], acc[i][j]);
            }
        }
    }
    float *part = a.partials + (size_t)blockIdx.x * kGramRows * kGramCols;
    if (I >= 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = 8 * I + i, c = 8 * J + j;
                if (r < kGramRows && c < kGramCols) part[(size_t)r * kGramCols + c] = acc[i][j];
            }
    }
}

size_t gram_fp32_smem() { return (size_t)kF32Rows * 256 * 4 + (kMaxB * kPsiStride + 64) * 8; }

cudaError_t launch_gram(int precision, const GramArgs &a, cudaStream_t s)
{
    const int grid = a.nprob * a.cpp;
    if (grid <= 0) return cudaSuccess;
    if (precision == kPrecFP32) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(gram_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)gram_fp32_smem());
            if (e != cudaSuccess) return e;
            attr = true;
        }
        gram_fp32_kernel<<<grid, kF32Threads, gram_fp32_smem(), s>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    auto kern = precision == kPrecBF16x3 ? gram_tc_kernel<kFmtBF16> : gram_tc_kernel<kFmtTF32>;
    static bool attr_set[2] = {false, false};
    const int ai = precision == kPrecBF16x3 ? 0 : 1;
    if (!attr_set[ai]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem());
        if (e != cudaSuccess) return e;
        attr_set[ai] = true;
    }
    kern<<<grid, kGramThreads + 32, gram_tc_smem(), s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace dpd
