/*
 * Portable SIMD + OpenMP CPU filter (contract in include/dpd_cpu.h).
 *
 * Arithmetic: per tap k the main and conjugate branches are regrouped into the
 * widely-linear form used by the GPU kernels,
 *   sum_p h_{p,k} |x|^{p-1} x + sum_q hbar_{q,k} |x|^{q-1} conj(x)
 *     = (P0(r) a + P1(r) b) + j (P2(r) a + P3(r) b),   x = a + j b, r = |x|^2,
 * four real polynomials of degree B-1 in r evaluated by Horner's rule.
 *
 * Data movement: each OpenMP thread takes blocks of kBlock samples, splits the
 * block and the 8 samples before it into real, imaginary and |x|^2 arrays
 * (zero before x[0]), and produces 12 outputs at a time from three 4-wide
 * vectors per quantity.  The window of tap k is the same arrays read k samples earlier
 * -- an unaligned vector load, the portable form of the paper's vext-style
 * regrouping of neighbouring vectors.  GCC vector extensions compile to NEON
 * on AArch64 and to SSE on x86-64; no architecture-specific code.
 */
#include "../../include/dpd_cpu.h"

#include <omp.h>
#include <string.h>

typedef float v4f __attribute__((vector_size(16)));

enum { kMaxB = 6, kMaxT = 8, kHist = 8, kBlock = 4096, kVec = 3, kStep = 4 * kVec };

static inline v4f load4(const float *p)
{
    v4f v;
    memcpy(&v, p, sizeof v);
    return v;
}

static inline v4f splat(float s) { return (v4f){s, s, s, s}; }

/*
 * kStep = 12 outputs from the split arrays (element 0 is the block's first
 * sample, elements -1 .. -kHist its history): three 4-wide vectors per
 * quantity, so each Horner step has 12 independent FMA chains (enough to keep
 * the vector FMA pipes of a core busy despite their latency).  BB, the number of
 * powers, is a compile-time constant in each instance so that the Horner loop
 * unrolls; T stays a run-time loop.
 */
#define DPD_CPU_BLOCK(BB)                                                                              \
    static void filter_block_##BB(int T, const float tab[kMaxT][kMaxB][4], float cr, float ci,         \
                                  const float *re, const float *im, const float *rr, int len, float *y) \
    {                                                                                                  \
        for (int j = 0; j < len; j += kStep) {                                                         \
            v4f yr[kVec], yi[kVec];                                                                    \
            for (int v = 0; v < kVec; ++v) {                                                           \
                yr[v] = splat(cr);                                                                     \
                yi[v] = splat(ci);                                                                     \
            }                                                                                          \
            for (int k = 0; k < T; ++k) {                                                              \
                const int o = j - k;                                                                   \
                v4f a[kVec], b[kVec], r[kVec], p0[kVec], p1[kVec], p2[kVec], p3[kVec];                 \
                for (int v = 0; v < kVec; ++v) {                                                       \
                    a[v] = load4(re + o + 4 * v);                                                      \
                    b[v] = load4(im + o + 4 * v);                                                      \
                    r[v] = load4(rr + o + 4 * v);                                                      \
                    p0[v] = splat(tab[k][BB - 1][0]);                                                  \
                    p1[v] = splat(tab[k][BB - 1][1]);                                                  \
                    p2[v] = splat(tab[k][BB - 1][2]);                                                  \
                    p3[v] = splat(tab[k][BB - 1][3]);                                                  \
                }                                                                                      \
                for (int m = BB - 2; m >= 0; --m) {                                                    \
                    const v4f c0 = splat(tab[k][m][0]), c1 = splat(tab[k][m][1]);                      \
                    const v4f c2 = splat(tab[k][m][2]), c3 = splat(tab[k][m][3]);                      \
                    for (int v = 0; v < kVec; ++v) {                                                   \
                        p0[v] = p0[v] * r[v] + c0;                                                     \
                        p1[v] = p1[v] * r[v] + c1;                                                     \
                        p2[v] = p2[v] * r[v] + c2;                                                     \
                        p3[v] = p3[v] * r[v] + c3;                                                     \
                    }                                                                                  \
                }                                                                                      \
                for (int v = 0; v < kVec; ++v) {                                                       \
                    yr[v] += p0[v] * a[v] + p1[v] * b[v];                                              \
                    yi[v] += p2[v] * a[v] + p3[v] * b[v];                                              \
                }                                                                                      \
            }                                                                                          \
            float outr[kStep], outi[kStep];                                                            \
            memcpy(outr, yr, sizeof outr);                                                             \
            memcpy(outi, yi, sizeof outi);                                                             \
            const int cnt = len - j < kStep ? len - j : kStep;                                         \
            float *yp = y + 2 * j;                                                                     \
            for (int q = 0; q < cnt; ++q) {                                                            \
                yp[2 * q] = outr[q];                                                                   \
                yp[2 * q + 1] = outi[q];                                                               \
            }                                                                                          \
        }                                                                                              \
    }
DPD_CPU_BLOCK(1)
DPD_CPU_BLOCK(2)
DPD_CPU_BLOCK(3)
DPD_CPU_BLOCK(4)
DPD_CPU_BLOCK(5)
DPD_CPU_BLOCK(6)
#undef DPD_CPU_BLOCK

static void filter_block(int B, int T, const float tab[kMaxT][kMaxB][4], float cr, float ci, const float *re,
                         const float *im, const float *rr, int len, float *y)
{
    switch (B) {
    case 1: filter_block_1(T, tab, cr, ci, re, im, rr, len, y); break;
    case 2: filter_block_2(T, tab, cr, ci, re, im, rr, len, y); break;
    case 3: filter_block_3(T, tab, cr, ci, re, im, rr, len, y); break;
    case 4: filter_block_4(T, tab, cr, ci, re, im, rr, len, y); break;
    case 5: filter_block_5(T, tab, cr, ci, re, im, rr, len, y); break;
    default: filter_block_6(T, tab, cr, ci, re, im, rr, len, y); break;
    }
}

int dpd_cpu_max_threads(void) { return omp_get_max_threads(); }

int dpd_cpu_apply(int P, int Q, int M, const float *h, const float *x, float *y, int64_t n, int threads)
{
    if (P < 1 || P > 11 || !(P & 1) || Q < 0 || Q > 11 || (Q && !(Q & 1)) || M < 0 || M >= kMaxT || n < 0 ||
        threads < 0)
        return -1;
    if (n == 0) return 0;
    if (!h || !x || !y) return -1;
    if ((const char *)y < (const char *)(x + 2 * n) && (const char *)x < (const char *)(y + 2 * n)) return -1;
    const int Bp = (P + 1) / 2, Bq = Q ? (Q + 1) / 2 : 0, B = Bp > Bq ? Bp : Bq, T = M + 1;
    const int K = (Bp + Bq) * T + 1;
    /* tab[k][m] = {P0, P1, P2, P3} of tap k, power r^m */
    float tab[kMaxT][kMaxB][4];
    memset(tab, 0, sizeof tab);
    for (int k = 0; k < T; ++k)
        for (int m = 0; m < B; ++m) {
            const float Ar = m < Bp ? h[2 * (m * T + k)] : 0.f, Ai = m < Bp ? h[2 * (m * T + k) + 1] : 0.f;
            const float Cr = m < Bq ? h[2 * ((Bp + m) * T + k)] : 0.f;
            const float Ci = m < Bq ? h[2 * ((Bp + m) * T + k) + 1] : 0.f;
            tab[k][m][0] = Ar + Cr;      /* P0 = Re(A + C) */
            tab[k][m][1] = -(Ai - Ci);   /* P1 = -Im(A - C) */
            tab[k][m][2] = Ai + Ci;      /* P2 = Im(A + C) */
            tab[k][m][3] = Ar - Cr;      /* P3 = Re(A - C) */
        }
    const float cr = h[2 * (K - 1)], ci = h[2 * (K - 1) + 1];
    const int64_t nblk = (n + kBlock - 1) / kBlock;
    const int nth = threads > 0 ? threads : omp_get_max_threads();

#pragma omp parallel for schedule(static) num_threads(nth)
    for (int64_t blk = 0; blk < nblk; ++blk) {
        float re[kHist + kBlock + kStep], im[kHist + kBlock + kStep], rr[kHist + kBlock + kStep];
        const int64_t s0 = blk * kBlock;
        const int len = (int)(n - s0 < kBlock ? n - s0 : kBlock);
        for (int i = 0; i < kHist + len; ++i) {   /* element i is sample s0 - kHist + i */
            const int64_t g = s0 - kHist + i;
            const float a = g >= 0 ? x[2 * g] : 0.f, b = g >= 0 ? x[2 * g + 1] : 0.f;
            re[i] = a;
            im[i] = b;
            rr[i] = a * a + b * b;
        }
        for (int i = kHist + len; i < kHist + kBlock + kStep; ++i) re[i] = im[i] = rr[i] = 0.f;
        filter_block(B, T, tab, cr, ci, re + kHist, im + kHist, rr + kHist, len, y + 2 * s0);
    }
    return 0;
}
