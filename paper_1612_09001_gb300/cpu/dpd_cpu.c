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
 * (zero before x[0]), and produces 8 outputs at a time from two 4-wide vectors
 * per quantity.  The window of tap k is the same arrays read k samples earlier
 * -- an unaligned vector load, the portable form of the paper's vext-style
 * regrouping of neighbouring vectors.  GCC vector extensions compile to NEON
 * on AArch64 and to SSE on x86-64; no architecture-specific code.
 */
#include "../../include/dpd_cpu.h"

#include <omp.h>
#include <string.h>

typedef float v4f __attribute__((vector_size(16)));

enum { kMaxB = 6, kMaxT = 8, kHist = 8, kBlock = 4096 };

static inline v4f load4(const float *p)
{
    v4f v;
    memcpy(&v, p, sizeof v);
    return v;
}

static inline v4f splat(float s) { return (v4f){s, s, s, s}; }

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
        float re[kHist + kBlock + 8], im[kHist + kBlock + 8], rr[kHist + kBlock + 8];
        const int64_t s0 = blk * kBlock;
        const int len = (int)(n - s0 < kBlock ? n - s0 : kBlock);
        for (int i = 0; i < kHist + len; ++i) {   /* element i is sample s0 - kHist + i */
            const int64_t g = s0 - kHist + i;
            const float a = g >= 0 ? x[2 * g] : 0.f, b = g >= 0 ? x[2 * g + 1] : 0.f;
            re[i] = a;
            im[i] = b;
            rr[i] = a * a + b * b;
        }
        for (int i = kHist + len; i < kHist + kBlock + 8; ++i) re[i] = im[i] = rr[i] = 0.f;
        for (int j = 0; j < len; j += 8) {
            v4f yr0 = splat(cr), yi0 = splat(ci), yr1 = splat(cr), yi1 = splat(ci);
            for (int k = 0; k < T; ++k) {
                const int o = kHist + j - k;
                const v4f a0 = load4(re + o), b0 = load4(im + o), r0 = load4(rr + o);
                const v4f a1 = load4(re + o + 4), b1 = load4(im + o + 4), r1 = load4(rr + o + 4);
                v4f p00 = splat(tab[k][B - 1][0]), p01 = splat(tab[k][B - 1][1]);
                v4f p02 = splat(tab[k][B - 1][2]), p03 = splat(tab[k][B - 1][3]);
                v4f p10 = p00, p11 = p01, p12 = p02, p13 = p03;
                for (int m = B - 2; m >= 0; --m) {
                    const v4f c0 = splat(tab[k][m][0]), c1 = splat(tab[k][m][1]);
                    const v4f c2 = splat(tab[k][m][2]), c3 = splat(tab[k][m][3]);
                    p00 = p00 * r0 + c0;
                    p01 = p01 * r0 + c1;
                    p02 = p02 * r0 + c2;
                    p03 = p03 * r0 + c3;
                    p10 = p10 * r1 + c0;
                    p11 = p11 * r1 + c1;
                    p12 = p12 * r1 + c2;
                    p13 = p13 * r1 + c3;
                }
                yr0 += p00 * a0 + p01 * b0;
                yi0 += p02 * a0 + p03 * b0;
                yr1 += p10 * a1 + p11 * b1;
                yi1 += p12 * a1 + p13 * b1;
            }
            float outr[8], outi[8];
            memcpy(outr, &yr0, 16);
            memcpy(outr + 4, &yr1, 16);
            memcpy(outi, &yi0, 16);
            memcpy(outi + 4, &yi1, 16);
            const int cnt = len - j < 8 ? len - j : 8;
            float *yp = y + 2 * (s0 + j);
            for (int q = 0; q < cnt; ++q) {
                yp[2 * q] = outr[q];
                yp[2 * q + 1] = outi[q];
            }
        }
    }
    return 0;
}
