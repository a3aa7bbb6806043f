/*
 * Portable SIMD + OpenMP CPU implementation of the APH DPD filter (Eq. 1 /
 * Algorithm 1), the counterpart of the paper's multicore-CPU design (Sec. 3.2.2
 * vectorised across samples, Sec. 3.3.3 tap windows regrouped from registers):
 * a like-for-like CPU comparison for the GPU library.  FP32 throughout.
 *
 * Not the correctness oracle (that is the FP64 code under oracle/); this
 * library is a CPU product path and is checked against the oracle like the
 * GPU one.
 */
#ifndef DPD_CPU_H
#define DPD_CPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * y = DPD(x) for n complex samples, zero history before x[0].
 *   P, Q, M : as dpd_create (odd P, Q <= 11 or Q = 0, 0 <= M <= 7).
 *   h       : K = (B_p + B_q) (M + 1) + 1 complex coefficients as interleaved
 *             floats (re, im), stacking order of Sec. 2.2.
 *   x, y    : 2 n floats each (interleaved complex), not overlapping.
 *   threads : OpenMP threads (0: the runtime's default).
 * Returns 0, or -1 for invalid arguments (nothing written).  n == 0 returns 0.
 */
int dpd_cpu_apply(int P, int Q, int M, const float *h, const float *x, float *y, int64_t n, int threads);

/* Number of threads an OpenMP parallel region uses with threads = 0. */
int dpd_cpu_max_threads(void);

#ifdef __cplusplus
}
#endif

#endif /* DPD_CPU_H */
