/*
 * CPU oracle for SOFA's exact k-NN hot path (Schaefer et al., "Fast and Exact
 * Similarity Search in less than a Blink of an Eye").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA library; the two never call
 * each other.
 *
 * Everything here is plain, slow, sequential FP64 arithmetic written from the
 * definitions in the paper:
 *   - z-normalisation and the z-normalised Euclidean distance  (Sec. II, Def. z-ED)
 *   - the discrete Fourier transform                           (Sec. IV-SFA, Alg. 1/2, Eq. 1)
 *   - brute-force squared distances for the exact k-NN          (Sec. II, NN problem)
 *
 * Build with -ffp-contract=off so that no multiply-add is fused: every sum is
 * the left-to-right sequence of IEEE operations written below, on any CPU.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of host threads OpenMP will use (1 when built without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * z-normalisation (Sec. II, Definition "z-normalized Euclidean distance"):
 *   mu    = (sum_t x_t) / n                      left-to-right FP64 sum
 *   sigma = sqrt((sum_t (x_t - mu)^2) / n)       population deviation, FP64
 *   Z_t   = fp32( (x_t - mu) * (1 / sigma) )     rounded to nearest
 * A constant series (sigma == 0) maps to the all-zero series.
 * x and z are N x n row-major; mu_out / sigma_out may be NULL.
 */
void orc_znorm(const float* x, int64_t N, int32_t n, float* z,
               double* mu_out, double* sigma_out) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < N; ++i) {
    const float* r = x + i * (int64_t)n;
    float* o = z + i * (int64_t)n;
    double s = 0.0;
    for (int32_t t = 0; t < n; ++t) s = s + (double)r[t];
    double mu = s / (double)n;
    double ss = 0.0;
    for (int32_t t = 0; t < n; ++t) {
      double d = (double)r[t] - mu;
      ss = ss + d * d;
    }
    double sigma = sqrt(ss / (double)n);
    if (mu_out) mu_out[i] = mu;
    if (sigma_out) sigma_out[i] = sigma;
    if (sigma == 0.0) {
      for (int32_t t = 0; t < n; ++t) o[t] = 0.0f;
      continue;
    }
    double inv = 1.0 / sigma;
    for (int32_t t = 0; t < n; ++t) o[t] = (float)(((double)r[t] - mu) * inv);
  }
}

/*
 * Orthonormal DFT of one real series (Alg. 1 step 1, Alg. 2 step 1, Eq. 1):
 *   X_k = n^{-1/2} * sum_t Z_t * exp(-2 pi i k t / n),   k = 0 .. floor(n/2).
 * With this scaling Parseval holds exactly, which is what makes Eq. (1) a
 * lower bound.  The angle is formed from (k*t mod n) so it stays in [0, 2pi).
 * re / im receive floor(n/2)+1 values each.
 */
void orc_dft(const float* z, int32_t n, double* re, double* im) {
  const double two_pi = 6.283185307179586476925286766559;
  double scale = 1.0 / sqrt((double)n);
  for (int32_t k = 0; k <= n / 2; ++k) {
    double a = 0.0, b = 0.0;
    for (int32_t t = 0; t < n; ++t) {
      int64_t m = ((int64_t)k * (int64_t)t) % (int64_t)n;
      double ang = two_pi * (double)m / (double)n;
      a = a + (double)z[t] * cos(ang);
      b = b - (double)z[t] * sin(ang);
    }
    re[k] = a * scale;
    im[k] = b * scale;
  }
}

/* DFT of N rows (OpenMP over rows).  re/im are N x (n/2+1). */
void orc_dft_rows(const float* z, int64_t N, int32_t n, double* re, double* im) {
  int64_t i;
  int32_t K = n / 2 + 1;
#pragma omp parallel for schedule(static)
  for (i = 0; i < N; ++i)
    orc_dft(z + i * (int64_t)n, n, re + i * (int64_t)K, im + i * (int64_t)K);
}

/*
 * Squared Euclidean distances between one query and N series (Sec. II, NN
 * problem; the k-NN extension of Sec. IV "Exact Similarity Search"):
 *   d2[i] = sum_t (q_t - X_{i,t})^2,  each difference and square in FP64,
 *   summed left to right.  Inputs are already z-normalised fp32 series.
 */
void orc_sqdist(const float* X, int64_t N, int32_t n, const float* q, double* d2) {
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < N; ++i) {
    const float* r = X + i * (int64_t)n;
    double acc = 0.0;
    for (int32_t t = 0; t < n; ++t) {
      double d = (double)q[t] - (double)r[t];
      acc = acc + d * d;
    }
    d2[i] = acc;
  }
}
