/*
 * ORACLE -- test infrastructure only.  Nothing in the product links this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Near-field direct image sum (Sec. 2.1, Eq. 3 with the kernel of Eq. 1):
 *
 *     phi_near(y) = sum_{p in images} sum_i q_i K(y - x_i + p),
 *     K(r) = 1/|r|  (r != 0),   K(0) = 0,
 *
 * with the image vectors p = (i1 d1, i2 d2, i3 d3), |i_k| <= K_k (Eq. 2 restricted
 * to the block Omega_b of (2K1+1)(2K2+1)(2K3+1) boxes), and its gradient with
 * respect to y,
 *
 *     grad phi_near(y) = - sum_p sum_i q_i (y - x_i + p) / |y - x_i + p|^3.
 *
 * Plain loops in double precision, one target at a time; targets are spread
 * over OpenMP threads, which does not change the order of any target's sum.
 *
 * With Rb > 0 the near set is trimmed to the ball (algorithm "get", step 2): a source
 * image x_i - p (sources are indexed x_j = x_i - p, Sec. 2.1) is kept only if
 * |x_i - p| <= Rb.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_near_sum_ball(int64_t n_targets, const double *y,
                          int64_t n_sources, const double *x, const double *q,
                          const double *d, const int32_t *K, double Rb,
                          double *phi, double *grad);

void oracle_near_sum(int64_t n_targets, const double *y,
                     int64_t n_sources, const double *x, const double *q,
                     const double *d, const int32_t *K,
                     double *phi, double *grad)
{
    oracle_near_sum_ball(n_targets, y, n_sources, x, q, d, K, 0.0, phi, grad);
}

void oracle_near_sum_ball(int64_t n_targets, const double *y,
                          int64_t n_sources, const double *x, const double *q,
                          const double *d, const int32_t *K, double Rb,
                          double *phi, double *grad)
{
    int64_t j;
#pragma omp parallel for schedule(dynamic, 8)
    for (j = 0; j < n_targets; ++j) {
        double s = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int i1 = -K[0]; i1 <= K[0]; ++i1)
        for (int i2 = -K[1]; i2 <= K[1]; ++i2)
        for (int i3 = -K[2]; i3 <= K[2]; ++i3) {
            const double p1 = i1 * d[0], p2 = i2 * d[1], p3 = i3 * d[2];
            for (int64_t i = 0; i < n_sources; ++i) {
                if (Rb > 0.0) {
                    const double s1 = x[3 * i + 0] - p1, s2 = x[3 * i + 1] - p2, s3 = x[3 * i + 2] - p3;
                    if (s1 * s1 + s2 * s2 + s3 * s3 > Rb * Rb)
                        continue;           /* outside the ball S_b: part of the far field */
                }
                const double r1 = y[3 * j + 0] - x[3 * i + 0] + p1;
                const double r2 = y[3 * j + 1] - x[3 * i + 1] + p2;
                const double r3 = y[3 * j + 2] - x[3 * i + 2] + p3;
                const double rr = r1 * r1 + r2 * r2 + r3 * r3;
                if (rr == 0.0)
                    continue;               /* K(0) = 0, Eq. 1 */
                const double r = sqrt(rr);
                const double k = 1.0 / r;
                s += q[i] * k;
                if (grad) {
                    const double k3 = q[i] * k / rr;
                    gx -= k3 * r1;
                    gy -= k3 * r2;
                    gz -= k3 * r3;
                }
            }
        }
        phi[j] = s;
        if (grad) {
            grad[3 * j + 0] = gx;
            grad[3 * j + 1] = gy;
            grad[3 * j + 2] = gz;
        }
    }
}
