/* Direct trapezoid sum for the boundary potential (section 4, eq. TrapOrig2D
 * and its 3-D analogue).  Oracle code: test infrastructure only.
 *
 *   g(x_b) = sum_p G(|x_b - s_p|) rho_p * prod_s h_s
 *
 * over the listed source points p (the non-zero interior values of rho).
 * G(r) = |r|/2 in 1-D, log(r)/(2 pi) in 2-D and -1/(4 pi r) in 3-D (section 1).  Each sum
 * is accumulated with Neumaier's compensated summation in double precision;
 * boundary targets run in parallel with OpenMP.
 */
#include <math.h>
#include <stdint.h>

static double green(int d, double r2)
{
    const double pi = 3.14159265358979323846;
    if (d == 1) return 0.5 * sqrt(r2);               /* |r| / 2 */
    if (d == 2) return 0.5 * log(r2) / (2.0 * pi);   /* log(r) = log(r^2)/2 */
    return -1.0 / (4.0 * pi * sqrt(r2));
}

/* d: dimension (1, 2 or 3); h[d]: mesh widths;
 * nsrc sources: src_idx[nsrc*d] integer node indices, src_val[nsrc] values;
 * ntgt targets: tgt_idx[ntgt*d] integer node indices; out[ntgt] receives g. */
void oracle_boundary_direct(int d, const double *h, int64_t nsrc,
                            const int32_t *src_idx, const double *src_val,
                            int64_t ntgt, const int32_t *tgt_idx, double *out)
{
    double w = 1.0;
    for (int s = 0; s < d; ++s) w *= h[s];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < ntgt; ++t) {
        double sum = 0.0, comp = 0.0;
        for (int64_t p = 0; p < nsrc; ++p) {
            double r2 = 0.0;
            for (int s = 0; s < d; ++s) {
                double dx = (double)(tgt_idx[t * d + s] - src_idx[p * d + s]) * h[s];
                r2 += dx * dx;
            }
            double term = green(d, r2) * src_val[p];
            double nsum = sum + term;
            if (fabs(sum) >= fabs(term)) comp += (sum - nsum) + term;
            else comp += (term - nsum) + sum;
            sum = nsum;
        }
        out[t] = (sum + comp) * w;
    }
}
