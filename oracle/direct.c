/* Exact lattice sum u(n) = sum_m G(n - m) f(m) over the active points
 * (Eq. dpoissonsoln), FP64.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle; the CUDA library never links it.
 *
 * G is read from a dense table of |offset| triples, tab[(a*(V+1)+b)*(V+1)+c] =
 * G(a, b, c) for 0 <= a, b, c <= V, which the reflection symmetry of G (Sec. 2.1)
 * makes sufficient.  Each target's sum uses Neumaier's compensated summation so
 * the result carries ~1 ulp of error regardless of the number of sources.
 * Parallel over targets with OpenMP.
 *
 * pts   : n x 3 source coordinates (x, y, z), int32
 * f     : n source values
 * tgt   : nt x 3 target coordinates
 * u     : nt outputs
 * returns 0, or -1 if some offset exceeds V on an axis (u is then incomplete).
 */
#include <stdint.h>
#include <stdlib.h>

int lgf_direct_sum(const int32_t *pts, const double *f, int64_t n,
                   const double *tab, int32_t V,
                   const int32_t *tgt, int64_t nt, double *u)
{
    const int64_t W = (int64_t)V + 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t i = 0; i < nt; ++i) {
        const int32_t tx = tgt[3 * i], ty = tgt[3 * i + 1], tz = tgt[3 * i + 2];
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int32_t a = abs(tx - pts[3 * j]);
            int32_t b = abs(ty - pts[3 * j + 1]);
            int32_t d = abs(tz - pts[3 * j + 2]);
            if (a > V || b > V || d > V) { bad = 1; continue; }
            double term = tab[(a * W + b) * W + d] * f[j];
            double t = s + term;
            if ((s >= 0 ? s : -s) >= (term >= 0 ? term : -term))
                c += (s - t) + term;
            else
                c += (term - t) + s;
            s = t;
        }
        u[i] = s + c;
    }
    return bad ? -1 : 0;
}
