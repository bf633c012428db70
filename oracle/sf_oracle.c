/*
 * sf_oracle.c -- FP64 brute-force reference for adaptive KDE over a region of
 * interest (ScaleFree, arXiv 2601.20758, Sec. 3.1).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the bench
 * use it. It shares no code, header or constant table with the CUDA library.
 *
 * Everything here is the plain definition evaluated over all pairs, in double
 * precision, with no spatial index, blocking or reordering. The only
 * parallelism is an OpenMP loop over independent outputs (one query point or
 * one target position per iteration); the arithmetic for each output is the
 * sequential sum over j = 0 .. n-1 in index order.
 *
 * Build with -ffp-contract=off: every product and sum below is a separately
 * rounded IEEE double operation, so the distance d^2 is exactly
 * ((dx*dx) + (dy*dy)) + (dz*dz) with dx = (double)x_i - (double)x_j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_K_EPAN 0
#define OR_K_GAUSS3 1

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * k nearest neighbours by brute force.
 *
 * For each query index qi = q[t], the neighbours are the k points j != qi with
 * the smallest squared distance d2 = ((dx*dx)+(dy*dy))+(dz*dz) in double,
 * ties broken by the smaller original index j. The bandwidth is
 * h = (float) sqrt(d2 of the k-th neighbour) (one correctly rounded double
 * square root, then rounding to float). This is the per-point bandwidth
 * rule of the kNN configurations; the paper's own rule (Eqs. 1-6) is
 * evaluated in Python on top of or_density_at.
 *
 * nbr_out (nullable): nq*k original indices, ascending by (d2, j).
 * d2_out  (nullable): nq*k squared distances matching nbr_out.
 * Returns 0, or -1 if k < 1 or n <= k.
 */
int or_knn(const float *xyz, int64_t n, int k, const int64_t *q, int64_t nq,
           float *h_out, int64_t *nbr_out, double *d2_out) {
    if (k < 1 || n <= k) return -1;
    int64_t t;
#pragma omp parallel for schedule(dynamic, 16)
    for (t = 0; t < nq; ++t) {
        int64_t qi = q[t];
        double xi = (double)xyz[3 * qi + 0];
        double yi = (double)xyz[3 * qi + 1];
        double zi = (double)xyz[3 * qi + 2];
        double *bd = (double *)malloc(sizeof(double) * (size_t)k);
        int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == qi) continue;
            double dx = xi - (double)xyz[3 * j + 0];
            double dy = yi - (double)xyz[3 * j + 1];
            double dz = zi - (double)xyz[3 * j + 2];
            double d2 = ((dx * dx) + (dy * dy)) + (dz * dz);
            if (cnt == k) {
                /* list full: (d2, j) must be strictly smaller than the last */
                if (d2 > bd[k - 1] || (d2 == bd[k - 1] && j > bj[k - 1])) continue;
            }
            /* insertion into the ascending list (d2, j) */
            int pos = (cnt < k) ? cnt : k - 1;
            while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bj[pos - 1] > j))) {
                bd[pos] = bd[pos - 1];
                bj[pos] = bj[pos - 1];
                --pos;
            }
            bd[pos] = d2;
            bj[pos] = j;
            if (cnt < k) ++cnt;
        }
        h_out[t] = (float)sqrt(bd[k - 1]);
        if (nbr_out)
            for (int m = 0; m < k; ++m) nbr_out[t * k + m] = bj[m];
        if (d2_out)
            for (int m = 0; m < k; ++m) d2_out[t * k + m] = bd[m];
        free(bd);
        free(bj);
    }
    return 0;
}

/*
 * Kernel density at m target positions r (m x 3 doubles).
 *
 * rho(r) = inv_neff * sum_j K(r - y_j ; l_j)   over members j (Eq. 7 with the
 * per-particle smoothing lengths l_j = (lx, ly, lz), ell = n x 3 doubles).
 *
 * With q = (dx/lx)^2 + (dy/ly)^2 + (dz/lz)^2:
 *   EPAN   (Eqs. 4 and 7):  K = 15/(8 pi) / (lx ly lz) * (1 - q)            if q < 1
 *   GAUSS3 (truncated):    K = exp(-q/2) / ((2 pi)^(3/2) lx ly lz P3)      if q < 9
 * where P3 = P(chi^2_3 <= 9) renormalises the Gaussian truncated at 3 l so
 * that a full kernel integrates to one. p3 is passed in by the caller.
 * A particle with any l_k <= 0 has no support and contributes nothing.
 *
 * member (nullable): n flags; 0 excludes particle j (the ROI clip scope).
 * wpeak (nullable): inv_neff * sum over in-support j of K(0; l_j).
 * amb   (nullable): inv_neff * sum of |K| (untruncated profile) over pairs with
 *                   |q/qmax - 1| < amb_band on either side of the cutoff: the mass
 *                   whose in/out decision depends on rounding alone (1e-6 for
 *                   an FP32 evaluation of q; wider for reduced-precision ones).
 * pairs (nullable): number of in-support (q < qmax) pairs per target.
 */
void or_density_at(const float *xyz, int64_t n, const double *ell,
                   const uint8_t *member, double inv_neff, int kernel, double p3,
                   const double *r, int64_t m, double *rho, double *wpeak,
                   double *amb, int64_t *pairs, double amb_band) {
    const double pi = 3.14159265358979323846;
    const double qmax = (kernel == OR_K_EPAN) ? 1.0 : 9.0;
    const double cnorm = (kernel == OR_K_EPAN) ? 15.0 / (8.0 * pi)
                                               : 1.0 / (pow(2.0 * pi, 1.5) * p3);
    int64_t t;
#pragma omp parallel for schedule(dynamic, 64)
    for (t = 0; t < m; ++t) {
        double rx = r[3 * t + 0], ry = r[3 * t + 1], rz = r[3 * t + 2];
        double sum = 0.0, wsum = 0.0, asum = 0.0;
        int64_t np = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (member && !member[j]) continue;
            double lx = ell[3 * j + 0], ly = ell[3 * j + 1], lz = ell[3 * j + 2];
            if (!(lx > 0.0) || !(ly > 0.0) || !(lz > 0.0)) continue;
            double ux = (rx - (double)xyz[3 * j + 0]) / lx;
            double uy = (ry - (double)xyz[3 * j + 1]) / ly;
            double uz = (rz - (double)xyz[3 * j + 2]) / lz;
            double qq = ((ux * ux) + (uy * uy)) + (uz * uz);
            /* pairs this close to the cutoff are in or out by rounding order alone:
               their kernel value counts as ambiguous on both sides of q = qmax */
            int ambiguous = fabs(qq / qmax - 1.0) < amb_band;
            if (!(qq < qmax) && !ambiguous) continue;
            double peak = cnorm / ((lx * ly) * lz);
            double val = (kernel == OR_K_EPAN) ? peak * (1.0 - qq) : peak * exp(-0.5 * qq);
            if (ambiguous) asum += fabs(val);
            if (!(qq < qmax)) continue;
            sum += val;
            wsum += peak;
            ++np;
        }
        rho[t] = inv_neff * sum;
        if (wpeak) wpeak[t] = inv_neff * wsum;
        if (amb) amb[t] = inv_neff * asum;
        if (pairs) pairs[t] = np;
    }
}
