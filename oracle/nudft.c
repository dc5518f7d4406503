/*
 * Oracle (test infrastructure only): direct FP64 nonuniform DFT.
 *
 *   J[k][j] = sum_n c[k][n] * exp(-i 2 pi f_{idx[j]} t_n),   f_i = f_lo + i*df
 *
 * This is the eigencoefficient sum of Sec. 3.2, Eq. (eigencoefficients), and
 * Table 1 step 4, evaluated term by term with no transform: the bracketed
 * factor w_k^*(t_n) x(t_n) is passed in as c[k][n].  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg call it.
 *
 * Phase: the cycle count f_i * t_n is formed without rounding loss.  With
 * f_i = f_lo + i*df taken as an exact real number,
 *     f_i t_n = f_lo t_n + i (df t_n),
 * each product is split into a rounded part and its exact error term with
 * fma, and the integer part is removed before the sine and cosine are taken.
 * The phase therefore carries an absolute error of a few 1e-16 cycles for any
 * size of t_n, instead of eps * |f t|.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* fractional cycles of a*b, in [-0.5, 0.5] plus a tiny error term */
static double frac_of_product(double a, double b)
{
    double p = a * b;
    double e = fma(a, b, -p);      /* a*b = p + e exactly */
    return (p - nearbyint(p)) + e;
}

int m2o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * t      [N]          sampling times
 * cre/cim[K*N]        real and imaginary parts of c[k][n] (cim may be NULL)
 * idx    [nidx]       band indices i to evaluate
 * Jre/Jim[K*nidx]     output, J[k][j] for band idx[j]
 * nthreads            0 = OpenMP default
 */
void m2o_nudft(int64_t N, const double* t, int K, const double* cre, const double* cim,
               double f_lo, double df, int64_t nidx, const int64_t* idx,
               double* Jre, double* Jim, int nthreads)
{
    double* a  = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* bh = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* bl = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t n = 0; n < N; ++n) {
        a[n]  = frac_of_product(f_lo, t[n]);
        bh[n] = df * t[n];
        bl[n] = fma(df, t[n], -bh[n]);
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < nidx; ++j) {
        double sre[64], sim[64];
        double* accr = sre;
        double* acci = sim;
        double* heap = NULL;
        if (K > 64) {
            heap = (double*)malloc(sizeof(double) * 2 * (size_t)K);
            accr = heap;
            acci = heap + K;
        }
        for (int k = 0; k < K; ++k) { accr[k] = 0.0; acci[k] = 0.0; }
        const double di = (double)idx[j];
        for (int64_t n = 0; n < N; ++n) {
            /* cycles = frac(f_lo t) + frac(i * bh) + i * bl */
            double ph = a[n] + frac_of_product(di, bh[n]) + di * bl[n];
            ph -= nearbyint(ph);
            double s = sin(two_pi * ph), c = cos(two_pi * ph);
            /* exp(-i 2 pi ph) = c - i s */
            for (int k = 0; k < K; ++k) {
                double xr = cre[(int64_t)k * N + n];
                double xi = cim ? cim[(int64_t)k * N + n] : 0.0;
                accr[k] += xr * c + xi * s;
                acci[k] += xi * c - xr * s;
            }
        }
        for (int k = 0; k < K; ++k) {
            Jre[(int64_t)k * nidx + j] = accr[k];
            Jim[(int64_t)k * nidx + j] = acci[k];
        }
        free(heap);
    }
    free(a);
    free(bh);
    free(bl);
}
