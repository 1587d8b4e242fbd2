/*
 * FP64 CPU oracle for the light-pollution convolution of Bara et al.,
 * "Fast Fourier-transform calculation of artificial night sky brightness
 * maps" (arXiv:1907.02891).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline arm do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, written out as plainly as possible:
 *
 *  (1) oracle_conv_points: the discrete form of the shift-invariant
 *      superposition integral, Sec. 2.3 Eq. (7) (B(r) = integral of
 *      K(r - r') L1(r') d^2 r'), i.e. Eq. (2) with the factorable source of
 *      Eq. (3) and the shift-invariant PSF of Sec. 2.3.  On a pixel grid with
 *      0-based indices
 *
 *          Bfull[i][j] = sum_{i'=0}^{H-1} sum_{j'=0}^{W-1}
 *                            L[i'][j'] * K[i - i'][j - j']
 *
 *      for 0 <= i < H + hk - 1 and 0 <= j < W + wk - 1, with K taken as zero
 *      outside [0,hk) x [0,wk).  This is the full linear (non-circular)
 *      convolution whose size is the padded size N_L + N_K - 1 of Sec. 2.5.
 *      The pixel-area factor of Eq. (2) is not applied: a caller folds it
 *      into K.  Sums run in FP64 in a fixed loop order (i' outer, j' inner),
 *      from the FP32 radiance promoted exactly and the FP64 kernel.
 *
 *  (2) oracle_dft2_points: the two-dimensional DFT of Sec. 2.3 Eq. (10),
 *
 *          F(k,l) = sum_n sum_m f(n,m) exp{-i 2 pi [k n / N + l m / M]}
 *
 *      written with 0-based indices (Eq. (10) is 1-based; substituting
 *      k-1 -> k, n-1 -> n gives this form), evaluated directly by the
 *      O(N M) double sum for each requested frequency.  The phase
 *      (k n mod N) / N is reduced in integer arithmetic before the
 *      trigonometric call so that large products lose no precision.
 *
 * Both are O(work) direct sums over every term; OpenMP spreads the requested
 * output points over the host cores.  Return value: 0 on success, -1 on an
 * invalid argument.
 */
#include <math.h>
#include <stdint.h>

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

/* One output pixel of the full linear convolution, Eq. (7) discretised. */
static double conv_one(const float *L, int64_t H, int64_t W, int64_t ldl,
                       const double *K, int64_t hk, int64_t wk,
                       int64_t i, int64_t j)
{
    /* K[i - i'][j - j'] is non-zero only for 0 <= i - i' < hk. */
    int64_t i0 = i - (hk - 1);
    if (i0 < 0) i0 = 0;
    int64_t i1 = i;
    if (i1 > H - 1) i1 = H - 1;
    int64_t j0 = j - (wk - 1);
    if (j0 < 0) j0 = 0;
    int64_t j1 = j;
    if (j1 > W - 1) j1 = W - 1;
    double acc = 0.0;
    for (int64_t ip = i0; ip <= i1; ++ip) {
        const float *Lrow = L + ip * ldl;
        const double *Krow = K + (i - ip) * wk;
        for (int64_t jp = j0; jp <= j1; ++jp)
            acc += (double)Lrow[jp] * Krow[j - jp];
    }
    return acc;
}

/*
 * Full-coordinate output points (ii[p], jj[p]), 0 <= ii < H+hk-1,
 * 0 <= jj < W+wk-1.  Points outside that range are zero by definition.
 */
int oracle_conv_points(const float *L, int64_t H, int64_t W, int64_t ldl,
                       const double *K, int64_t hk, int64_t wk,
                       const int64_t *ii, const int64_t *jj, int64_t npts,
                       double *out)
{
    if (!L || !K || !out || H < 1 || W < 1 || ldl < W || hk < 1 || wk < 1 ||
        npts < 0 || (npts > 0 && (!ii || !jj)))
        return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npts; ++p) {
        int64_t i = ii[p], j = jj[p];
        if (i < 0 || j < 0 || i > H + hk - 2 || j > W + wk - 2)
            out[p] = 0.0;
        else
            out[p] = conv_one(L, H, W, ldl, K, hk, wk, i, j);
    }
    return 0;
}

/* Whole full-size map, row-major (H+hk-1) x (W+wk-1). */
int oracle_conv_full(const float *L, int64_t H, int64_t W, int64_t ldl,
                     const double *K, int64_t hk, int64_t wk, double *Bfull)
{
    if (!L || !K || !Bfull || H < 1 || W < 1 || ldl < W || hk < 1 || wk < 1)
        return -1;
    const int64_t Ho = H + hk - 1, Wo = W + wk - 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < Ho; ++i)
        for (int64_t j = 0; j < Wo; ++j)
            Bfull[i * Wo + j] = conv_one(L, H, W, ldl, K, hk, wk, i, j);
    return 0;
}

/*
 * Eq. (10) at the frequencies (kk[p], ll[p]) for a real FP64 N x M matrix f
 * (row-major, leading dimension ldf).  out_re/out_im receive the real and
 * imaginary parts.
 */
int oracle_dft2_points(const double *f, int64_t N, int64_t M, int64_t ldf,
                       const int64_t *kk, const int64_t *ll, int64_t npts,
                       double *out_re, double *out_im)
{
    if (!f || N < 1 || M < 1 || ldf < M || npts < 0 ||
        (npts > 0 && (!kk || !ll || !out_re || !out_im)))
        return -1;
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < npts; ++p) {
        int64_t k = ((kk[p] % N) + N) % N;
        int64_t l = ((ll[p] % M) + M) % M;
        double sr = 0.0, si = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            int64_t kn = (k * n) % N;
            for (int64_t m = 0; m < M; ++m) {
                int64_t lm = (l * m) % M;
                /* phase = kn/N + lm/M, reduced to [0,1) exactly in integers */
                int64_t num = kn * M + lm * N;
                num %= (N * M);
                double ph = two_pi * (double)num / (double)(N * M);
                double v = f[n * ldf + m];
                sr += v * cos(ph);
                si -= v * sin(ph);
            }
        }
        out_re[p] = sr;
        out_im[p] = si;
    }
    return 0;
}
