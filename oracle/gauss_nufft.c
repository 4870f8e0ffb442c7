/*
 * O2: FP64 Gaussian-gridding NUFFT following Section 2 of Jiang, Greengard & Bao
 * (arXiv 1311.4120), itself after Greengard & Lee.  TEST INFRASTRUCTURE ONLY: the product
 * path never links or calls this file.
 *
 * Sums (t_j in (-pi, pi)^d, modes m in [-N/2, N/2)^d):
 *   type 2 (eq. 2.2):  F_j = sum_m f_m exp(-i t_j . m)
 *   type 1 (eq. 2.1):  u_m = sum_j c_j exp(+i t_j . m)      (no 1/N factor here)
 *
 * Steps (Section 2, eqs. 2.3-2.6), per axis with the periodic heat kernel
 *   g_tau(x) = sum_p exp(-(x - 2 pi p)^2 / (4 tau)),
 * whose Fourier coefficients are int_0^{2pi} g_tau(x) e^{-ikx} dx = 2 sqrt(pi tau) e^{-k^2 tau}:
 *   type 1: spread f_tau(x_l) = sum_j c_j g_tau(x_l - t_j) on the fine grid x_l = 2 pi l / Mr
 *           (eq. 2.6, nearest w points), FFT (eq. 2.5), then divide each mode by the heat
 *           kernel's coefficient:  u_m = (2 pi / Mr) e^{m^2 tau} / (2 sqrt(pi tau)) sum_l ...
 *   type 2: the same steps in reverse: deconvolve the modes, FFT to the fine grid, then
 *           interpolate with g_tau at each t_j.
 * The paper's parameters are Mr = 2N, tau = 12/N^2 with 24 points (about 12 digits) and
 * tau = 6/N^2 with 12 points (about 6 digits).  The caller picks (Mr, w, tau).
 *
 * Array conventions: grids are C-order with the first array axis slowest; node coordinates
 * t are stored (t_x, t_y[, t_z]) per node, where t_x pairs with the LAST (fastest) array axis.
 * Complex values are interleaved (re, im) doubles.
 *
 * The FFT is a plain recursive mixed-radix Cooley-Tukey transform (smallest prime factor
 * first, direct DFT for a prime length); it is checked against numpy.fft in the tests.
 * Spreading runs in parallel over blocks of the fine grid coloured so that no two blocks of
 * one colour touch the same fine-grid point; the sum is unchanged up to rounding order.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex dcx;

/* ------------------------------------------------------------------------- FFT */
static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

/* y[k] = sum_{j<n} x[j*s] * W^{jk}, W = exp(sign 2 pi i / n); tw[a] = exp(sign 2 pi i a / Ntw). */
static void fft_rec(const dcx *x, long s, int n, dcx *y, const dcx *tw, int Ntw) {
    if (n == 1) { y[0] = x[0]; return; }
    int p = smallest_factor(n);
    int m = n / p;
    if (m == 1) {                       /* prime length: direct DFT */
        for (int k = 0; k < n; k++) {
            dcx acc = 0;
            for (int j = 0; j < n; j++)
                acc += x[(long)j * s] * tw[((long)j * k % n) * (Ntw / n)];
            y[k] = acc;
        }
        return;
    }
    for (int r = 0; r < p; r++) fft_rec(x + (long)r * s, s * p, m, y + (long)r * m, tw, Ntw);
    dcx t[64];
    dcx *tb = p <= 64 ? t : (dcx *)malloc(sizeof(dcx) * p);
    for (int k = 0; k < m; k++) {
        for (int r = 0; r < p; r++)
            tb[r] = y[(long)r * m + k] * tw[((long)r * k % n) * (Ntw / n)];
        for (int q = 0; q < p; q++) {
            dcx acc = 0;
            for (int r = 0; r < p; r++) acc += tb[r] * tw[((long)r * q % p) * (Ntw / p)];
            y[(long)q * m + k] = acc;
        }
    }
    if (tb != t) free(tb);
}

/* In-place transform of every line along array axis `ax` of a C-order grid of extent Mr^d. */
static void fft_axis(dcx *g, int d, int Mr, int ax, int sign, int nthreads) {
    dcx *tw = (dcx *)malloc(sizeof(dcx) * Mr);
    for (int a = 0; a < Mr; a++) tw[a] = cexp(sign * 2.0 * M_PI * I * (double)a / Mr);
    long stride = 1;
    for (int a = d - 1; a > ax; a--) stride *= Mr;
    long total = 1;
    for (int a = 0; a < d; a++) total *= Mr;
    long nlines = total / Mr;
#pragma omp parallel num_threads(nthreads)
    {
        dcx *in = (dcx *)malloc(sizeof(dcx) * Mr);
        dcx *out = (dcx *)malloc(sizeof(dcx) * Mr);
#pragma omp for schedule(static)
        for (long L = 0; L < nlines; L++) {
            long outer = L / stride, inner = L % stride;
            long base = outer * stride * Mr + inner;
            for (int a = 0; a < Mr; a++) in[a] = g[base + (long)a * stride];
            fft_rec(in, 1, Mr, out, tw, Mr);
            for (int a = 0; a < Mr; a++) g[base + (long)a * stride] = out[a];
        }
        free(in);
        free(out);
    }
    free(tw);
}

int orc_fft(int d, int Mr, int sign, double *data, int nthreads) {
    for (int ax = 0; ax < d; ax++) fft_axis((dcx *)data, d, Mr, ax, sign, nthreads);
    return 0;
}

/* --------------------------------------------------------------------- Gaussian stencil */
typedef struct { int Mr, w, weff; double tau, dx; } gparam;

/* Weights of the periodic heat kernel at the stencil points of one coordinate t. */
static void stencil1d(const gparam *gp, double t, int *idx, double *wt) {
    int w = gp->weff;
    long l0;
    if (gp->weff == gp->Mr) l0 = (long)floor(t / gp->dx) - gp->Mr / 2 + 1;
    else l0 = (long)ceil(t / gp->dx - 0.5 * w);
    for (int a = 0; a < w; a++) {
        long l = l0 + a;
        double dist = l * gp->dx - t;
        double s = 0.0;
        for (int p = -3; p <= 3; p++) {
            double e = dist - 2.0 * M_PI * p;
            s += exp(-e * e / (4.0 * gp->tau));
        }
        wt[a] = s;
        long lm = l % gp->Mr;
        if (lm < 0) lm += gp->Mr;
        idx[a] = (int)lm;
    }
}

static double deconv1d(double m, double tau) {   /* 1 / (2 sqrt(pi tau) e^{-m^2 tau}) */
    return exp(m * m * tau) / (2.0 * sqrt(M_PI * tau));
}

/* ------------------------------------------------------------------------- type 2 */
int orc_type2(int d, int N, const double *f, long M, const double *t, double *out,
              int Mr, int w, double tau, int nthreads) {
    if (d < 2 || d > 3 || N < 2 || Mr < N) return -1;
    gparam gp = {Mr, w, w < Mr ? w : Mr, tau, 2.0 * M_PI / Mr};
    long tot = 1, nmodes = 1;
    for (int a = 0; a < d; a++) { tot *= Mr; nmodes *= N; }
    dcx *g = (dcx *)calloc(tot, sizeof(dcx));
    if (!g) return -2;
    const dcx *fc = (const dcx *)f;
    /* deconvolve and place mode m at fine index m mod Mr */
    for (long i = 0; i < nmodes; i++) {
        long rem = i, fi = 0;
        double fac = 1.0;
        long mul = 1;
        for (int a = d - 1; a >= 0; a--) {
            long ia = rem % N;
            rem /= N;
            long m = ia - N / 2;
            fac *= deconv1d((double)m, tau);
            long l = ((m % Mr) + Mr) % Mr;
            fi += l * mul;
            mul *= Mr;
        }
        g[fi] = fc[i] * fac;
    }
    orc_fft(d, Mr, -1, (double *)g, nthreads);
    double scale = pow(2.0 * M_PI / Mr, d);
    dcx *o = (dcx *)out;
#pragma omp parallel num_threads(nthreads)
    {
        int *ix = (int *)malloc(sizeof(int) * 3 * gp.weff);
        double *wx = (double *)malloc(sizeof(double) * 3 * gp.weff);
#pragma omp for schedule(dynamic, 256)
        for (long j = 0; j < M; j++) {
            /* axis a (array order) uses coordinate t[d-1-a] */
            for (int a = 0; a < d; a++)
                stencil1d(&gp, t[j * d + (d - 1 - a)], ix + a * gp.weff, wx + a * gp.weff);
            dcx acc = 0;
            int W = gp.weff;
            if (d == 3) {
                for (int a0 = 0; a0 < W; a0++)
                    for (int a1 = 0; a1 < W; a1++) {
                        double w01 = wx[a0] * wx[W + a1];
                        const dcx *row = g + ((long)ix[a0] * Mr + ix[W + a1]) * Mr;
                        for (int a2 = 0; a2 < W; a2++)
                            acc += w01 * wx[2 * W + a2] * row[ix[2 * W + a2]];
                    }
            } else {
                for (int a0 = 0; a0 < W; a0++) {
                    const dcx *row = g + (long)ix[a0] * Mr;
                    for (int a1 = 0; a1 < W; a1++) acc += wx[a0] * wx[W + a1] * row[ix[W + a1]];
                }
            }
            o[j] = scale * acc;
        }
        free(ix);
        free(wx);
    }
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------- type 1 */
int orc_type1(int d, int N, long M, const double *t, const double *c, double *out,
              int Mr, int w, double tau, int nthreads) {
    if (d < 2 || d > 3 || N < 2 || Mr < N) return -1;
    gparam gp = {Mr, w, w < Mr ? w : Mr, tau, 2.0 * M_PI / Mr};
    long tot = 1, nmodes = 1;
    for (int a = 0; a < d; a++) { tot *= Mr; nmodes *= N; }
    dcx *g = (dcx *)calloc(tot, sizeof(dcx));
    if (!g) return -2;
    const dcx *cc = (const dcx *)c;

    /* blocks on the two slowest array axes (one in 2D); block edge >= stencil width */
    int W = gp.weff;
    int nb = Mr / (W > 0 ? W : 1);
    if (nb % 2) nb -= 1;
    if (nb < 2) nb = 1;
    int bs = Mr / nb;                          /* last block absorbs the remainder */
    int nbz = nb, nby = (d == 3) ? nb : 1;
    long nblk = (long)nbz * nby;
    long *cnt = (long *)calloc(nblk + 1, sizeof(long));
    long *order = (long *)malloc(sizeof(long) * (M > 0 ? M : 1));
    int *blk = (int *)malloc(sizeof(int) * (M > 0 ? M : 1));
    for (long j = 0; j < M; j++) {
        int b[2] = {0, 0};
        for (int a = 0; a < (d == 3 ? 2 : 1); a++) {
            double tt = t[j * d + (d - 1 - a)];
            long l0 = (W == Mr) ? 0 : (long)ceil(tt / gp.dx - 0.5 * W);
            long lm = ((l0 % Mr) + Mr) % Mr;
            int bb = (int)(lm / bs);
            if (bb >= nb) bb = nb - 1;
            b[a] = bb;
        }
        blk[j] = b[0] * nby + b[1];
        cnt[blk[j] + 1]++;
    }
    for (long q = 0; q < nblk; q++) cnt[q + 1] += cnt[q];
    long *pos = (long *)malloc(sizeof(long) * (nblk + 1));
    memcpy(pos, cnt, sizeof(long) * (nblk + 1));
    for (long j = 0; j < M; j++) order[pos[blk[j]]++] = j;
    free(pos);

    int ncol = (nb == 1) ? 1 : 2;
    for (int cz = 0; cz < ncol; cz++)
        for (int cy = 0; cy < (d == 3 ? ncol : 1); cy++) {
#pragma omp parallel num_threads(nthreads)
            {
                int *ix = (int *)malloc(sizeof(int) * 3 * W);
                double *wx = (double *)malloc(sizeof(double) * 3 * W);
#pragma omp for schedule(dynamic, 1)
                for (long q = 0; q < nblk; q++) {
                    int bz = (int)(q / nby), by = (int)(q % nby);
                    if (bz % ncol != cz || (d == 3 && by % ncol != cy)) continue;
                    for (long e = cnt[q]; e < cnt[q + 1]; e++) {
                        long j = order[e];
                        for (int a = 0; a < d; a++)
                            stencil1d(&gp, t[j * d + (d - 1 - a)], ix + a * W, wx + a * W);
                        dcx cj = cc[j];
                        if (d == 3) {
                            for (int a0 = 0; a0 < W; a0++)
                                for (int a1 = 0; a1 < W; a1++) {
                                    dcx v = cj * (wx[a0] * wx[W + a1]);
                                    dcx *row = g + ((long)ix[a0] * Mr + ix[W + a1]) * Mr;
                                    for (int a2 = 0; a2 < W; a2++) row[ix[2 * W + a2]] += v * wx[2 * W + a2];
                                }
                        } else {
                            for (int a0 = 0; a0 < W; a0++) {
                                dcx *row = g + (long)ix[a0] * Mr;
                                for (int a1 = 0; a1 < W; a1++) row[ix[W + a1]] += cj * (wx[a0] * wx[W + a1]);
                            }
                        }
                    }
                }
                free(ix);
                free(wx);
            }
        }
    free(cnt);
    free(order);
    free(blk);

    orc_fft(d, Mr, +1, (double *)g, nthreads);
    double scale = pow(2.0 * M_PI / Mr, d);
    dcx *o = (dcx *)out;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long i = 0; i < nmodes; i++) {
        long rem = i, fi = 0, mul = 1;
        double fac = 1.0;
        for (int a = d - 1; a >= 0; a--) {
            long ia = rem % N;
            rem /= N;
            long m = ia - N / 2;
            fac *= deconv1d((double)m, tau);
            long l = ((m % Mr) + Mr) % Mr;
            fi += l * mul;
            mul *= Mr;
        }
        o[i] = scale * fac * g[fi];
    }
    free(g);
    return 0;
}
