/*
 * Plain CPU NFFT (OpenMP, FP64): the timed CPU baseline of the method.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only tests/ and the
 * CPU-baseline legs of bench.py load it (through oracle/cpu_nfft.py).  It
 * shares no code with the CUDA library.
 *
 * The paper (Sec. 2.2.1) evaluates the series with the NFFT library on the
 * CPU, cost O(N log N + M |log eps|^3), and states no window.  This file
 * implements the same standard NFFT steps as oracle/nfft_cpu.py, in C with
 * OpenMP threads, so that the CPU method can be timed at full size:
 *
 *   window  phi(tau) = sinh(b s) / (pi s),  s = sqrt(alpha^2 - tau^2), on
 *           -alpha < tau <= alpha (b / pi where s = 0), alpha = m + 1/2,
 *           b = pi (2 - N/n); its transform Phi(k/n) = I0(alpha sqrt(b^2 - (2 pi k / n)^2))
 *   step 1  G[k mod n] = c_k prod_d (-1)^k_d / Phi(k_d / n_d), zero elsewhere
 *   step 2  g = unnormalised inverse FFT of G (done by the caller's CPU FFT)
 *   step 3  f_j = sum over the (2m+1)^3 nodes l, l_d = ceil(u_d - alpha) + a,
 *           u_d = n_d (x_d + 1/2) with x wrapped onto [-1/2, 1/2), of
 *           g[l mod n] prod_d phi(u_d - l_d)
 *   adjoint spread (transpose of step 3), forward FFT (caller), then
 *           h_k = H[k mod n] prod_d (-1)^k_d / Phi(k_d / n_d).
 *
 * Complex arrays are interleaved (re, im) doubles; grids are n1 x n2 x n3
 * row-major in FFT order, coefficients N1 x N2 x N3 in centred order
 * (entry i_d holds k_d = i_d - N_d/2), points M x 3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846264338327950288

void cpu_nfft_set_threads(int t)
{
#ifdef _OPENMP
    omp_set_num_threads(t > 0 ? t : 1);
#else
    (void)t;
#endif
}

int cpu_nfft_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* I0 by its power series sum ((z/2)^2)^j / (j!)^2 (all terms positive). */
static double bessel_i0(double z)
{
    double q = 0.25 * z * z, term = 1.0, sum = 1.0;
    for (int j = 1; j < 500; j++) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* dec[i] = (-1)^k / Phi(k / n), k = i - N/2, i in [0, N). */
void cpu_nfft_tables(int N, int n, int m, double *dec)
{
    double b = PI * (2.0 - (double)N / (double)n), al = m + 0.5;
    for (int i = 0; i < N; i++) {
        int k = i - N / 2;
        double nu = 2.0 * PI * (double)k / (double)n;
        dec[i] = ((k % 2) ? -1.0 : 1.0) / bessel_i0(al * sqrt(b * b - nu * nu));
    }
}

/* Step 1: G (zeroed here) gets c_k dec1 dec2 dec3 at k mod n. */
void cpu_nfft_deconv(int N1, int N2, int N3, int n1, int n2, int n3, const double *c,
                     const double *d1, const double *d2, const double *d3, double *G)
{
    int64_t total = (int64_t)n1 * n2 * n3;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < 2 * total; e++) G[e] = 0.0;
#pragma omp parallel for schedule(static)
    for (int i1 = 0; i1 < N1; i1++) {
        int l1 = (i1 - N1 / 2 + n1) % n1;
        for (int i2 = 0; i2 < N2; i2++) {
            int l2 = (i2 - N2 / 2 + n2) % n2;
            const double *cr = c + 2 * (((int64_t)i1 * N2 + i2) * N3);
            double *gr = G + 2 * (((int64_t)l1 * n2 + l2) * n3);
            for (int i3 = 0; i3 < N3; i3++) {
                int l3 = (i3 - N3 / 2 + n3) % n3;
                double d = d1[i1] * d2[i2] * d3[i3];
                gr[2 * l3] = cr[2 * i3] * d;
                gr[2 * l3 + 1] = cr[2 * i3 + 1] * d;
            }
        }
    }
}

/* Adjoint's last step: h (N1 N2 N3, centred) = H[k mod n] dec1 dec2 dec3. */
void cpu_nfft_deconv_adj(int N1, int N2, int N3, int n1, int n2, int n3, const double *H,
                         const double *d1, const double *d2, const double *d3, double *h)
{
#pragma omp parallel for schedule(static)
    for (int i1 = 0; i1 < N1; i1++) {
        int l1 = (i1 - N1 / 2 + n1) % n1;
        for (int i2 = 0; i2 < N2; i2++) {
            int l2 = (i2 - N2 / 2 + n2) % n2;
            double *hr = h + 2 * (((int64_t)i1 * N2 + i2) * N3);
            const double *gr = H + 2 * (((int64_t)l1 * n2 + l2) * n3);
            for (int i3 = 0; i3 < N3; i3++) {
                int l3 = (i3 - N3 / 2 + n3) % n3;
                double d = d1[i1] * d2[i2] * d3[i3];
                hr[2 * i3] = gr[2 * l3] * d;
                hr[2 * i3 + 1] = gr[2 * l3 + 1] * d;
            }
        }
    }
}

/* The 2m+1 window values of one coordinate and its first node (wrapped). */
static int window_row(double x, int n, int m, double b, double *w)
{
    double xw = x - floor(x + 0.5), al = m + 0.5;
    double u = (double)n * (xw + 0.5);
    double l0 = ceil(u - al);
    for (int a = 0; a <= 2 * m; a++) {
        double tau = u - (l0 + a);
        double q = (al - tau) * (al + tau);
        double s = q > 0 ? sqrt(q) : 0.0;
        double v = s > 0 ? sinh(b * s) / (PI * s) : b / PI;
        w[a] = (tau > -al && tau <= al) ? v : 0.0;
    }
    long long l = (long long)l0 % n;
    return (int)(l < 0 ? l + n : l);
}

/* Step 3: f_j for all points, threads over points. */
void cpu_nfft_gather(int N1, int N2, int N3, int n1, int n2, int n3, const double *g, int64_t M,
                     const double *x, int m, double *f)
{
    int W = 2 * m + 1;
    double b1 = PI * (2.0 - (double)N1 / n1), b2 = PI * (2.0 - (double)N2 / n2),
           b3 = PI * (2.0 - (double)N3 / n3);
#pragma omp parallel
    {
        double w1[17], w2[17], w3[17];
        int i3[17];
#pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < M; j++) {
            int l1 = window_row(x[3 * j], n1, m, b1, w1);
            int l2 = window_row(x[3 * j + 1], n2, m, b2, w2);
            int l3 = window_row(x[3 * j + 2], n3, m, b3, w3);
            for (int c = 0; c < W; c++) i3[c] = (l3 + c) % n3;
            double fr = 0, fi = 0;
            for (int a = 0; a < W; a++) {
                int p1 = (l1 + a) % n1;
                double sr = 0, si = 0;
                for (int bb = 0; bb < W; bb++) {
                    const double *row = g + 2 * (((int64_t)p1 * n2 + (l2 + bb) % n2) * n3);
                    double rr = 0, ri = 0;
                    for (int c = 0; c < W; c++) {
                        rr += w3[c] * row[2 * i3[c]];
                        ri += w3[c] * row[2 * i3[c] + 1];
                    }
                    sr += w2[bb] * rr;
                    si += w2[bb] * ri;
                }
                fr += w1[a] * sr;
                fi += w1[a] * si;
            }
            f[2 * j] = fr;
            f[2 * j + 1] = fi;
        }
    }
}

/*
 * Adjoint spread: H (zeroed here) += f_j prod_d phi(u_d - l_d) over each
 * point's (2m+1)^3 nodes.  Points are bucketed by their first node l0_1;
 * the n1 planes of first nodes are cut into an even number of slabs of at
 * least 2m+1 planes, and the even slabs, then the odd ones, run in parallel:
 * the nodes a slab's points touch (its planes plus the next 2m) never meet
 * those of another slab of the same parity, so no two threads add to the
 * same node at once.
 */
void cpu_nfft_spread(int N1, int N2, int N3, int n1, int n2, int n3, double *H, int64_t M,
                     const double *x, const double *f, int m)
{
    int W = 2 * m + 1;
    double b1 = PI * (2.0 - (double)N1 / n1), b2 = PI * (2.0 - (double)N2 / n2),
           b3 = PI * (2.0 - (double)N3 / n3);
    int64_t total = (int64_t)n1 * n2 * n3;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < 2 * total; e++) H[e] = 0.0;
    /* bucket the points by l0_1 (counting sort) */
    int64_t *start = calloc((size_t)n1 + 1, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    int *plane = malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) {
        double w[17];
        plane[j] = window_row(x[3 * j], n1, m, b1, w);
    }
    for (int64_t j = 0; j < M; j++) start[plane[j] + 1]++;
    for (int p = 0; p < n1; p++) start[p + 1] += start[p];
    {
        int64_t *fill = malloc(sizeof(int64_t) * (size_t)n1);
        memcpy(fill, start, sizeof(int64_t) * (size_t)n1);
        for (int64_t j = 0; j < M; j++) order[fill[plane[j]]++] = j;
        free(fill);
    }
    int nthreads = cpu_nfft_threads();
    int nslab = 2 * nthreads;
    while (nslab > 2 && n1 / nslab < W) nslab -= 2;
    if (n1 / nslab < W) nslab = 1;
    for (int parity = 0; parity < (nslab > 1 ? 2 : 1); parity++) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int sl = parity; sl < nslab; sl += (nslab > 1 ? 2 : 1)) {
            int p0 = (int)((int64_t)n1 * sl / nslab), p1e = (int)((int64_t)n1 * (sl + 1) / nslab);
            double w1[17], w2[17], w3[17];
            int i3[17];
            for (int64_t q = start[p0]; q < start[p1e]; q++) {
                int64_t j = order[q];
                int l1 = window_row(x[3 * j], n1, m, b1, w1);
                int l2 = window_row(x[3 * j + 1], n2, m, b2, w2);
                int l3 = window_row(x[3 * j + 2], n3, m, b3, w3);
                for (int c = 0; c < W; c++) i3[c] = (l3 + c) % n3;
                double fr = f[2 * j], fi = f[2 * j + 1];
                for (int a = 0; a < W; a++) {
                    int pa = (l1 + a) % n1;
                    for (int bb = 0; bb < W; bb++) {
                        double wab = w1[a] * w2[bb];
                        double *row = H + 2 * (((int64_t)pa * n2 + (l2 + bb) % n2) * n3);
                        for (int c = 0; c < W; c++) {
                            row[2 * i3[c]] += fr * wab * w3[c];
                            row[2 * i3[c] + 1] += fi * wab * w3[c];
                        }
                    }
                }
            }
        }
    }
    free(start);
    free(order);
    free(plane);
}
