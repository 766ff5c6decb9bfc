/*
 * FP64 direct-summation oracle for the 3D truncated Fourier series.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py load it (through oracle/__init__.py).
 *
 * What it computes (plain definitions, no fast algorithm):
 *   forward  (type 2)  f_j   = sum_k c_k exp(+2 pi i k.x_j)
 *   gradient           d_d f = sum_k (2 pi i k_d) c_k exp(+2 pi i k.x_j)
 *   adjoint  (type 1)  h_k   = sum_j f_j exp(-2 pi i k.x_j)
 * with k ranging over [-N1/2,N1/2) x [-N2/2,N2/2) x [-N3/2,N3/2).
 *
 * The series is the paper's eq. (fs) with its basis E_k written on the torus
 * [-1/2,1/2)^3 (Sec. 2.2, one-loop evaluation eq. (Fs), and the NFFT
 * definition of Sec. 2.2.1 with the + sign of the physical series); the
 * gradient is eq. (Lambda) in torus units (b_d - a_d = 1).
 *
 * Index convention: coefficient arrays are N1 x N2 x N3, row-major (i3
 * fastest), entry (i1,i2,i3) holding k_d = i_d - N_d/2 (the paper's
 * k_d - 1 - N_d/2 with 1-based k_d).  Complex numbers are interleaved
 * (re, im) doubles.  Points are M x 3 row-major doubles.
 *
 * Each exponential is evaluated directly (no recurrence): the phase k*x is
 * formed with an error-free product (fma), reduced to [-1/2,1/2] exactly,
 * and passed to cos/sin.  The triple sum is taken as nested per-dimension
 * sums (the distributive law applied to e^{2 pi i k.x} = prod_d
 * e^{2 pi i k_d x_d}, exactly as the paper's one-loop code does).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define TWO_PI 6.283185307179586476925286766559

/* e[i] = exp(sgn * 2 pi i k x), k = i - N/2, for i in [0, N). */
static void phase_row(int N, double x, double sgn, double *re, double *im)
{
    for (int i = 0; i < N; i++) {
        double k = (double)(i - N / 2);
        double p = k * x;
        double e = fma(k, x, -p);          /* k*x = p + e exactly */
        double r = (p - nearbyint(p)) + e; /* k*x mod 1, in [-1/2, 1/2] */
        re[i] = cos(TWO_PI * r);
        im[i] = sgn * sin(TWO_PI * r);
    }
}

/*
 * Forward series and (optionally) its gradient at M points.
 *   c     : N1*N2*N3 complex (2 doubles each), centred order
 *   x     : M*3 doubles
 *   f     : M complex out (may be NULL)
 *   grad  : M*3 complex out, grad[j*3+d] = d f / d x_d (may be NULL)
 */
void oracle_forward_grad(int N1, int N2, int N3, const double *c, int64_t M,
                         const double *x, double *f, double *grad)
{
#pragma omp parallel
    {
        double *e1r = malloc(sizeof(double) * N1), *e1i = malloc(sizeof(double) * N1);
        double *e2r = malloc(sizeof(double) * N2), *e2i = malloc(sizeof(double) * N2);
        double *e3r = malloc(sizeof(double) * N3), *e3i = malloc(sizeof(double) * N3);
#pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < M; j++) {
            phase_row(N1, x[3 * j + 0], 1.0, e1r, e1i);
            phase_row(N2, x[3 * j + 1], 1.0, e2r, e2i);
            phase_row(N3, x[3 * j + 2], 1.0, e3r, e3i);
            /* outer accumulators: f, d1 f, d2 f, d3 f (without the 2 pi i) */
            double fr = 0, fi = 0, g1r = 0, g1i = 0, g2r = 0, g2i = 0, g3r = 0, g3i = 0;
            for (int i1 = 0; i1 < N1; i1++) {
                double k1 = (double)(i1 - N1 / 2);
                double t0r = 0, t0i = 0, t2r = 0, t2i = 0, t3r = 0, t3i = 0;
                for (int i2 = 0; i2 < N2; i2++) {
                    double k2 = (double)(i2 - N2 / 2);
                    const double *row = c + 2 * ((int64_t)(i1 * N2 + i2) * N3);
                    double s0r = 0, s0i = 0, s3r = 0, s3i = 0;
                    if (grad) {
                        for (int i3 = 0; i3 < N3; i3++) {
                            double k3 = (double)(i3 - N3 / 2);
                            double cr = row[2 * i3], ci = row[2 * i3 + 1];
                            double pr = cr * e3r[i3] - ci * e3i[i3];
                            double pi = cr * e3i[i3] + ci * e3r[i3];
                            s0r += pr;
                            s0i += pi;
                            s3r += k3 * pr;
                            s3i += k3 * pi;
                        }
                    } else { /* value only: the same s0 sums without the k3 weights */
                        for (int i3 = 0; i3 < N3; i3++) {
                            double cr = row[2 * i3], ci = row[2 * i3 + 1];
                            s0r += cr * e3r[i3] - ci * e3i[i3];
                            s0i += cr * e3i[i3] + ci * e3r[i3];
                        }
                    }
                    double ar = s0r * e2r[i2] - s0i * e2i[i2];
                    double ai = s0r * e2i[i2] + s0i * e2r[i2];
                    t0r += ar;
                    t0i += ai;
                    t2r += k2 * ar;
                    t2i += k2 * ai;
                    t3r += s3r * e2r[i2] - s3i * e2i[i2];
                    t3i += s3r * e2i[i2] + s3i * e2r[i2];
                }
                double br = t0r * e1r[i1] - t0i * e1i[i1];
                double bi = t0r * e1i[i1] + t0i * e1r[i1];
                fr += br;
                fi += bi;
                g1r += k1 * br;
                g1i += k1 * bi;
                g2r += t2r * e1r[i1] - t2i * e1i[i1];
                g2i += t2r * e1i[i1] + t2i * e1r[i1];
                g3r += t3r * e1r[i1] - t3i * e1i[i1];
                g3i += t3r * e1i[i1] + t3i * e1r[i1];
            }
            if (f) {
                f[2 * j] = fr;
                f[2 * j + 1] = fi;
            }
            if (grad) {
                /* multiply by 2 pi i: (a + ib) * i = -b + ia */
                grad[6 * j + 0] = -TWO_PI * g1i;
                grad[6 * j + 1] = TWO_PI * g1r;
                grad[6 * j + 2] = -TWO_PI * g2i;
                grad[6 * j + 3] = TWO_PI * g2r;
                grad[6 * j + 4] = -TWO_PI * g3i;
                grad[6 * j + 5] = TWO_PI * g3r;
            }
        }
        free(e1r); free(e1i); free(e2r); free(e2i); free(e3r); free(e3i);
    }
}

/*
 * Adjoint (type 1): h_k = sum_j f_j exp(-2 pi i k.x_j), written into h
 * (N1*N2*N3 complex, centred order; overwritten).  Threads own disjoint i1
 * slabs of h, so no two threads write the same entry.
 */
void oracle_adjoint(int N1, int N2, int N3, int64_t M, const double *x,
                    const double *f, double *h)
{
    int64_t NN = (int64_t)N1 * N2 * N3;
    for (int64_t q = 0; q < 2 * NN; q++) h[q] = 0.0;
#pragma omp parallel
    {
        double *e1r = malloc(sizeof(double) * N1), *e1i = malloc(sizeof(double) * N1);
        double *e2r = malloc(sizeof(double) * N2), *e2i = malloc(sizeof(double) * N2);
        double *e3r = malloc(sizeof(double) * N3), *e3i = malloc(sizeof(double) * N3);
#pragma omp for schedule(static)
        for (int i1 = 0; i1 < N1; i1++) {
            for (int64_t j = 0; j < M; j++) {
                phase_row(N1, x[3 * j + 0], -1.0, e1r, e1i);
                phase_row(N2, x[3 * j + 1], -1.0, e2r, e2i);
                phase_row(N3, x[3 * j + 2], -1.0, e3r, e3i);
                double fr = f[2 * j], fi = f[2 * j + 1];
                double ar = fr * e1r[i1] - fi * e1i[i1];
                double ai = fr * e1i[i1] + fi * e1r[i1];
                for (int i2 = 0; i2 < N2; i2++) {
                    double br = ar * e2r[i2] - ai * e2i[i2];
                    double bi = ar * e2i[i2] + ai * e2r[i2];
                    double *row = h + 2 * ((int64_t)(i1 * N2 + i2) * N3);
                    for (int i3 = 0; i3 < N3; i3++) {
                        row[2 * i3] += br * e3r[i3] - bi * e3i[i3];
                        row[2 * i3 + 1] += br * e3i[i3] + bi * e3r[i3];
                    }
                }
            }
        }
        free(e1r); free(e1i); free(e2r); free(e2i); free(e3r); free(e3i);
    }
}

/*
 * Adjoint at selected frequencies: h_q = sum_j f_j exp(-2 pi i k_q.x_j) for
 * the nk frequency triples k (nk x 3 ints, each k_d any integer), over all M
 * points, for checking large adjoints on a sample of their outputs.  Each
 * phase k_d x_d is formed with an error-free product and reduced mod 1, the
 * three are added and reduced again, and the sum over j is compensated
 * (Neumaier), so the result stays accurate to rounding for M = 10^7.
 */
static void neumaier(double *s, double *comp, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *comp += (*s - t) + v;
    else
        *comp += (v - t) + *s;
    *s = t;
}

void oracle_adjoint_at(int nk, const int *k, int64_t M, const double *x,
                       const double *f, double *h)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nk; q++) {
        double sr = 0, cr = 0, si = 0, ci = 0;
        for (int64_t j = 0; j < M; j++) {
            double r = 0;
            for (int d = 0; d < 3; d++) {
                double kd = (double)k[3 * q + d];
                double p = kd * x[3 * j + d];
                double e = fma(kd, x[3 * j + d], -p);   /* k_d x_d = p + e exactly */
                r += (p - nearbyint(p)) + e;            /* each term in [-1/2, 1/2] */
            }
            r -= nearbyint(r);
            double er = cos(TWO_PI * r), ei = -sin(TWO_PI * r);
            double fr = f[2 * j], fi = f[2 * j + 1];
            neumaier(&sr, &cr, fr * er - fi * ei);
            neumaier(&si, &ci, fr * ei + fi * er);
        }
        h[2 * q] = sr + cr;
        h[2 * q + 1] = si + ci;
    }
}

/* Number of OpenMP threads the oracle runs with (for reporting). */
int oracle_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
