/* Fermi-Dirac integrals and the inverse of I_{1/2} for the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: compiled into liboracle_fd.so and called from
 * oracle/fermi_dirac.py; the CUDA library never links it.
 *
 * I_nu(eta) = int_0^inf x^nu / (1 + exp(x - eta)) dx (the finite-T Thomas-Fermi
 * ingredient of F_s^TF in Eq. 1).  With x = t^2 the integrand
 * 2 t^(2nu+1) / (1 + exp(t^2 - eta)) is analytic in t.  The range of the Fermi
 * argument u = t^2 - eta that matters, [max(-eta,-40), max(-eta,-40)+40] for
 * eta < 0 and [max(-eta,-40), 40] otherwise, is cut into 16 equal panels of at
 * most 5 units, each integrated by 20-point Gauss-Legendre in t; one more panel
 * covers t from 0 to the lower edge, where the occupation is 1 to 1e-17.
 */
#include <math.h>
#include <stddef.h>

#define NGL 20
#define NPAN 16

static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;

/* Gauss-Legendre nodes/weights by Newton on P_n (Golub-Welsch not needed). */
static void gl_init(void) {
    if (gl_ready) return;
    for (int i = 0; i < NGL; ++i) {
        double x = cos(M_PI * (i + 0.75) / (NGL + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= NGL; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = NGL * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) {
                /* recompute derivative at the final x for the weight */
                p0 = 1.0; p1 = x;
                for (int k = 2; k <= NGL; ++k) {
                    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                    p0 = p1; p1 = p2;
                }
                dp = NGL * (x * p1 - p0) / (x * x - 1.0);
                gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
                break;
            }
        }
        gl_x[i] = x;
    }
    gl_ready = 1;
}

static double occupation(double u) {
    if (u > 0) { double e = exp(-u); return e / (1.0 + e); }
    return 1.0 / (1.0 + exp(u));
}

/* I_{-1/2}, I_{1/2}, I_{3/2} at one eta (any pointer may be NULL). */
static void fd3(double eta, double* im, double* ih, double* i3) {
    double u_lo = -eta > -40.0 ? -eta : -40.0;
    double u_hi = eta < 0 ? u_lo + 40.0 : 40.0;
    double sm = 0, sh = 0, s3 = 0;
    double du = (u_hi - u_lo) / NPAN;
    for (int p = -1; p < NPAN; ++p) {
        double ta, tb;
        if (p < 0) { ta = 0.0; tb = sqrt(fmax(eta + u_lo, 0.0)); }
        else {
            ta = sqrt(fmax(eta + u_lo + du * p, 0.0));
            tb = sqrt(fmax(eta + u_lo + du * (p + 1), 0.0));
        }
        if (tb <= ta) continue;
        double half = 0.5 * (tb - ta), mid = 0.5 * (tb + ta);
        for (int j = 0; j < NGL; ++j) {
            double t = mid + half * gl_x[j];
            double w = 2.0 * half * gl_w[j] * occupation(t * t - eta);
            double t2 = t * t;
            sm += w;
            sh += w * t2;
            s3 += w * t2 * t2;
        }
    }
    if (im) *im = sm;
    if (ih) *ih = sh;
    if (i3) *i3 = s3;
}

void oracle_fd_integrals(const double* eta, long n, double* im, double* ih, double* i3) {
    gl_init();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        fd3(eta[i], im ? im + i : NULL, ih ? ih + i : NULL, i3 ? i3 + i : NULL);
}

/* eta with I_{1/2}(eta) = y: Newton on ln I_{1/2} kept inside the bracket
 * (ln u, max((3y/2)^(2/3), ln u + 0.44)), u = y / Gamma(3/2); bisection when a
 * Newton step leaves it.  eta0 (may be NULL) is only a starting guess.
 * Returns the number of points that failed to converge. */
long oracle_fd_inverse_half(const double* y, long n, const double* eta0, double* eta_out,
                            double tol) {
    gl_init();
    const double g32 = 0.5 * sqrt(M_PI);
    long bad = 0;
#pragma omp parallel for schedule(static) reduction(+:bad)
    for (long i = 0; i < n; ++i) {
        double yi = y[i];
        if (!(yi > 0)) { eta_out[i] = NAN; bad++; continue; }
        double lnu = log(yi / g32), lny = log(yi);
        double lo = lnu, hi = fmax(pow(1.5 * yi, 2.0 / 3.0), lnu + 0.44);
        double e;
        if (eta0) e = eta0[i];
        else e = yi < 1.0 ? lnu + yi / g32 / sqrt(8.0) : pow(1.5 * yi, 2.0 / 3.0);
        if (!(e > lo)) e = lo;
        if (!(e < hi)) e = hi;
        int ok = 0;
        for (int it = 0; it < 200; ++it) {
            double im, ih;
            fd3(e, &im, &ih, NULL);
            double F = log(ih) - lny;
            if (F < 0 && e > lo) lo = e;
            if (F > 0 && e < hi) hi = e;
            double next = e - F / (0.5 * im / ih);
            if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
            double d = fabs(next - e);
            e = next;
            if (d <= tol * fmax(1.0, fabs(e))) { ok = 1; break; }
        }
        eta_out[i] = e;
        if (!ok) bad++;
    }
    return bad;
}
