/*
 * heat_oracle.c -- plain, slow FP64 CPU oracle for the stochastic-heating method
 * of Porter & Vladimirov (HEATCODE, arXiv:1311.4627).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the library never does.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Every step is written out in the order and notation of the paper (Sec. 2):
 *   Omega(lambda) = W(lambda) sigma(lambda) with log-log interpolation (Eq. interpolation),
 *   heating elements T_ul, u > l (Eq. heating), in the wavelength-integral form,
 *   thermal-continuous cooling T_{f-1,f} (Eq. adjacent, Eq. cooling),
 *   thermal-discrete cooling T_lu, l < u (the approximation named beside Eq. adjacent)
 *   and the stationary solve of the full rate matrix (Eq. steady-state, Eq. level-sum),
 *   B_fj suffix sums (Eq. bmatrix, via the recurrence Eq. brecurrence),
 *   X recursion and renormalisation (Eq. xf, Eq. renormalization),
 *   emissivity (Eq. emission, Eq. emission-lambda),
 *   size integration (Eq. convolution).
 * Readings where the paper is silent or garbled (bin edges, top-bin overflow,
 * the intra-bin term, the h^2 c and c^2 constants, cooling beyond the grid,
 * power-of-two rescaling) are listed in the project's design notes and restated
 * next to the code that takes them.
 *
 * Units: CGS throughout.  lambda in cm, u_lambda in erg cm^-3 cm^-1, C_abs in
 * cm^2, enthalpies in erg, rates in s^-1, j_lambda in erg s^-1 sr^-1 cm^-1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact values (CGS). */
static const double H_PL = 6.62607015e-27;  /* erg s */
static const double C_LI = 2.99792458e10;   /* cm s^-1 */
static const double K_B = 1.380649e-16;     /* erg K^-1 */

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENUMERIC 4

static double hc(void) { return H_PL * C_LI; }

/* ------------------------------------------------------------------------- */
/* Planck function per unit wavelength, B_lambda(T) = 2hc^2 lambda^-5/(e^x-1),
 * x = hc/(lambda k T).  (Eq. emission-lambda written per unit wavelength.)   */
double orc_planck_lambda(double lambda, double T)
{
    double x = hc() / (lambda * K_B * T);
    if (x > 745.0) return 0.0;
    return 2.0 * H_PL * C_LI * C_LI / pow(lambda, 5.0) / expm1(x);
}

/* ------------------------------------------------------------------------- */
/* Omega on the grid and its log-log interpolant (Eq. interpolation).        */
/* A segment n joins nodes n and n+1; it is zero unless both ends are > 0.   */
static int seg_active(const double* om, int n) { return om[n] > 0.0 && om[n + 1] > 0.0; }

static double seg_slope(const double* lam, const double* om, int n)
{
    return log(om[n + 1] / om[n]) / log(lam[n + 1] / lam[n]);
}

/* Index n of the segment [lam[n], lam[n+1]] holding x (lam[0] <= x <= lam[N-1]). */
static int find_segment(int N, const double* lam, double x)
{
    int lo = 0, hi = N - 2;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (lam[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Omega(lambda) from the interpolant; zero outside the grid. */
double orc_omega_at(int N, const double* lam, const double* om, double x)
{
    if (!(x >= lam[0] && x <= lam[N - 1])) return 0.0;
    int n = find_segment(N, lam, x);
    if (!seg_active(om, n)) return 0.0;
    return om[n] * pow(x / lam[n], seg_slope(lam, om, n));
}

/* Integral over [x, y] (inside segment n) of Omega(lambda) lambda^p dlambda.
 * With Omega = om_n (lambda/lam_n)^s and q = s + p + 1:
 *   = om_n lam_n^(p+1) (x/lam_n)^q expm1(q ln(y/x)) / q,   q != 0
 *   = om_n lam_n^(p+1) ln(y/x),                              q == 0.          */
static double seg_integral(const double* lam, const double* om, int n, int p, double x, double y)
{
    if (!(y > x) || !seg_active(om, n)) return 0.0;
    double s = seg_slope(lam, om, n);
    double q = s + (double)p + 1.0;
    double base = om[n] * pow(lam[n], (double)p + 1.0);
    double L = log(y / x);
    if (q == 0.0) return base * L;
    return base * exp(q * log(x / lam[n])) * expm1(q * L) / q;
}

/* Integral of Omega(lambda) lambda^p over [a, b]; Omega = 0 outside the grid. */
double orc_range_integral(int N, const double* lam, const double* om, int p, double a, double b)
{
    if (a < lam[0]) a = lam[0];
    if (b > lam[N - 1]) b = lam[N - 1];
    if (!(b > a)) return 0.0;
    double sum = 0.0;
    int n_first = find_segment(N, lam, a), n_last = find_segment(N, lam, b);
    for (int n = n_first; n <= n_last; ++n) {
        double x = a > lam[n] ? a : lam[n];
        double y = b < lam[n + 1] ? b : lam[n + 1];
        if (y > x) sum += seg_integral(lam, om, n, p, x, y);
    }
    return sum;
}

/* ------------------------------------------------------------------------- */
/* Heating elements A[u][l] = T_ul, u > l (Eq. heating, integral form).
 * Reading: bins i = 0..M with centres E_i; lower edges Elo_0 = 0,
 * Elo_i = (E_{i-1}+E_i)/2; upper edges Ehi_i = Elo_{i+1}, Ehi_M = +inf.
 * A grain at E_l that absorbs a photon of energy e lands in bin u when
 * Elo_u <= E_l + e < Ehi_u, i.e. lambda in [hc/(Ehi_u-E_l), hc/(Elo_u-E_l)].
 * The absorption rate per unit wavelength is c u_lambda C_abs / (hc/lambda)
 * = Omega lambda / h, so A_ul = (1/h) int Omega lambda dlambda over that range
 * (the paper's point rule with the constant read as h^2 c instead of hc^2).
 * Intra-bin term: photons too soft to leave bin l (lambda > hc/(Elo_{l+1}-E_l))
 * deposit power W_l = c int Omega dlambda; it is carried by the adjacent
 * transition, A_{l+1,l} += W_l / (E_{l+1} - E_l).
 * A is row-major nb x nb, A[u*nb + l]; entries with u <= l are zero.          */
int orc_heating_matrix(int N, const double* lam, const double* om, int nb, const double* E, double* A)
{
    if (N < 2 || nb < 2) return ORC_EINVAL;
    const int M = nb - 1;
    double* Elo = (double*)malloc(sizeof(double) * (size_t)nb);
    if (!Elo) return ORC_ENOMEM;
    Elo[0] = 0.0;
    for (int i = 1; i < nb; ++i) Elo[i] = 0.5 * (E[i - 1] + E[i]);
    memset(A, 0, sizeof(double) * (size_t)nb * (size_t)nb);
    for (int u = 1; u <= M; ++u) {
        for (int l = 0; l < u; ++l) {
            double lb = hc() / (Elo[u] - E[l]);
            double la = (u == M) ? 0.0 : hc() / (Elo[u + 1] - E[l]);
            A[(size_t)u * nb + l] = orc_range_integral(N, lam, om, 1, la, lb) / H_PL;
        }
    }
    for (int l = 0; l < M; ++l) {
        double lsoft = hc() / (Elo[l + 1] - E[l]);
        double W = C_LI * orc_range_integral(N, lam, om, 0, lsoft, lam[N - 1]);
        A[(size_t)(l + 1) * nb + l] += W / (E[l + 1] - E[l]);
    }
    free(Elo);
    return ORC_OK;
}

/* The paper's point rule (Eq. heating): T_ul = Omega(lambda_ul) lambda_ul^3 dE_u / (h^2 c)
 * with lambda_ul = hc / (E_u - E_l) (bin centres), Omega from the log-log interpolant (zero
 * outside the grid) and dE_u the width of the upper bin, E^hi_u - E^lo_u; the top bin, whose
 * upper edge is open, takes E_M - E_{M-1}.  The constant: photons absorbed per unit
 * wavelength at Omega lambda / h, times the wavelength window lambda^2 dE / (h c) that a bin
 * of width dE covers.  No intra-bin term: the paper's rule has none.                    */
int orc_heating_matrix_point(int N, const double* lam, const double* om, int nb, const double* E, double* A)
{
    if (N < 2 || nb < 2) return ORC_EINVAL;
    const int M = nb - 1;
    memset(A, 0, sizeof(double) * (size_t)nb * (size_t)nb);
    for (int u = 1; u <= M; ++u) {
        const double lo = 0.5 * (E[u - 1] + E[u]);
        const double dE = (u < M) ? 0.5 * (E[u] + E[u + 1]) - lo : E[M] - E[M - 1];
        for (int l = 0; l < u; ++l) {
            const double x = hc() / (E[u] - E[l]);
            A[(size_t)u * nb + l] = orc_omega_at(N, lam, om, x) * x * x * x * dE / (H_PL * H_PL * C_LI);
        }
    }
    return ORC_OK;
}

/* B_fj = sum_{k >= f} T_kj for f > j (Eq. bmatrix), built with the suffix
 * recurrence B_{f,j} = B_{f+1,j} + T_{f,j}, B_{M,j} = T_{M,j} (Eq. brecurrence).
 * B is row-major nb x nb; entries with f <= j are zero.                        */
void orc_b_matrix(int nb, const double* A, double* B)
{
    const int M = nb - 1;
    memset(B, 0, sizeof(double) * (size_t)nb * (size_t)nb);
    for (int j = 0; j < M; ++j) B[(size_t)M * nb + j] = A[(size_t)M * nb + j];
    for (int f = M - 1; f >= 1; --f)
        for (int j = 0; j < f; ++j)
            B[(size_t)f * nb + j] = B[(size_t)(f + 1) * nb + j] + A[(size_t)f * nb + j];
}

/* X recursion (Eq. xf) and renormalisation (Eq. renormalization).
 * X_0 = 1, X_f = (sum_{j<f} B_fj X_j) / T_{f-1,f}; Cf[f] holds T_{f-1,f}.
 * Overflow guard: whenever X_f > 2^800 all X_0..X_f are multiplied by 2^-800
 * (a power of two, so the scaling itself is exact; the paper scales by 1e-30).
 * Cf[f] == 0 with a non-zero numerator has no steady state: ORC_ENUMERIC.    */
int orc_recursion(int nb, const double* B, const double* Cf, double* P)
{
    const double big = ldexp(1.0, 800), shrink = ldexp(1.0, -800);
    int status = ORC_OK;
    P[0] = 1.0;
    for (int f = 1; f < nb; ++f) {
        double S = 0.0;
        for (int j = 0; j < f; ++j) S += B[(size_t)f * nb + j] * P[j];
        if (Cf[f] > 0.0) {
            P[f] = S / Cf[f];
        } else {
            P[f] = 0.0;
            if (S != 0.0) status = ORC_ENUMERIC;
        }
        if (P[f] > big)
            for (int i = 0; i <= f; ++i) P[i] *= shrink;
    }
    double sum = 0.0;
    for (int i = 0; i < nb; ++i) sum += P[i];
    for (int i = 0; i < nb; ++i) P[i] = P[i] / sum;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Cooling (Eq. cooling): T_{f-1,f} = P_emit(T_f; E_f) / (E_f - E_{f-1}) with
 *   P_emit(T; Emax) = 4 pi int_{hc/Emax}^inf C(lambda) B_lambda(T) dlambda
 *                   = 4 pi (2 k^4 T^4 / (h^3 c^2)) int_0^{Emax/kT} C x^3/(e^x-1) dx,
 * x = hc/(lambda k T) (the paper's 8 pi / (h^3 c^3) read as 8 pi / (h^3 c^2)).
 * C(lambda) is the log-log interpolant of the C_abs nodes, continued beyond the
 * grid as a power law with the slope of the end segment (the cold bins emit
 * longward of the grid).  The integral is done by adaptive Gauss-Legendre with
 * breakpoints at the grid nodes.                                              */

#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

/* Gauss-Legendre nodes and weights on [-1, 1], by Newton iteration on P_n. */
static void gl_init(void)
{
    if (gl_ready) return;
    const int n = GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

typedef struct {
    int N;
    const double* lam;
    const double* cabs;
    double T;
} cool_ctx;

/* C(lambda) with power-law continuation beyond the grid. */
static double cabs_at(const cool_ctx* c, double x_lam)
{
    const int N = c->N;
    const double* lam = c->lam;
    const double* cb = c->cabs;
    if (x_lam < lam[0]) {
        if (!(cb[0] > 0.0 && cb[1] > 0.0)) return 0.0;
        return cb[0] * pow(x_lam / lam[0], seg_slope(lam, cb, 0));
    }
    if (x_lam > lam[N - 1]) {
        if (!(cb[N - 2] > 0.0 && cb[N - 1] > 0.0)) return 0.0;
        return cb[N - 1] * pow(x_lam / lam[N - 1], seg_slope(lam, cb, N - 2));
    }
    return orc_omega_at(N, lam, cb, x_lam);
}

/* integrand in x = hc/(lambda k T): C(lambda(x)) x^3 / (e^x - 1) */
static double cool_integrand(const cool_ctx* c, double x)
{
    if (x <= 0.0) return 0.0;
    double lam = hc() / (x * K_B * c->T);
    return cabs_at(c, lam) * x * x * x / expm1(x);
}

static double gl_panel(const cool_ctx* c, double a, double b)
{
    double m = 0.5 * (a + b), r = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < GL_N; ++i) s += gl_w[i] * cool_integrand(c, m + r * gl_x[i]);
    return s * r;
}

static double adapt(const cool_ctx* c, double a, double b, double whole, double tol, int depth)
{
    double m = 0.5 * (a + b);
    double left = gl_panel(c, a, m), right = gl_panel(c, m, b);
    double diff = fabs(left + right - whole);
    /* stop when converged to the requested tolerance or to rounding level */
    if (depth >= 30 || diff <= tol || diff <= 1e-15 * fabs(left + right)) return left + right;
    return adapt(c, a, m, left, 0.5 * tol, depth + 1) + adapt(c, m, b, right, 0.5 * tol, depth + 1);
}

/* int_xmin^xmax C(lambda(x)) x^3/(e^x-1) dx, split at the grid nodes. */
static double cool_x_window(const cool_ctx* c, double xmin, double xmax)
{
    const int N = c->N;
    if (xmax > 800.0) xmax = 800.0;     /* integrand < 1e-340 relative beyond */
    if (xmin < 0.0) xmin = 0.0;
    if (!(xmax > xmin)) return 0.0;
    /* breakpoints: x_n = hc/(lam_n k T) (descending in n) inside the window, plus
     * geometric panels towards x -> 0 (lambda -> infinity) below the grid's end. */
    int cap = N + 200;
    double* pts = (double*)malloc(sizeof(double) * (size_t)cap);
    int np = 0;
    double xlast = hc() / (c->lam[N - 1] * K_B * c->T);
    double g = (xlast < xmax ? xlast : xmax);
    for (int k = 0; k < 120 && np < cap - N - 3 && g > xmin; ++k) { pts[np++] = g; g *= 0.5; }
    pts[np++] = xmin;
    for (int n = N - 1; n >= 0; --n) {
        double xn = hc() / (c->lam[n] * K_B * c->T);
        if (xn > xlast && xn < xmax && xn > xmin) pts[np++] = xn;
    }
    pts[np++] = xmax;
    /* sort ascending (insertion sort, small) */
    for (int i = 1; i < np; ++i) {
        double v = pts[i];
        int k = i - 1;
        while (k >= 0 && pts[k] > v) { pts[k + 1] = pts[k]; --k; }
        pts[k + 1] = v;
    }
    double coarse = 0.0;
    for (int i = 0; i + 1 < np; ++i)
        if (pts[i + 1] > pts[i]) coarse += gl_panel(c, pts[i], pts[i + 1]);
    double tol = 1e-16 * fabs(coarse);
    double total = 0.0;
    for (int i = 0; i + 1 < np; ++i) {
        if (!(pts[i + 1] > pts[i])) continue;
        double w = gl_panel(c, pts[i], pts[i + 1]);
        total += adapt(c, pts[i], pts[i + 1], w, tol, 0);
    }
    free(pts);
    return total;
}

static double cool_x_integral(const cool_ctx* c, double xmax) { return cool_x_window(c, 0.0, xmax); }

/* Emitted power P_emit(T; Emax) in erg/s (Eq. cooling numerator). */
double orc_emitted_power(int N, const double* lam, const double* cabs, double T, double Emax)
{
    gl_init();
    cool_ctx c = {N, lam, cabs, T};
    double pref = 4.0 * M_PI * 2.0 * pow(K_B * T, 4.0) / (pow(H_PL, 3.0) * C_LI * C_LI);
    return pref * cool_x_integral(&c, Emax / (K_B * T));
}

/* The same power restricted to photon energies in [Emin, Emax]. */
double orc_emitted_power_window(int N, const double* lam, const double* cabs, double T, double Emin, double Emax)
{
    gl_init();
    cool_ctx c = {N, lam, cabs, T};
    double pref = 4.0 * M_PI * 2.0 * pow(K_B * T, 4.0) / (pow(H_PL, 3.0) * C_LI * C_LI);
    return pref * cool_x_window(&c, Emin / (K_B * T), Emax / (K_B * T));
}

/* Cf[f] = T_{f-1,f} for f = 1..M; Cf[0] = 0. */
int orc_cooling(int N, const double* lam, const double* cabs, int nb, const double* T, const double* E, double* Cf)
{
    if (N < 2 || nb < 2) return ORC_EINVAL;
    gl_init();
    Cf[0] = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int f = 1; f < nb; ++f)
        Cf[f] = orc_emitted_power(N, lam, cabs, T[f], E[f]) / (E[f] - E[f - 1]);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Thermal-discrete cooling (the approximation the paper names next to Eq. adjacent; its
 * source's formulas are not in the paper, so this is the reading): a grain in bin u emits
 * as a body at T_u, with the power per unit photon energy of Eq. cooling's integrand, and a
 * photon of energy e leaves it in the bin l with Elo_l <= E_u - e < Ehi_l.  The rate to l is
 * the power emitted in that window of photon energies divided by the transition's energy:
 *   D[l][u] = P_emit(T_u; window of l) / (E_u - E_l),   window of l = [E_u - Ehi_l, E_u - Elo_l]
 * for l < u - 1, and for l = u - 1 the window [0, E_u - Elo_{u-1}]: photons too soft to
 * leave bin u are carried by the adjacent transition, as the heating's intra-bin term is.
 * The windows tile [0, E_u], so sum_l D[l][u] (E_u - E_l) = P_emit(T_u; E_u), the power the
 * thermal-continuous rate T_{u-1,u} carries (Eq. cooling); with all power in the adjacent
 * window the two treatments coincide.  D is row-major nb x nb, D[l*nb + u], zero for l >= u. */
/* Power of Eq. cooling's integrand at T over a narrow window of photon energies written in
 * the grain's energy after the emission, e in [e0, e0 + de] (photon energy E_u - e): its
 * limits are bin edges, so the window's width de is exact even where it is a tiny fraction
 * of the photon energy (a hot bin's photon that leaves the grain near the bottom), which the
 * difference of two photon-energy limits would lose.  Gauss-Legendre pieces between the
 * grid nodes that fall inside (the cross-section's log-log kinks).  Over a window narrower
 * than 1e-2 of the photon energy the Planck factor changes by at most e^7.45 (x <= 745), which
 * 16 Gauss-Legendre nodes integrate to rounding.                                            */
static double emitted_power_narrow(int N, const double* lam, const double* cabs, double T, double Eu, double e0,
                                   double de)
{
    cool_ctx c = {N, lam, cabs, T};
    double cut[64];
    int nc = 0;
    cut[nc++] = 0.0;
    for (int n = 0; n < N && nc < 62; ++n) {  /* node offsets inside (0, de) */
        double o = (Eu - hc() / lam[n]) - e0;
        if (o > 0.0 && o < de) cut[nc++] = o;
    }
    cut[nc++] = de;
    for (int i = 1; i < nc; ++i) {  /* ascending */
        double v = cut[i];
        int k = i - 1;
        while (k >= 0 && cut[k] > v) { cut[k + 1] = cut[k]; --k; }
        cut[k + 1] = v;
    }
    double pref = 8.0 * M_PI / (pow(H_PL, 3.0) * C_LI * C_LI);
    double acc = 0.0;
    for (int i = 0; i + 1 < nc; ++i) {
        double r = 0.5 * (cut[i + 1] - cut[i]), m = cut[i] + r;
        if (!(r > 0.0)) continue;
        double s = 0.0;
        for (int k = 0; k < GL_N; ++k) {
            double eps = Eu - (e0 + m + r * gl_x[k]);  /* photon energy */
            double x = eps / (K_B * T);
            if (!(eps > 0.0) || x > 745.0) continue;
            s += gl_w[k] * cabs_at(&c, hc() / eps) * eps * eps * eps / expm1(x);
        }
        acc += s * r;
    }
    return pref * acc;
}

int orc_cooling_discrete(int N, const double* lam, const double* cabs, int nb, const double* T, const double* E,
                         double* D)
{
    if (N < 2 || nb < 2) return ORC_EINVAL;
    gl_init();
    for (size_t k = 0; k < (size_t)nb * nb; ++k) D[k] = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int u = 1; u < nb; ++u) {
        for (int l = 0; l < u; ++l) {
            double elo_l = l == 0 ? 0.0 : 0.5 * (E[l - 1] + E[l]);
            double ehi_l = 0.5 * (E[l] + E[l + 1]);  /* l < u <= nb - 1, so E[l+1] exists */
            double emin = l == u - 1 ? 0.0 : E[u] - ehi_l;
            double emax = E[u] - elo_l;
            double p;
            if (l < u - 1 && ehi_l - elo_l < 1e-2 * emin)  /* narrow: in the grain's final energy */
                p = emitted_power_narrow(N, lam, cabs, T[u], E[u], elo_l, ehi_l - elo_l);
            else
                p = orc_emitted_power_window(N, lam, cabs, T[u], emin, emax);
            D[(size_t)l * nb + u] = p / (E[u] - E[l]);
        }
    }
    return ORC_OK;
}

/* Stationary distribution of the full rate matrix (Eq. steady-state with Eq. level-sum):
 * upward rates A[u*nb + l] = T_ul (u > l), downward rates D[l*nb + u] = T_lu (l < u).  By
 * state reduction (Grassmann, Taksar and Heyman): states n = nb-1 .. 1 are removed in turn;
 * the rates of n are redistributed over the remaining states, q_ij += q_in q_nj / s_n with
 * s_n = sum_{j<n} q_nj, every term a sum or product of non-negative numbers, so that small
 * probabilities keep their relative accuracy.  Then X_0 = 1, X_n = sum_{i<n} X_i q_in / s_n,
 * rescaled by 2^-800 whenever X_n > 2^800 (exact), and P = X / sum X.  A state with no
 * downward rate and non-zero inflow has no steady state (ORC_ENUMERIC).  O(nb^3).          */
int orc_solve_full(int nb, const double* A, const double* D, double* P)
{
    size_t nn = (size_t)nb * nb;
    double* q = (double*)malloc(sizeof(double) * nn);  /* q[i*nb + j]: rate from i to j */
    double* s = (double*)malloc(sizeof(double) * (size_t)nb);
    if (!q || !s) { free(q); free(s); return ORC_ENOMEM; }
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j)
            q[(size_t)i * nb + j] = i == j ? 0.0 : (j > i ? A[(size_t)j * nb + i] : D[(size_t)j * nb + i]);
    int st = ORC_OK;
    for (int n = nb - 1; n >= 1; --n) {
        double sn = 0.0;
        for (int j = 0; j < n; ++j) sn += q[(size_t)n * nb + j];
        s[n] = sn;
        if (sn == 0.0) continue;  /* nothing leaves n downward: X_n is 0 or undefined (below) */
        for (int i = 0; i < n; ++i) {
            double qin = q[(size_t)i * nb + n];
            if (qin == 0.0) continue;
            for (int j = 0; j < n; ++j)
                if (j != i) q[(size_t)i * nb + j] += qin * q[(size_t)n * nb + j] / sn;
        }
    }
    double total = 1.0;
    P[0] = 1.0;
    for (int n = 1; n < nb; ++n) {
        double in = 0.0;
        for (int i = 0; i < n; ++i) in += P[i] * q[(size_t)i * nb + n];
        if (s[n] == 0.0) {
            if (in != 0.0) st = ORC_ENUMERIC;
            P[n] = 0.0;
            continue;
        }
        P[n] = in / s[n];
        total += P[n];
        if (P[n] > 0x1p800) {
            for (int i = 0; i <= n; ++i) P[i] *= 0x1p-800;
            total *= 0x1p-800;
        }
    }
    for (int n = 0; n < nb; ++n) P[n] /= total;
    free(q); free(s);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Emissivity (Eq. emission, Eq. emission-lambda), per unit wavelength:
 *   j(lambda_n) = C_abs(lambda_n) sum_i P_i B_lambda_n(T_i) [E_i >= hc/lambda_n].
 * (The second P_i inside the paper's Lambda is read as a typo.)              */
void orc_emissivity(int N, const double* lam, const double* cabs, int nb, const double* T, const double* E,
                    const double* P, double* j)
{
    for (int n = 0; n < N; ++n) {
        double ecut = hc() / lam[n];
        double s = 0.0;
        for (int i = 0; i < nb; ++i)
            if (E[i] >= ecut) s += P[i] * orc_planck_lambda(lam[n], T[i]);
        j[n] = cabs[n] * s;
    }
}

/* Energy ledger: out[0] = sum_l P_l sum_{u>l} T_ul (E_u - E_l)  (absorbed, model)
 *                out[1] = sum_f P_f T_{f-1,f} (E_f - E_{f-1})   (emitted, model)
 * Summing Eq. bequation times (E_f - E_{f-1}) over f makes the two equal.   */
void orc_ledger(int nb, const double* A, const double* E, const double* Cf, const double* P, double* out)
{
    double ab = 0.0, em = 0.0;
    for (int l = 0; l < nb; ++l)
        for (int u = l + 1; u < nb; ++u) ab += P[l] * A[(size_t)u * nb + l] * (E[u] - E[l]);
    for (int f = 1; f < nb; ++f) em += P[f] * Cf[f] * (E[f] - E[f - 1]);
    out[0] = ab;
    out[1] = em;
}

/* The same ledger with thermal-discrete cooling: out[1] = sum_u P_u sum_{l<u} D_lu (E_u - E_l). */
void orc_ledger_full(int nb, const double* A, const double* D, const double* E, const double* P, double* out)
{
    double ab = 0.0, em = 0.0;
    for (int l = 0; l < nb; ++l)
        for (int u = l + 1; u < nb; ++u) {
            ab += P[l] * A[(size_t)u * nb + l] * (E[u] - E[l]);
            em += P[u] * D[(size_t)l * nb + u] * (E[u] - E[l]);
        }
    out[0] = ab;
    out[1] = em;
}

/* One (cell, grain) spectrum with thermal-discrete cooling: heating matrix (integral form),
 * the full stationary solve with the grain's downward rates D, emissivity and ledger. */
int orc_solve_spectrum_discrete(int N, const double* lam, const double* cabs, int nb, const double* T,
                                const double* E, const double* D, const double* u, double* P, double* j,
                                double* ledger)
{
    size_t nn = (size_t)nb * (size_t)nb;
    double* om = (double*)malloc(sizeof(double) * (size_t)N);
    double* A = (double*)malloc(sizeof(double) * nn);
    if (!om || !A) { free(om); free(A); return ORC_ENOMEM; }
    for (int n = 0; n < N; ++n) om[n] = u[n] * cabs[n];
    int st = orc_heating_matrix(N, lam, om, nb, E, A);
    if (st == ORC_OK) {
        st = orc_solve_full(nb, A, D, P);
        if (j) orc_emissivity(N, lam, cabs, nb, T, E, P, j);
        if (ledger) orc_ledger_full(nb, A, D, E, P, ledger);
    }
    free(om); free(A);
    return st;
}

/* Batch of thermal-discrete solves: as orc_solve_batch, with the grains' downward rates
 * D_g (nb_g x nb_g each, back to back in grain order) in Dall. */
int orc_solve_batch_discrete(int N, const double* lam, int G, const double* cabs, const int* bin_off,
                             const double* T, const double* E, const double* Dall, int cells, const double* u,
                             double* P, double* j, double* ledger, int n_threads)
{
    int status = ORC_OK;
    const long total = (long)cells * G;
    const int nbt = bin_off[G];
    size_t* doff = (size_t*)malloc(sizeof(size_t) * (size_t)(G + 1));
    if (!doff) return ORC_ENOMEM;
    doff[0] = 0;
    for (int g = 0; g < G; ++g) {
        size_t nb = (size_t)(bin_off[g + 1] - bin_off[g]);
        doff[g + 1] = doff[g] + nb * nb;
    }
#ifdef _OPENMP
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (long s = 0; s < total; ++s) {
        int c = (int)(s / G), g = (int)(s % G);
        int off = bin_off[g], nb = bin_off[g + 1] - bin_off[g];
        int st = orc_solve_spectrum_discrete(N, lam, cabs + (size_t)g * N, nb, T + off, E + off, Dall + doff[g],
                                             u + (size_t)c * N, P + (size_t)c * nbt + off,
                                             j ? j + ((size_t)c * G + g) * N : NULL,
                                             ledger ? ledger + ((size_t)c * G + g) * 2 : NULL);
        if (st != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (status == ORC_OK) status = st; }
        }
    }
    free(doff);
    (void)n_threads;
    return status;
}

/* One (cell, grain) spectrum end to end.  P[nb], j[N] (may be NULL),
 * ledger[2] (may be NULL).  Work buffers are allocated here.                 */
int orc_solve_spectrum(int N, const double* lam, const double* cabs, int nb, const double* T, const double* E,
                       const double* Cf, const double* u, double* P, double* j, double* ledger, int heating)
{
    size_t nn = (size_t)nb * (size_t)nb;
    double* om = (double*)malloc(sizeof(double) * (size_t)N);
    double* A = (double*)malloc(sizeof(double) * nn);
    double* B = (double*)malloc(sizeof(double) * nn);
    if (!om || !A || !B) { free(om); free(A); free(B); return ORC_ENOMEM; }
    for (int n = 0; n < N; ++n) om[n] = u[n] * cabs[n];
    int st = heating == 1 ? orc_heating_matrix_point(N, lam, om, nb, E, A) : orc_heating_matrix(N, lam, om, nb, E, A);
    if (st == ORC_OK) {
        orc_b_matrix(nb, A, B);
        st = orc_recursion(nb, B, Cf, P);
        if (j) orc_emissivity(N, lam, cabs, nb, T, E, P, j);
        if (ledger) orc_ledger(nb, A, E, Cf, P, ledger);
    }
    free(om); free(A); free(B);
    return st;
}

/* Batch over cells x grains (OpenMP over spectra, dynamic schedule as in the
 * paper's field-parallel loop).  Layout:
 *   cabs [G][N], bin_off [G+1], T/E/Cf [bin_off[G]], u [cells][N],
 *   P [cells][bin_off[G]], j [cells][G][N] (or NULL), ledger [cells][G][2] (or NULL).
 * Returns the first non-OK status seen (all spectra are still computed).     */
int orc_solve_batch(int N, const double* lam, int G, const double* cabs, const int* bin_off, const double* T,
                    const double* E, const double* Cf, int cells, const double* u, double* P, double* j,
                    double* ledger, int n_threads, int heating)
{
    int status = ORC_OK;
    const long total = (long)cells * G;
    const int nbt = bin_off[G];
#ifdef _OPENMP
    /* a thread count for this call only (the process-wide setting is left as it was) */
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (long s = 0; s < total; ++s) {
        int c = (int)(s / G), g = (int)(s % G);
        int off = bin_off[g], nb = bin_off[g + 1] - bin_off[g];
        int st = orc_solve_spectrum(N, lam, cabs + (size_t)g * N, nb, T + off, E + off, Cf + off,
                                    u + (size_t)c * N, P + (size_t)c * nbt + off,
                                    j ? j + ((size_t)c * G + g) * N : NULL,
                                    ledger ? ledger + ((size_t)c * G + g) * 2 : NULL, heating);
        if (st != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (status == ORC_OK) status = st; }
        }
    }
    (void)n_threads;
    return status;
}

/* Size integration (Eq. convolution, discretised): J[c][n] = sum_g w_g j[c][g][n]. */
void orc_size_integrate(int cells, int G, int N, const double* w, const double* j, double* J)
{
    for (int c = 0; c < cells; ++c)
        for (int n = 0; n < N; ++n) {
            double s = 0.0;
            for (int g = 0; g < G; ++g) s += w[g] * j[((size_t)c * G + g) * N + n];
            J[(size_t)c * N + n] = s;
        }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
