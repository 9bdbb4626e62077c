/*
 * Plain FP64 CPU oracle for one source iteration of the time-dependent,
 * multi-group, mixed-frame SHDOM step (Tominaga, Shibata & Blinnikov,
 * arXiv:1507.05141).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code with
 * the CUDA library and is written for a reader checking it against the
 * paper: no blocking, no fusion, no reordering beyond what the method
 * defines.  Loops over nodes / (ordinate, group) pairs carry plain OpenMP
 * pragmas so that the CPU baseline can use the host cores; results do not
 * depend on the thread count.
 *
 * Layout of every discrete-ordinate array: [c][g][k] with
 *   c = (iz*ny + iy)*nx + ix       (node)
 *   g                               (frequency group, ascending energy)
 *   k = a*nphi + b                  (ordinate: mu_a ascending Gauss-Legendre,
 *                                    phi_b = 2 pi b / nphi)
 * Spherical-harmonic arrays: [c][g][p], p = l*l + l + m.
 *
 * Paper passages followed (section / equation):
 *   static transfer equation and Lambda iteration ........ Sec. 2, eq:shdom
 *   time term via modified chi~, eta~ .................... Sec. 2.1, eq:time
 *   Lorentz frequency shift / aberration / invariants .... Sec. 2.2,
 *                                     eq:lorentzfreq, eq:lorentzray
 *   SH source S_lm = omega chi_l/(2l+1) I_lm + T_lm ...... Sec. 2.3
 *   Thomson and Klein-Nishina kernels, multigroup ........ Sec. 2.3,
 *                                     eq:comptoncross
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   ordinates: Gauss-Legendre mu x uniform phi starting at 0;
 *   real orthonormal SH without Condon-Shortley phase, full l <= L;
 *   angle remap: bilinear in (mu, phi) on the target frame's ordinate mesh,
 *     linear to a pole value (ring average) beyond the outermost ring;
 *   frequency remap: geometric (log-log) between group centres when both
 *     values are positive, linear in log(eps) otherwise; nearest group
 *     between the outer centre and the outer edge; zero beyond the edges
 *     (extinction: nearest group);
 *   transfer: linear-in-tau short characteristic with the upwind point on
 *     the face crossed first (largest |n_a|/h_a, ties to the lowest axis);
 *   one source iteration per time step, backward-Euler time term;
 *   KN kernel with the textbook squared (eps1/eps)^2 prefactor.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    int L, nmu, nphi;
    int G;
    const double *edges;     /* [G+1] ascending, units of m_e c^2            */
    const double *alpha0;    /* [c][g] comoving absorption coefficient        */
    const double *ne;        /* [c]    scattering coefficient scale (n_e sT)  */
    const double *u;         /* [c][3] spatial 4-velocity Gamma v / c         */
    const double *emis0;     /* [c][g] comoving isotropic emissivity          */
    const double *K;         /* [L+1][G][G] scattering kernel, row = out grp  */
    const double *sigma_out; /* [G] out-scattering cross-section / sigma_T    */
    double kappa;            /* 1/(c dt); 0 for the static problem            */
    int bc_mode;             /* 0 vacuum, 1 isotropic per group, 2 full array */
    const double *bc;        /* mode 1: [G]; mode 2: [c][g][k]                */
    int integrator;          /* 0 linear-in-tau, 1 cubic Bezier (sweep_pair) */
    /* thermal electrons (nth > 0): kernels tabulated on the temperature grid
     * theta_i = 10^(th_lg0 + i th_dlg), i < nth (K_th [nth][L+1][G][G],
     * so_th [nth][G], by orc_kn_thermal_table), and the node temperatures
     * theta_e [c] = kT_e / m_e c^2; they replace K and sigma_out */
    int nth;
    double th_lg0, th_dlg;
    const double *K_th, *so_th, *theta_e;
} orc_problem;

/* ------------------------------------------------------------------------ */
/* Quadrature and spherical harmonics                                        */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton's method
 * on the Legendre recurrence (n+1)P_{n+1} = (2n+1)xP_n - nP_{n-1}. */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            /* P_n = p1, P_{n-1} = p0 */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        /* cos guess is descending in i: store reversed for ascending order */
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Ordinate set: Gauss-Legendre in mu times uniform phi_b = 2 pi b / nphi.
 * dirs[k][3] = (sin th cos phi, sin th sin phi, mu); W[k] = w_a 2 pi / nphi,
 * so that sum_k W_k = 4 pi.  Direction components whose magnitude is below
 * 1e-12 are set to exactly zero (a ray parallel to a face has no inflow
 * face on that axis). */
int orc_ordinates(int nmu, int nphi, double *mu, double *wmu, double *dirs, double *W)
{
    if (orc_gauss_legendre(nmu, mu, wmu)) return -1;
    for (int a = 0; a < nmu; ++a) {
        double st = sqrt(1.0 - mu[a] * mu[a]);
        for (int b = 0; b < nphi; ++b) {
            int k = a * nphi + b;
            double phi = 2.0 * ORC_PI * b / nphi;
            double n[3] = {st * cos(phi), st * sin(phi), mu[a]};
            for (int i = 0; i < 3; ++i) {
                if (fabs(n[i]) < 1e-12) n[i] = 0.0;
                dirs[3 * k + i] = n[i];
            }
            W[k] = wmu[a] * 2.0 * ORC_PI / nphi;
        }
    }
    return 0;
}

static double factorial_ratio(int l, int m) /* (l-m)!/(l+m)!, m >= 0 */
{
    double r = 1.0;
    for (int i = l - m + 1; i <= l + m; ++i) r /= i;
    return r;
}

/* Real orthonormal spherical harmonics (Sec. 2.3), no Condon-Shortley phase:
 *   Y_lm = N_lm P_l^|m|(mu) * { cos(m phi) m>0 ; 1 m=0 ; sin(|m| phi) m<0 },
 *   N_lm = sqrt((2 - delta_m0)(2l+1)/(4 pi) (l-|m|)!/(l+|m|)!).
 * Output Y[p], p = l*l + l + m, for all l <= L. */
void orc_ylm(int L, double mu, double phi, double *Y)
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    for (int m = 0; m <= L; ++m) {
        /* P_m^m = (2m-1)!! sin^m */
        double pmm = 1.0;
        for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * st;
        double plm2 = 0.0, plm1 = 0.0;
        for (int l = m; l <= L; ++l) {
            double plm;
            if (l == m) plm = pmm;
            else if (l == m + 1) plm = mu * (2.0 * m + 1.0) * pmm;
            else plm = ((2.0 * l - 1.0) * mu * plm1 - (l + m - 1.0) * plm2) / (l - m);
            plm2 = plm1;
            plm1 = plm;
            double norm = sqrt((m == 0 ? 1.0 : 2.0) * (2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial_ratio(l, m));
            if (m == 0) {
                Y[l * l + l] = norm * plm;
            } else {
                Y[l * l + l + m] = norm * plm * cos(m * phi);
                Y[l * l + l - m] = norm * plm * sin(m * phi);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Lorentz transformation (Sec. 2.2)                                         */
/* ------------------------------------------------------------------------ */

/* Laboratory direction n -> comoving direction n0 for a fluid with spatial
 * 4-velocity u (eq:lorentzray written with u = Gamma v/c).  Returns the
 * frequency ratio nu0/nu = Gamma - u.n (eq:lorentzfreq), evaluated as
 * 1/(Gamma+|u|) + |u| |n - u^|^2 / 2, which equals Gamma - |u| cos(psi)
 * without the cancellation at large Gamma. */
double orc_lab_to_comoving(const double *u, const double *n, double *n0)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (uu == 0.0) {
        n0[0] = n[0]; n0[1] = n[1]; n0[2] = n[2];
        return 1.0;
    }
    double gam = sqrt(1.0 + uu), um = sqrt(uu);
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    double d2 = 0.0;
    for (int i = 0; i < 3; ++i) { double d = n[i] - u[i] / um; d2 += d * d; }
    double r = 1.0 / (gam + um) + 0.5 * um * d2;
    double f = 1.0 - un / (gam + 1.0);
    for (int i = 0; i < 3; ++i) n0[i] = (n[i] - u[i] * f) / r;
    return r;
}

/* Comoving direction n0 -> laboratory direction n (the inverse boost, u -> -u).
 * Returns nu/nu0 = Gamma + u.n0. */
double orc_comoving_to_lab(const double *u, const double *n0, double *n)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (uu == 0.0) {
        n[0] = n0[0]; n[1] = n0[1]; n[2] = n0[2];
        return 1.0;
    }
    double gam = sqrt(1.0 + uu), um = sqrt(uu);
    double un = u[0] * n0[0] + u[1] * n0[1] + u[2] * n0[2];
    double d2 = 0.0;
    for (int i = 0; i < 3; ++i) { double d = n0[i] + u[i] / um; d2 += d * d; }
    double q = 1.0 / (gam + um) + 0.5 * um * d2;
    double f = 1.0 + un / (gam + 1.0);
    for (int i = 0; i < 3; ++i) n[i] = (n0[i] + u[i] * f) / q;
    return q;
}

/* ------------------------------------------------------------------------ */
/* Remapping onto the other frame's mesh (Sec. 2.2, last paragraph)          */
/* ------------------------------------------------------------------------ */

/* Value of an ordinate field F[k*stride] at direction n: bilinear in
 * (mu, phi) over the ordinate mesh; phi periodic; beyond the outermost
 * Gauss ring, linear in mu towards the pole value, which is the average of
 * that ring. */
double orc_interp_angle(int nmu, int nphi, const double *mu, const double *F, long stride, const double *n)
{
    double m = n[2];
    if (m > 1.0) m = 1.0;
    if (m < -1.0) m = -1.0;
    double phi = atan2(n[1], n[0]);
    if (phi < 0.0) phi += 2.0 * ORC_PI;
    double x = phi / (2.0 * ORC_PI / nphi);
    int b = (int)floor(x);
    double tp = x - b;
    if (b >= nphi) b -= nphi;
    if (b < 0) b += nphi;
    int b1 = (b + 1) % nphi;

#define RING(a) ((1.0 - tp) * F[(long)((a) * nphi + b) * stride] + tp * F[(long)((a) * nphi + b1) * stride])
    if (m < mu[0]) {
        double pole = 0.0;
        for (int j = 0; j < nphi; ++j) pole += F[(long)j * stride];
        pole /= nphi;
        double t = (m + 1.0) / (mu[0] + 1.0);
        return (1.0 - t) * pole + t * RING(0);
    }
    if (m > mu[nmu - 1]) {
        double pole = 0.0;
        for (int j = 0; j < nphi; ++j) pole += F[(long)((nmu - 1) * nphi + j) * stride];
        pole /= nphi;
        double t = (1.0 - m) / (1.0 - mu[nmu - 1]);
        return (1.0 - t) * pole + t * RING(nmu - 1);
    }
    if (nmu == 1) return RING(0);
    int a = 0;
    while (a < nmu - 2 && m > mu[a + 1]) ++a;
    double t = (m - mu[a]) / (mu[a + 1] - mu[a]);
    return (1.0 - t) * RING(a) + t * RING(a + 1);
#undef RING
}

/* Value of a group field F[g*stride] at energy eps.  Between group centres
 * ebar_g = sqrt(e_g e_{g+1}): geometric (F_g^{1-t} F_{g+1}^t, t linear in
 * log eps) when both values are positive, else linear in log eps.  Between
 * an outer centre and the outer edge: that group's value.  Beyond the
 * edges: 0, or the nearest group's value when nearest_outside is set (used
 * for the extinction coefficient). */
double orc_interp_freq(int G, const double *edges, const double *F, long stride, double eps, int nearest_outside)
{
    if (eps < edges[0]) return nearest_outside ? F[0] : 0.0;
    if (eps > edges[G]) return nearest_outside ? F[(long)(G - 1) * stride] : 0.0;
    double c0 = sqrt(edges[0] * edges[1]);
    double cl = sqrt(edges[G - 1] * edges[G]);
    if (eps <= c0) return F[0];
    if (eps >= cl) return F[(long)(G - 1) * stride];
    int g = 0;
    while (g < G - 2 && eps >= sqrt(edges[g + 1] * edges[g + 2])) ++g;
    double ca = sqrt(edges[g] * edges[g + 1]);
    double cb = sqrt(edges[g + 1] * edges[g + 2]);
    double t = log(eps / ca) / log(cb / ca);
    double fa = F[(long)g * stride], fb = F[(long)(g + 1) * stride];
    if (fa > 0.0 && fb > 0.0) return fa * exp(t * log(fb / fa));
    return (1.0 - t) * fa + t * fb;
}

/* ------------------------------------------------------------------------ */
/* Klein-Nishina multigroup kernel (Sec. 2.3, eq:comptoncross)               */
/* ------------------------------------------------------------------------ */

/* Differential cross-section per unit solid angle in units of sigma_T for a
 * photon of energy eps (m_e c^2) scattered through cos(Theta) = mu:
 *   (3/(16 pi)) r^2 (1/r + r - sin^2 Theta),   r = eps1/eps,
 *   eps1 = eps / (1 + eps (1 - mu)).
 * (r0^2/2 = 3 sigma_T/(16 pi); squared prefactor as in the textbook form.) */
static double kn_dsdo(double eps, double mu)
{
    double r = 1.0 / (1.0 + eps * (1.0 - mu));
    return 3.0 / (16.0 * ORC_PI) * r * r * (1.0 / r + r - (1.0 - mu * mu));
}

static double legendre_p(int l, double x)
{
    if (l == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= l; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

#define KN_NQ 32
static double kn_x[KN_NQ], kn_w[KN_NQ];
static int kn_ready = 0;

/* Inner integral over scattering angle, for incident eps, of
 *   P_l(mu) dsdo(eps, mu) (eps1/eps)^ew   over eps1 in [lo, hi],
 * done in sigma = ln(eps1): mu = 1 + 1/eps - 1/eps1, dmu = d sigma / eps1. */
static double kn_inner(int l, int ew, double eps, double lo, double hi)
{
    if (!(hi > lo)) return 0.0;
    double s0 = log(lo), s1 = log(hi);
    double hs = 0.5 * (s1 - s0), ms = 0.5 * (s1 + s0);
    double acc = 0.0;
    for (int i = 0; i < KN_NQ; ++i) {
        double e1 = exp(ms + hs * kn_x[i]);
        double mu = 1.0 + 1.0 / eps - 1.0 / e1;
        if (mu > 1.0) mu = 1.0;
        if (mu < -1.0) mu = -1.0;
        double f = legendre_p(l, mu) * kn_dsdo(eps, mu) / e1;
        if (ew) f *= e1 / eps;
        acc += kn_w[i] * f;
    }
    return acc * hs;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* K_l[g][g'] = (2 pi / de_g) Int_{g'} d eps Int d mu P_l(mu) dsdo (eps1/eps)^ew
 *              over the angles whose scattered energy eps1 falls in group g.
 * With ew = 1 this is the energy-intensity kernel used by the source
 * (S_lm(g) = n_e/chi0 * sum_g' K_l[g][g'] I_lm(g') + T_lm); with ew = 0 it
 * counts photons.  sigma_out[g'] = (1/de_g') Int_{g'} sigma_KN(eps) d eps
 * (in sigma_T), evaluated with the same angular quadrature over all angles.
 * The outer energy integral is split where an edge of group g stops being
 * reachable (eps = e, eps = e/(1-2e)) and done in log(eps). */
int orc_kn_table(int G, const double *edges, int L, int ew, double *K, double *sigma_out)
{
    if (!kn_ready) {
        orc_gauss_legendre(KN_NQ, kn_x, kn_w);
        kn_ready = 1;
    }
    double *bp = (double *)malloc(sizeof(double) * (2 * (G + 1) + 2));
    for (int gp = 0; gp < G; ++gp) {
        double ea = edges[gp], eb = edges[gp + 1];
        int nb = 0;
        bp[nb++] = ea;
        bp[nb++] = eb;
        for (int j = 0; j <= G; ++j) {
            double e = edges[j];
            if (e > ea && e < eb) bp[nb++] = e;
            if (e < 0.5) {
                double e2 = e / (1.0 - 2.0 * e);
                if (e2 > ea && e2 < eb) bp[nb++] = e2;
            }
        }
        qsort(bp, nb, sizeof(double), cmp_double);
        double tot = 0.0;
        for (int l = 0; l <= L; ++l)
            for (int g = 0; g < G; ++g) K[((long)l * G + g) * G + gp] = 0.0;
        for (int s = 0; s + 1 < nb; ++s) {
            if (!(bp[s + 1] > bp[s])) continue;
            double t0 = log(bp[s]), t1 = log(bp[s + 1]);
            double ht = 0.5 * (t1 - t0), mt = 0.5 * (t1 + t0);
            for (int i = 0; i < KN_NQ; ++i) {
                double eps = exp(mt + ht * kn_x[i]);
                double wq = kn_w[i] * ht * eps; /* d eps = eps d ln(eps) */
                double e1min = eps / (1.0 + 2.0 * eps), e1max = eps;
                tot += wq * 2.0 * ORC_PI * kn_inner(0, 0, eps, e1min, e1max);
                for (int g = 0; g < G; ++g) {
                    double lo = fmax(edges[g], e1min), hi = fmin(edges[g + 1], e1max);
                    if (!(hi > lo)) continue;
                    for (int l = 0; l <= L; ++l)
                        K[((long)l * G + g) * G + gp] += wq * kn_inner(l, ew, eps, lo, hi);
                }
            }
        }
        for (int l = 0; l <= L; ++l)
            for (int g = 0; g < G; ++g)
                K[((long)l * G + g) * G + gp] *= 2.0 * ORC_PI / (edges[g + 1] - edges[g]);
        sigma_out[gp] = tot / (eb - ea);
    }
    free(bp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Compton scattering off thermal electrons (reading of Sec. 2.3 for a       */
/* temperature field; the paper's kernel is the cold-electron one)            */
/* ------------------------------------------------------------------------ */

/* Total Klein-Nishina cross-section of a photon of energy x (m_e c^2) on an
 * electron at rest, in units of sigma_T (the textbook closed form; the
 * Thomson limit 1 - 2x below x = 1e-4). */
static double sigma_kn_total(double x)
{
    if (x < 1e-4) return 1.0 - 2.0 * x + 5.2 * x * x;
    double l = log1p(2.0 * x);
    return 0.75 * ((1.0 + x) / (x * x * x) * (2.0 * x * (1.0 + x) / (1.0 + 2.0 * x) - l) + l / (2.0 * x) -
                   (1.0 + 3.0 * x) / ((1.0 + 2.0 * x) * (1.0 + 2.0 * x)));
}

/* Quadrature of the thermal kernel: NE points in ln(eps) per incident group,
 * NMU in the laboratory scattering cosine, and over the isotropic
 * Maxwell-Juttner electrons NS in s = sqrt((gamma - 1)/theta) on [0, SMAX],
 * NME in the electron's direction cosine and NPHI in its azimuth (midpoints). */
#define TH_NE 16
#define TH_NMU 48
#define TH_NS 24
#define TH_SMAX 6.324555320336759 /* sqrt(40) */
#define TH_NME 16
#define TH_NPHI 16

/* K_l^theta[g][g'] = (2 pi / de_g) Int_{g'} d eps Int d mu P_l(mu)
 *      < (dsigma/dOmega1)_e (eps1/eps)^ew 1[eps1 in g] >_theta,
 * sigma_out^theta[g'] = (1/de_g') Int_{g'} d eps < (1 - beta mu_e) sigma_KN(eps') >_theta
 * for a photon along z scattered into the direction at cosine mu (azimuth
 * 0; the average over isotropic electrons does not depend on it), and an
 * electron of Lorentz factor gamma, speed beta, direction n_e
 * (mu_e = n_e.z, mu_e1 = n_e.n1), all in units of m_e c^2 and sigma_T:
 *   eps'  = gamma eps (1 - beta mu_e)                   (electron rest frame)
 *   eps1  = eps (1 - beta mu_e) / ((1 - beta mu_e1) + (eps/gamma)(1 - mu))
 *   eps1' = gamma eps1 (1 - beta mu_e1),  1 - cos T' = 1/eps1' - 1/eps'
 *   (dsigma/dOmega1)_e = (1 - beta mu_e) (3/16 pi) (eps1/eps')^2
 *                        (eps'/eps1' + eps1'/eps' - sin^2 T')
 * (energy-momentum conservation; the rest-frame Klein-Nishina cross-section
 * carried to the laboratory solid angle and weighted by the relative flux).
 * The electron average uses the Maxwell-Juttner density gamma^2 beta
 * e^{-(gamma-1)/theta} on the quadrature above, normalised on it.  With
 * beta = 0 this is the cold kernel of orc_kn_table. */
int orc_kn_thermal_table(int G, const double *edges, int L, int ew, double theta, double *K, double *sigma_out)
{
    double xs[TH_NS], ws[TH_NS], xme[TH_NME], wme[TH_NME], xmu[TH_NMU], wmu[TH_NMU], xe[TH_NE], we[TH_NE];
    orc_gauss_legendre(TH_NS, xs, ws);
    orc_gauss_legendre(TH_NME, xme, wme);
    orc_gauss_legendre(TH_NMU, xmu, wmu);
    orc_gauss_legendre(TH_NE, xe, we);
    /* electrons: gamma, beta and weight per s node */
    double gam[TH_NS], bet[TH_NS], wel[TH_NS], wsum = 0.0;
    for (int i = 0; i < TH_NS; ++i) {
        double sv = 0.5 * TH_SMAX * (xs[i] + 1.0);
        gam[i] = 1.0 + theta * sv * sv;
        bet[i] = sqrt(1.0 - 1.0 / (gam[i] * gam[i]));
        /* d gamma = 2 theta s ds; density gamma^2 beta e^{-s^2} */
        wel[i] = 0.5 * TH_SMAX * ws[i] * gam[i] * gam[i] * bet[i] * exp(-sv * sv) * 2.0 * theta * sv;
        wsum += wel[i];
    }
    for (int i = 0; i < TH_NS; ++i) wel[i] /= wsum;
    for (long i = 0; i < (long)(L + 1) * G * G; ++i) K[i] = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int gp = 0; gp < G; ++gp) {
        double *acc = (double *)calloc((size_t)(L + 1) * G, sizeof(double));
        double pl[32];
        double tot = 0.0;
        double t0 = log(edges[gp]), t1 = log(edges[gp + 1]);
        double ht = 0.5 * (t1 - t0), mt = 0.5 * (t1 + t0);
        for (int ie = 0; ie < TH_NE; ++ie) {
            double eps = exp(mt + ht * xe[ie]);
            double weps = we[ie] * ht * eps;
            /* total cross-section: electrons only */
            double avg = 0.0;
            for (int is = 0; is < TH_NS; ++is)
                for (int im = 0; im < TH_NME; ++im) {
                    double f = 1.0 - bet[is] * xme[im];
                    avg += wel[is] * 0.5 * wme[im] * f * sigma_kn_total(gam[is] * eps * f);
                }
            tot += weps * avg;
            for (int iu = 0; iu < TH_NMU; ++iu) {
                double mu = xmu[iu];
                double smu = sqrt(1.0 - mu * mu);
                pl[0] = 1.0;
                if (L >= 1) pl[1] = mu;
                for (int l = 2; l <= L; ++l) pl[l] = ((2.0 * l - 1.0) * mu * pl[l - 1] - (l - 1.0) * pl[l - 2]) / l;
                for (int is = 0; is < TH_NS; ++is)
                    for (int im = 0; im < TH_NME; ++im) {
                        double cme = xme[im], sme = sqrt(1.0 - cme * cme);
                        for (int ip = 0; ip < TH_NPHI; ++ip) {
                            double phe = 2.0 * ORC_PI * (ip + 0.5) / TH_NPHI;
                            double b = bet[is], gm = gam[is];
                            double mue1 = sme * cos(phe) * smu + cme * mu; /* n_e . n1, n1 = (sin, 0, mu) */
                            double a = 1.0 - b * cme;
                            double eps1 = eps * a / ((1.0 - b * mue1) + (eps / gm) * (1.0 - mu));
                            int g = -1;
                            for (int q = 0; q < G; ++q)
                                if (eps1 >= edges[q] && eps1 < edges[q + 1]) { g = q; break; }
                            if (g < 0) continue;
                            double ep = gm * eps * a, e1p = gm * eps1 * (1.0 - b * mue1);
                            double ct = 1.0 - (1.0 / e1p - 1.0 / ep);
                            double r = eps1 / ep;
                            double dsdo = a * 3.0 / (16.0 * ORC_PI) * r * r * (ep / e1p + e1p / ep - (1.0 - ct * ct));
                            if (ew) dsdo *= eps1 / eps;
                            double wgt = weps * wmu[iu] * wel[is] * 0.5 * wme[im] / TH_NPHI * dsdo;
                            for (int l = 0; l <= L; ++l) acc[(long)l * G + g] += wgt * pl[l];
                        }
                    }
            }
        }
        for (int l = 0; l <= L; ++l)
            for (int g = 0; g < G; ++g)
                K[((long)l * G + g) * G + gp] = 2.0 * ORC_PI * acc[(long)l * G + g] / (edges[g + 1] - edges[g]);
        sigma_out[gp] = tot / (edges[gp + 1] - edges[gp]);
        free(acc);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The step                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, NLM, G;
    double *mu, *wmu, *dirs, *W, *Y; /* Y[k][p] */
    double *centre;
} orc_mesh;

static void mesh_init(const orc_problem *P, orc_mesh *M)
{
    M->N = P->nmu * P->nphi;
    M->NLM = (P->L + 1) * (P->L + 1);
    M->G = P->G;
    M->mu = (double *)malloc(sizeof(double) * P->nmu);
    M->wmu = (double *)malloc(sizeof(double) * P->nmu);
    M->dirs = (double *)malloc(sizeof(double) * 3 * M->N);
    M->W = (double *)malloc(sizeof(double) * M->N);
    M->Y = (double *)malloc(sizeof(double) * M->N * M->NLM);
    M->centre = (double *)malloc(sizeof(double) * P->G);
    orc_ordinates(P->nmu, P->nphi, M->mu, M->wmu, M->dirs, M->W);
    for (int a = 0; a < P->nmu; ++a)
        for (int b = 0; b < P->nphi; ++b) {
            int k = a * P->nphi + b;
            orc_ylm(P->L, M->mu[a], 2.0 * ORC_PI * b / P->nphi, M->Y + (long)k * M->NLM);
        }
    for (int g = 0; g < P->G; ++g) M->centre[g] = sqrt(P->edges[g] * P->edges[g + 1]);
}

static void mesh_free(orc_mesh *M)
{
    free(M->mu); free(M->wmu); free(M->dirs); free(M->W); free(M->Y); free(M->centre);
}

static int is_rest(const double *u) { return u[0] == 0.0 && u[1] == 0.0 && u[2] == 0.0; }

/* Temperature bracket of node c on the tabulated grid: tables i and i+1
 * with weight w of the second, linear in log10(theta), theta clamped into
 * the grid (a node at or below zero temperature takes the first table). */
static void thermal_bracket(const orc_problem *P, long c, int *i, double *w)
{
    double th = P->theta_e[c];
    double x = th > 0.0 ? (log10(th) - P->th_lg0) / P->th_dlg : 0.0;
    if (x < 0.0) x = 0.0;
    if (x > P->nth - 1) x = P->nth - 1;
    int i0 = (int)floor(x);
    if (i0 > P->nth - 2) i0 = P->nth - 2;
    if (i0 < 0) i0 = 0;
    *i = i0;
    *w = P->nth > 1 ? x - i0 : 0.0;
}

/* sigma_out(g) and K_l[g][g'] of node c: the global ones, or with thermal
 * electrons the blend of the node's two bracketing tables. */
static double sigma_out_of(const orc_problem *P, long c, int g)
{
    if (P->nth <= 0) return P->sigma_out[g];
    int i;
    double w;
    thermal_bracket(P, c, &i, &w);
    double a = P->so_th[(long)i * P->G + g];
    double b = P->nth > 1 ? P->so_th[(long)(i + 1) * P->G + g] : a;
    return (1.0 - w) * a + w * b;
}

static double kernel_of(const orc_problem *P, long c, int l, int g, int gp)
{
    int G = P->G;
    if (P->nth <= 0) return P->K[((long)l * G + g) * G + gp];
    int i;
    double w;
    thermal_bracket(P, c, &i, &w);
    long per = (long)(P->L + 1) * G * G;
    double a = P->K_th[(long)i * per + ((long)l * G + g) * G + gp];
    double b = P->nth > 1 ? P->K_th[(long)(i + 1) * per + ((long)l * G + g) * G + gp] : a;
    return (1.0 - w) * a + w * b;
}

/* Comoving extinction chi0(c,g) = alpha0 + n_e sigma_out(g). */
static double chi0_of(const orc_problem *P, long c, int g)
{
    return P->alpha0[c * P->G + g] + P->ne[c] * sigma_out_of(P, c, g);
}

/* Stage a1 + a1': Lorentz-transform the laboratory intensity to comoving
 * ordinates and groups, project onto spherical harmonics, and take the
 * laboratory-frame angular moments (Sec. 2.2 frame order; Sec. 2.3 SH).
 *   I0(k0,g0) = (ebar_g0/eps)^3 I_lab(n(k0), eps),  eps = ebar_g0 (Gamma + u.n_k0)
 *   I_p(g0)   = sum_k0 W_k0 Y_p(n_k0) I0(k0,g0)
 *   J = (1/4pi) sum W I,  H_i = (1/4pi) sum W n_i I,  K_ij = (1/4pi) sum W n_i n_j I
 * K stored as xx, yy, zz, xy, xz, yz.  Any of the outputs may be NULL. */
int orc_project(const orc_problem *P, const double *I, double *Ip, double *J, double *H, double *Kt)
{
    orc_mesh M;
    mesh_init(P, &M);
    long Nc = (long)P->nx * P->ny * P->nz;
    int N = M.N, G = P->G, NLM = M.NLM;
#pragma omp parallel
    {
        double *I0 = (double *)malloc(sizeof(double) * G * N);
        double *A = (double *)malloc(sizeof(double) * G);
#pragma omp for schedule(dynamic, 16)
        for (long c = 0; c < Nc; ++c) {
            const double *Ic = I + c * G * N;
            const double *u = P->u + 3 * c;
            if (is_rest(u)) {
                memcpy(I0, Ic, sizeof(double) * G * N);
            } else {
                for (int k0 = 0; k0 < N; ++k0) {
                    double n[3];
                    double q = orc_comoving_to_lab(u, M.dirs + 3 * k0, n); /* nu/nu0 */
                    for (int g = 0; g < G; ++g) A[g] = orc_interp_angle(P->nmu, P->nphi, M.mu, Ic + (long)g * N, 1, n);
                    for (int g0 = 0; g0 < G; ++g0) {
                        double eps = M.centre[g0] * q;
                        I0[(long)g0 * N + k0] = orc_interp_freq(G, P->edges, A, 1, eps, 0) / (q * q * q);
                    }
                }
            }
            if (Ip) {
                for (int g = 0; g < G; ++g)
                    for (int p = 0; p < NLM; ++p) {
                        double s = 0.0;
                        for (int k = 0; k < N; ++k) s += M.W[k] * M.Y[(long)k * NLM + p] * I0[(long)g * N + k];
                        Ip[(c * G + g) * NLM + p] = s;
                    }
            }
            for (int g = 0; g < G; ++g) {
                double m[10] = {0};
                for (int k = 0; k < N; ++k) {
                    const double *d = M.dirs + 3 * k;
                    double wi = M.W[k] * Ic[(long)g * N + k];
                    m[0] += wi;
                    m[1] += wi * d[0]; m[2] += wi * d[1]; m[3] += wi * d[2];
                    m[4] += wi * d[0] * d[0]; m[5] += wi * d[1] * d[1]; m[6] += wi * d[2] * d[2];
                    m[7] += wi * d[0] * d[1]; m[8] += wi * d[0] * d[2]; m[9] += wi * d[1] * d[2];
                }
                for (int i = 0; i < 10; ++i) m[i] /= 4.0 * ORC_PI;
                if (J) J[c * G + g] = m[0];
                if (H) for (int i = 0; i < 3; ++i) H[(c * G + g) * 3 + i] = m[1 + i];
                if (Kt) for (int i = 0; i < 6; ++i) Kt[(c * G + g) * 6 + i] = m[4 + i];
            }
        }
        free(I0);
        free(A);
    }
    mesh_free(&M);
    return 0;
}

/* Stage a2: comoving source in spherical harmonics (Sec. 2.3)
 *   S_p(c,g) = n_e(c)/chi0(c,g) sum_g' K_l(p)[g][g'] I_p(c,g')
 *              + delta_p0 sqrt(4 pi) eta0(c,g)/chi0(c,g).
 * A node with chi0 = 0 has S = 0.  With thermal electrons K and sigma_out
 * are the node's blend (kernel_of, sigma_out_of). */
int orc_source(const orc_problem *P, const double *Ip, double *Sp)
{
    long Nc = (long)P->nx * P->ny * P->nz;
    int G = P->G, L = P->L, NLM = (L + 1) * (L + 1);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < Nc; ++c) {
        for (int g = 0; g < G; ++g) {
            double chi = chi0_of(P, c, g);
            for (int l = 0; l <= L; ++l)
                for (int m = -l; m <= l; ++m) {
                    int p = l * l + l + m;
                    double s = 0.0;
                    if (chi > 0.0) {
                        double acc = 0.0;
                        for (int gp = 0; gp < G; ++gp) acc += kernel_of(P, c, l, g, gp) * Ip[(c * G + gp) * NLM + p];
                        s = P->ne[c] / chi * acc;
                        if (p == 0) s += sqrt(4.0 * ORC_PI) * P->emis0[c * G + g] / chi;
                    }
                    Sp[(c * G + g) * NLM + p] = s;
                }
        }
    }
    return 0;
}

/* Stage a3: SH -> comoving ordinates, then comoving -> laboratory
 * (Sec. 2.2: S/nu^3 and chi nu are invariant).  For laboratory (c,k,g):
 *   D = nu0/nu = Gamma - u.n_k,  n0 = comoving direction,  eps0 = ebar_g D,
 *   S_lab   = D^-3 S0(n0, eps0)        (angle bilinear, frequency geometric)
 *   chi_lab = D chi0(eps0)
 *   eta_lab = chi_lab S_lab.
 * Outputs eta_lab, chi_lab in [c][g][k]. */
int orc_sh2lab(const orc_problem *P, const double *Sp, double *eta_lab, double *chi_lab)
{
    orc_mesh M;
    mesh_init(P, &M);
    long Nc = (long)P->nx * P->ny * P->nz;
    int N = M.N, G = P->G, NLM = M.NLM;
#pragma omp parallel
    {
        double *S0 = (double *)malloc(sizeof(double) * G * N);
        double *A = (double *)malloc(sizeof(double) * G);
        double *ch = (double *)malloc(sizeof(double) * G);
#pragma omp for schedule(dynamic, 16)
        for (long c = 0; c < Nc; ++c) {
            for (int g = 0; g < G; ++g) {
                ch[g] = chi0_of(P, c, g);
                for (int k = 0; k < N; ++k) {
                    double s = 0.0;
                    for (int p = 0; p < NLM; ++p) s += M.Y[(long)k * NLM + p] * Sp[(c * G + g) * NLM + p];
                    S0[(long)g * N + k] = s;
                }
            }
            const double *u = P->u + 3 * c;
            if (is_rest(u)) {
                for (int g = 0; g < G; ++g)
                    for (int k = 0; k < N; ++k) {
                        long o = (c * G + g) * N + k;
                        chi_lab[o] = ch[g];
                        eta_lab[o] = ch[g] * S0[(long)g * N + k];
                    }
                continue;
            }
            for (int k = 0; k < N; ++k) {
                double n0[3];
                double D = orc_lab_to_comoving(u, M.dirs + 3 * k, n0);
                for (int g = 0; g < G; ++g) A[g] = orc_interp_angle(P->nmu, P->nphi, M.mu, S0 + (long)g * N, 1, n0);
                for (int g = 0; g < G; ++g) {
                    double eps0 = M.centre[g] * D;
                    double s_lab = orc_interp_freq(G, P->edges, A, 1, eps0, 0) / (D * D * D);
                    double c_lab = orc_interp_freq(G, P->edges, ch, 1, eps0, 1) * D;
                    long o = (c * G + g) * N + k;
                    chi_lab[o] = c_lab;
                    eta_lab[o] = c_lab * s_lab;
                }
            }
        }
        free(S0);
        free(A);
        free(ch);
    }
    mesh_free(&M);
    return 0;
}

/* Linear-in-tau short-characteristic weights: with e = exp(-x),
 *   I_P = I_U e + S_P (1 - (1-e)/x) + S_U ((1-e)/x - e).
 * Taylor series below x = 1e-3. */
static void sc_weights(double x, double *e, double *wp, double *wu)
{
    if (x < 1e-3) {
        double x2 = x * x, x3 = x2 * x, x4 = x3 * x;
        *e = 1.0 - x + x2 / 2.0 - x3 / 6.0 + x4 / 24.0;
        *wp = x / 2.0 - x2 / 6.0 + x3 / 24.0 - x4 / 120.0;
        *wu = x / 2.0 - x2 / 3.0 + x3 / 8.0 - x4 / 30.0;
        return;
    }
    double em1 = -expm1(-x); /* 1 - e */
    *e = 1.0 - em1;
    double a0 = em1 / x;
    *wp = 1.0 - a0;
    *wu = a0 - *e;
}

/* Cubic Bezier short characteristic (Sec. 2: the paper's ray tracing uses a
 * cubic Bezier interpolant, after de la Cruz Rodriguez & Piskunov 2013).
 * On a segment of optical depth x from U to P the source is the cubic
 * Bezier curve with end values S_U, S_P and control points C_U, C_P:
 *   S(u) = S_U (1-u)^3 + 3 C_U u (1-u)^2 + 3 C_P u^2 (1-u) + S_P u^3,
 * u = t/x, so that
 *   I_P = I_U e^-x + wU S_U + wCU C_U + wCP C_P + wP S_P,
 * the weights being x times the integrals of the Bernstein polynomials
 * against e^-(x - t) over the segment.  With E_k = int_0^1 v^k e^(-x v) dv
 * (v = 1 - u):  wU = x E3,  wCU = 3x (E2 - E3),  wCP = 3x (E1 - 2E2 + E3),
 * wP = x (E0 - 3E1 + 3E2 - E3).  E_k is summed as its power series
 * sum_m (-x)^m / (m! (k + m + 1)) below x = 1, and from the closed forms
 * E0 = (1 - e)/x, E_k = (k E_(k-1) - e)/x (e = e^-x) above. */
void orc_bezier_weights(double x, double *w /* [5]: e, wU, wCU, wCP, wP */)
{
    double E[4];
    double e = exp(-x);
    if (x < 1.0) {
        for (int k = 0; k < 4; ++k) {
            double term = 1.0, sum = 0.0;
            for (int m = 0; m < 40; ++m) {
                sum += term / (k + m + 1);
                term *= -x / (m + 1);
            }
            E[k] = sum;
        }
    } else {
        E[0] = -expm1(-x) / x;
        for (int k = 1; k < 4; ++k) E[k] = (k * E[k - 1] - e) / x;
    }
    w[0] = e;
    w[1] = x * E[3];
    w[2] = 3.0 * x * (E[2] - E[3]);
    w[3] = 3.0 * x * (E[1] - 2.0 * E[2] + E[3]);
    w[4] = x * (E[0] - 3.0 * E[1] + 3.0 * E[2] - E[3]);
}

/* Derivative of the source along the ray at a node from the slopes of its
 * upwind and downwind segments (optical depths xu, xd): Fritsch and
 * Butland's weighted harmonic mean when both slopes have the same sign,
 *   S' = du dd / (a dd + (1 - a) du),  a = (1 + xd/(xu + xd))/3,
 * else 0 (a local extremum). */
static double fb_derivative(double du, double dd, double xu, double xd)
{
    if (!(du * dd > 0.0)) return 0.0;
    double a = (1.0 + xd / (xu + xd)) / 3.0;
    return du * dd / (a * dd + (1.0 - a) * du);
}

static double clamp_between(double v, double a, double b)
{
    double lo = a < b ? a : b, hi = a < b ? b : a;
    return v < lo ? lo : (v > hi ? hi : v);
}

static double bc_value(const orc_problem *P, long c, int g, int k, int N)
{
    if (P->bc_mode == 1) return P->bc[g];
    if (P->bc_mode == 2) return P->bc[(c * P->G + g) * N + k];
    return 0.0;
}

/* Sweep of one (ordinate k, group g) pair over the whole grid (Sec. 2,
 * eq:shdom; Sec. 2.1, eq:time):
 *   chi~ = chi_lab + kappa,   S~ = (eta_lab + kappa I^n) / chi~,
 * kappa = 1/(c dt).  The upwind point U = P - s n lies on the face crossed
 * first, s = min_a h_a/|n_a|; I, S~ and chi~ at U are bilinear in the four
 * nodes of that face; dtau = s (chi~_U + chi~_P)/2.  Nodes on an inflow face
 * take the boundary intensity.  Nodes are visited in the octant order of n,
 * so every upwind node is final before it is used.  In, eta, chi and out
 * hold element c at index c * stride (out may alias In); St, Ct, Iw and Dw
 * are work arrays of Nc reals.  P->integrator selects the source
 * interpolation along the segment: linear in tau (sc_weights) or the cubic
 * Bezier curve (orc_bezier_weights), whose end derivatives need the
 * downwind point D = P + s n as well and are kept per node in Dw. */
static void sweep_pair(const orc_problem *P, const orc_mesh *M, int k, int g, const double *In, const double *eta_lab,
                       const double *chi_lab, long stride, double *out, double *St, double *Ct, double *Iw,
                       double *Dw)
{
    int nx = P->nx, ny = P->ny, nz = P->nz;
    long Nc = (long)nx * ny * nz;
    int N = M->N;
    int dim[3] = {nx, ny, nz};
    double h[3] = {P->lx / (nx - 1), P->ly / (ny - 1), P->lz / (nz - 1)};
    double kap = P->kappa;
    const double *n = M->dirs + 3 * k;
    /* face crossed first */
    int d = 0;
    double best = fabs(n[0]) / h[0];
    for (int a = 1; a < 3; ++a)
        if (fabs(n[a]) / h[a] > best) { best = fabs(n[a]) / h[a]; d = a; }
    double s = h[d] / fabs(n[d]);
    int sg[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        sg[a] = (n[a] > 0.0) - (n[a] < 0.0);
        fr[a] = s * fabs(n[a]) / h[a];
    }
    int e1 = (d == 0) ? 1 : 0, e2 = (d == 2) ? 1 : 2;
    for (long c = 0; c < Nc; ++c) {
        Ct[c] = chi_lab[c * stride] + kap;
        St[c] = Ct[c] > 0.0 ? (eta_lab[c * stride] + kap * In[c * stride]) / Ct[c] : 0.0;
    }
    int lo[3], hi[3], st[3];
    for (int a = 0; a < 3; ++a) {
        if (sg[a] >= 0) { lo[a] = 0; hi[a] = dim[a]; st[a] = 1; }
        else { lo[a] = dim[a] - 1; hi[a] = -1; st[a] = -1; }
    }
    for (int iz = lo[2]; iz != hi[2]; iz += st[2])
        for (int iy = lo[1]; iy != hi[1]; iy += st[1])
            for (int ix = lo[0]; ix != hi[0]; ix += st[0]) {
                int idx[3] = {ix, iy, iz};
                long c = ((long)iz * ny + iy) * nx + ix;
                int inflow = 0;
                for (int a = 0; a < 3; ++a)
                    if (sg[a] != 0 && idx[a] == (sg[a] > 0 ? 0 : dim[a] - 1)) inflow = 1;
                /* the downwind point D = P + s n (cubic Bezier only): on
                 * the next face along n, bilinear in its four nodes; absent
                 * when any of them lies outside the grid */
                int has_d = 0;
                double sd_ = 0.0, cd_ = 0.0;
                if (P->integrator == 1) {
                    has_d = 1;
                    for (int j1 = 0; j1 < 2 && has_d; ++j1)
                        for (int j2 = 0; j2 < 2; ++j2) {
                            double w = (j1 ? fr[e1] : 1.0 - fr[e1]) * (j2 ? fr[e2] : 1.0 - fr[e2]);
                            if (w == 0.0) continue;
                            int q[3] = {ix, iy, iz};
                            q[d] += sg[d];
                            q[e1] += j1 * sg[e1];
                            q[e2] += j2 * sg[e2];
                            if (q[0] < 0 || q[0] >= nx || q[1] < 0 || q[1] >= ny || q[2] < 0 || q[2] >= nz) {
                                has_d = 0;
                                break;
                            }
                            long cq = ((long)q[2] * ny + q[1]) * nx + q[0];
                            sd_ += w * St[cq];
                            cd_ += w * Ct[cq];
                        }
                }
                double xd = s * 0.5 * (Ct[c] + cd_);
                if (inflow) {
                    Iw[c] = bc_value(P, c, g, k, N);
                    /* an inflow node's derivative is its downwind slope; with
                     * no downwind point either it has none (NaN) */
                    if (P->integrator == 1) Dw[c] = has_d ? (xd > 0.0 ? (sd_ - St[c]) / xd : 0.0) : NAN;
                    continue;
                }
                /* the four face nodes: (e1, e2) offsets 0 or -sg */
                double wsum_i = 0.0, wsum_s = 0.0, wsum_c = 0.0, wsum_d = 0.0, wdv = 0.0;
                for (int j1 = 0; j1 < 2; ++j1)
                    for (int j2 = 0; j2 < 2; ++j2) {
                        double w = (j1 ? fr[e1] : 1.0 - fr[e1]) * (j2 ? fr[e2] : 1.0 - fr[e2]);
                        if (w == 0.0) continue;
                        int q[3] = {ix, iy, iz};
                        q[d] -= sg[d];
                        q[e1] -= j1 * sg[e1];
                        q[e2] -= j2 * sg[e2];
                        long cu = ((long)q[2] * ny + q[1]) * nx + q[0];
                        wsum_i += w * Iw[cu];
                        wsum_s += w * St[cu];
                        wsum_c += w * Ct[cu];
                        if (P->integrator == 1 && !isnan(Dw[cu])) {
                            wsum_d += w * Dw[cu];
                            wdv += w;
                        }
                    }
                double dtau = s * 0.5 * (wsum_c + Ct[c]);
                if (P->integrator == 1) {
                    /* end derivatives: at P by Fritsch-Butland from the
                     * upwind and downwind slopes (the upwind slope alone
                     * without D); at U bilinear in the derivatives kept at
                     * the upwind face nodes that have one (weights
                     * renormalised; the segment's slope if none has).
                     * Control points one third of the segment along them,
                     * clamped into [S_U, S_P] (no overshoot: the curve stays
                     * in their convex hull). */
                    double du = dtau > 0.0 ? (St[c] - wsum_s) / dtau : 0.0;
                    double dp = du;
                    if (has_d) dp = (dtau > 0.0 && xd > 0.0) ? fb_derivative(du, (sd_ - St[c]) / xd, dtau, xd) : 0.0;
                    Dw[c] = dp;
                    double dU = wdv > 0.0 ? wsum_d / wdv : du;
                    double cu = clamp_between(wsum_s + dtau * dU / 3.0, wsum_s, St[c]);
                    double cp = clamp_between(St[c] - dtau * dp / 3.0, wsum_s, St[c]);
                    double w[5];
                    orc_bezier_weights(dtau, w);
                    Iw[c] = wsum_i * w[0] + w[1] * wsum_s + w[2] * cu + w[3] * cp + w[4] * St[c];
                    continue;
                }
                double e, wp, wu;
                sc_weights(dtau, &e, &wp, &wu);
                Iw[c] = wsum_i * e + St[c] * wp + wsum_s * wu;
            }
    for (long c = 0; c < Nc; ++c) out[c * stride] = Iw[c];
}

/* Stage a4: the sweep of every (ordinate, group) pair (sweep_pair), on
 * arrays in the [c][g][k] layout. */
int orc_sweep(const orc_problem *P, const double *In, const double *eta_lab, const double *chi_lab, double *Inew)
{
    orc_mesh M;
    mesh_init(P, &M);
    long Nc = (long)P->nx * P->ny * P->nz;
    int N = M.N, G = P->G;
#pragma omp parallel
    {
        double *St = (double *)malloc(sizeof(double) * Nc);
        double *Ct = (double *)malloc(sizeof(double) * Nc);
        double *Iw = (double *)malloc(sizeof(double) * Nc);
        double *Dw = (double *)malloc(sizeof(double) * Nc);
#pragma omp for schedule(dynamic, 1)
        for (long kg = 0; kg < (long)N * G; ++kg) {
            int k = (int)(kg / G), g = (int)(kg % G);
            long off = (long)g * N + k;
            sweep_pair(P, &M, k, g, In + off, eta_lab + off, chi_lab + off, (long)G * N, Inew + off, St, Ct, Iw,
                       Dw);
        }
        free(St);
        free(Ct);
        free(Iw);
        free(Dw);
    }
    mesh_free(&M);
    return 0;
}

/* Stage a4 for a chosen list of (ordinate kk[i], group gg[i]) pairs only,
 * each on its own column: In, eta_lab, chi_lab and Inew are [i][c].  The
 * arithmetic is sweep_pair's; this form lets a check sample the sweep of a
 * problem whose full [c][g][k] arrays would not fit in host memory. */
int orc_sweep_pairs(const orc_problem *P, int npairs, const int *kk, const int *gg, const double *In,
                    const double *eta_lab, const double *chi_lab, double *Inew)
{
    orc_mesh M;
    mesh_init(P, &M);
    long Nc = (long)P->nx * P->ny * P->nz;
#pragma omp parallel
    {
        double *St = (double *)malloc(sizeof(double) * Nc);
        double *Ct = (double *)malloc(sizeof(double) * Nc);
        double *Iw = (double *)malloc(sizeof(double) * Nc);
        double *Dw = (double *)malloc(sizeof(double) * Nc);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < npairs; ++i) {
            long off = (long)i * Nc;
            sweep_pair(P, &M, kk[i], gg[i], In + off, eta_lab + off, chi_lab + off, 1, Inew + off, St, Ct, Iw, Dw);
        }
        free(St);
        free(Ct);
        free(Iw);
        free(Dw);
    }
    mesh_free(&M);
    return 0;
}

/* Stage a5: FP64 diagnostics of a projected state.
 *   energy  = sum_c sum_g 4 pi J(c,g) de_g
 *   photons = sum_c sum_g 4 pi J(c,g) de_g / ebar_g
 *   resid   = ||S_new - S_old||_2 / ||S_new||_2 over all (c, g, p)
 * (S_old may be NULL, resid is then 0). */
int orc_sums(const orc_problem *P, const double *J, const double *Snew, const double *Sold, double *out3)
{
    long Nc = (long)P->nx * P->ny * P->nz;
    int G = P->G, NLM = (P->L + 1) * (P->L + 1);
    double e = 0.0, ph = 0.0;
    for (long c = 0; c < Nc; ++c)
        for (int g = 0; g < G; ++g) {
            double de = P->edges[g + 1] - P->edges[g];
            double cen = sqrt(P->edges[g] * P->edges[g + 1]);
            e += 4.0 * ORC_PI * J[c * G + g] * de;
            ph += 4.0 * ORC_PI * J[c * G + g] * de / cen;
        }
    double num = 0.0, den = 0.0;
    if (Sold) {
        for (long i = 0; i < Nc * G * NLM; ++i) {
            double d = Snew[i] - Sold[i];
            num += d * d;
            den += Snew[i] * Snew[i];
        }
    }
    out3[0] = e;
    out3[1] = ph;
    out3[2] = (Sold && den > 0.0) ? sqrt(num / den) : 0.0;
    return 0;
}

/* One source iteration per time step (Sec. 2 frame order, Sec. 2.1 time
 * term): project I^n, build the comoving source, transform it to the
 * laboratory ordinates, sweep.  I is updated in place (I^n -> I^{n+1}).
 * Sprev ([c][g][p]) holds the previous iteration's S_p on entry (or NULL)
 * and this step's S_p on return.  sums (optional, 3 doubles) receives
 * energy and photon number of I^n and the relative S change. */
int orc_step(const orc_problem *P, double *I, double *Sprev, double *sums)
{
    long Nc = (long)P->nx * P->ny * P->nz;
    int N = P->nmu * P->nphi, G = P->G, NLM = (P->L + 1) * (P->L + 1);
    long nDO = Nc * G * N, nSH = Nc * G * NLM;
    double *Ip = (double *)malloc(sizeof(double) * nSH);
    double *Sp = (double *)malloc(sizeof(double) * nSH);
    double *J = (double *)malloc(sizeof(double) * Nc * G);
    double *eta = (double *)malloc(sizeof(double) * nDO);
    double *chi = (double *)malloc(sizeof(double) * nDO);
    if (!Ip || !Sp || !J || !eta || !chi) {
        free(Ip); free(Sp); free(J); free(eta); free(chi);
        return -2;
    }
    orc_project(P, I, Ip, J, NULL, NULL);
    orc_source(P, Ip, Sp);
    if (sums) orc_sums(P, J, Sp, Sprev, sums);
    if (Sprev) memcpy(Sprev, Sp, sizeof(double) * nSH);
    orc_sh2lab(P, Sp, eta, chi);
    orc_sweep(P, I, eta, chi, I);
    free(Ip); free(Sp); free(J); free(eta); free(chi);
    return 0;
}
