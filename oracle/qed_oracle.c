/*
 * qed_oracle.c -- plain, slow FP64 CPU oracle of the QED particle step of
 * Gonoskov et al., "Extended PIC schemes for physics in ultra-strong laser
 * fields: review and developments" (arXiv:1412.6426).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests, the smoke check and the timed CPU
 * baseline can compare the CUDA library against an independent, obviously
 * correct statement of the method.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Units ("Compton units"): momentum in m c, energy in m c^2, time in
 * hbar/(m c^2), length in hbar/(m c), electric and magnetic fields in the
 * Sauter-Schwinger field E_S = m^2 c^3/(e hbar) (Sec. V.B).  In these units
 * the bracket [dt e^2 m c / hbar^2] of Eqs. (24), (27), (30) is alpha*dt and
 * the Lorentz force on a charge q (in units of e) is q (E + v x B).
 *
 * Equation numbers follow the paper's sequential numbering:
 *   (3) H_eff, (4) chi, (20)/(21) classical/quantum spectra, (24) P(delta),
 *   (25) P_m, (27)-(29) emission time-step requirements, (30) P_p,
 *   (31) chi_gamma, (32) H_eff for photons, (33) pair time-step requirement.
 *
 * Every function evaluates the definition as written, in FP64, with no
 * tabulation, fusion or reordering beyond what the formula states.
 * Compiled with -ffp-contract=off so that x86 and Arm builds agree bitwise.
 *
 * What pins each part (tests/test_oracle_*.py):
 *   F1, F2          scipy.special.kv + quadrature; x->0 limits from the K_nu
 *                   series; int F1 = 8 pi/(9 sqrt 3); max F2 = 0.607 (paper 0.6)
 *   G, P, P_m       classical power (2/3) chi^2 (1 - 5.95 chi + 48 chi^2);
 *                   0.37 chi^{2/3} at chi >> 1; 0.5176 chi^{2/3} delta^{-2/3}
 *                   (paper 0.52); scipy-K density; max P_m vs Eq. (27)
 *   P_p             Erber small-chi asymptote; delta_e <-> 1-delta_e symmetry
 *   generator       sampled spectrum vs the analytic one down to delta=1e-10
 *   Boris           exact rotation angle (electron, proton, a doubly charged
 *                   ion), exact E acceleration, E x B drift
 *   AEG             few large steps vs many unsubdivided small steps
 *   events          3-momentum exact in uniform E; energy up to the closed-
 *                   form defects in uniform B
 *   pairs, products photons convert at 1 - (1 - int P_p)^N per step and split
 *                   by P_p; products evolve for exactly the rest of the step
 *   boundaries      open boxes absorb and periodic ones wrap on all six faces
 *   ions            pushed only: no emission, no sub-intervals, |p| kept in B
 *   Yee, CIC,       discrete dispersion relation; div B; linear fields exact;
 *   Esirkepov       discrete continuity equation
 *   ensembles       one ensemble reproduces the single-field runs exactly;
 *                   ensembles run together equal ensembles run alone
 *   f_g, N_g        parents' histories identical to f_g = N_g = 1; product
 *                   weight and spectrum unbiased (Sec. VI)
 *   thinning        total weight of each group conserved; groups at or
 *                   below the limit untouched; survivors binomial
 *   Schwinger pairs the pair count of a uniform-field box against the sum of
 *                   P_S (binomial), the unit conversion of R_S V c dt against
 *                   the formula evaluated in SI units, positions uniform in
 *                   the cells, pairs at rest, none in weak fields; on a mesh
 *                   the field at the cell centre
 *   generators      standard (inverse transform): W(x)/W(1) against scipy's
 *                   K-function quadrature, total W(1) against the number
 *                   rate; alternative: P(delta) against Eq. (24); the three
 *                   generators' frozen spectra (the paper's Fig. "generators")
 *   Philox4x32-10   word for word against two independent implementations:
 *                   PyTorch's ATen Philox engine (CPU) and cuRAND's
 *                   curand_Philox4x32_10 (GPU), on 10^4 seeded (counter, key)
 *                   pairs and the all-zero / all-one corners; uniformity and
 *                   decorrelation of the draws are checked statistically.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ALPHA 7.2973525693e-3 /* fine-structure constant, CODATA 2018 */
#define OR_PI 3.14159265358979323846

enum { OR_ELECTRON = 0, OR_POSITRON = 1, OR_PHOTON = 2, OR_ION = 3, OR_NSPECIES = 4 };
enum { OR_PURPOSE_EMIT = 1, OR_PURPOSE_PAIR = 2, OR_PURPOSE_CHILD = 3, OR_PURPOSE_KEEP = 4,
       OR_PURPOSE_THIN = 5, OR_PURPOSE_SCHWINGER = 6 };
#define OR_SCHWINGER_KIND 0x80   /* flag in the product kind of vacuum pairs */
enum { OR_FIELD_GRID = 0, OR_FIELD_UNIFORM = 1, OR_FIELD_GAUSSIAN_LP = 2, OR_FIELD_ROTATING_E = 3,
       OR_FIELD_ENSEMBLE = 4, OR_FIELD_STANDING_WAVE = 5 };
#define OR_ENS_STRIDE 10  /* per ensemble: E0, omega, phase, Eu[3], Bu[3], thin_scale */
/* photon-emission event generators of Sec. IV.F-G */
enum { OR_GEN_MODIFIED = 0, OR_GEN_ALTERNATIVE = 1, OR_GEN_STANDARD = 2 };

/* ------------------------------------------------------------------------ */
/* Synchrotron functions (Sec. IV.E, below Eq. (20) and Eq. (21)):
 *   F1(x) = x * int_x^inf K_{5/3}(t) dt,   F2(x) = x * K_{2/3}(x).
 * Both are evaluated from the integral representations
 *   K_nu(x)            = int_0^inf exp(-x cosh u) cosh(nu u) du,
 *   int_x^inf K_nu(t)dt = int_0^inf exp(-x cosh u) cosh(nu u) / cosh(u) du,
 * by the trapezoidal rule on the half line.  The integrands are even and
 * analytic in a strip around the real axis, so the rule converges
 * exponentially; the step is small enough for the Gaussian core of width
 * 1/sqrt(x) at large x, and the sum runs past the peak at
 * u = asinh((2/3)/x) until the terms fall below 1e-18 of the partial sums. */
void or_synchrotron(double x, double *f1, double *f2)
{
    if (!(x > 0.0)) { *f1 = 0.0; *f2 = 0.0; return; }
    if (x > 745.0) { *f1 = 0.0; *f2 = 0.0; return; } /* exp(-x) underflows */
    double h = 0.5 / sqrt(x);
    if (h > 0.1) h = 0.1;
    double upeak = asinh((2.0 / 3.0) / x);
    double e0 = exp(-x);
    double s1 = 0.5 * e0, s2 = 0.5 * e0; /* u = 0 terms carry weight 1/2 */
    for (long k = 1; k < 2000000; ++k) {
        double u = (double)k * h;
        double e = exp(-x * cosh(u));
        double t1 = e * cosh(5.0 * u / 3.0) / cosh(u);
        double t2 = e * cosh(2.0 * u / 3.0);
        s1 += t1;
        s2 += t2;
        if (u > upeak && t1 <= 1e-18 * s1 && t2 <= 1e-18 * s2) break;
    }
    *f1 = x * h * s1;
    *f2 = x * h * s2;
}

double or_F1(double x) { double a, b; or_synchrotron(x, &a, &b); return a; }
double or_F2(double x) { double a, b; or_synchrotron(x, &a, &b); return b; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
 * Shaw (SC'11), written from its published definition: ten rounds of two
 * 32x32->64 multiplies with the round keys bumped by the Weyl constants. */
static void or_philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        or_philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* A uniform double strictly inside (0,1) from 52 random bits: the top 26 bits
 * of a and of b, offset by one half so that neither 0 nor 1 can occur. */
double or_u52(uint32_t a, uint32_t b)
{
    double k = (double)(a >> 6) * 67108864.0 + (double)(b >> 6);
    return (k + 0.5) * (1.0 / 4503599627370496.0);
}

/* The stream of a particle: key = its 64-bit id, counter = (step, sub-step,
 * purpose, seed).  Returns r1 and r2 for the event generators. */
void or_draw(uint64_t id, uint32_t step, uint32_t sub, uint32_t purpose, uint32_t seed,
             double *r1, double *r2)
{
    uint32_t ctr[4] = {step, sub, purpose, seed};
    uint32_t key[2] = {(uint32_t)id, (uint32_t)(id >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    *r1 = or_u52(o[0], o[1]);
    *r2 = or_u52(o[2], o[3]);
}

/* Identity of a particle created by an event: a Philox mix of the parent id,
 * the step, the sub-step and the child's species, so that ids (and with them
 * the children's random streams) do not depend on the order of creation. */
uint64_t or_child_id(uint64_t parent, uint32_t step, uint32_t sub, uint32_t kind, uint32_t seed)
{
    uint32_t ctr[4] = {step, sub, OR_PURPOSE_CHILD | (kind << 8), seed};
    uint32_t key[2] = {(uint32_t)parent, (uint32_t)(parent >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    return (uint64_t)o[0] | ((uint64_t)o[1] << 32);
}

/* ------------------------------------------------------------------------ */
/* Emission density, Eq. (24), without the prefactor [dt e^2 m c/hbar^2]/gamma:
 *   G(delta, chi) = sqrt(3)/(2 pi) chi (1-delta)/delta
 *                   { F1(z_q) + (3/2) delta chi z_q F2(z_q) },
 *   z_q = (2/3) chi^{-1} delta/(1-delta)            (Eq. (21)). */
double or_G(double delta, double chi)
{
    if (!(delta > 0.0) || !(delta < 1.0) || !(chi > 0.0)) return 0.0;
    double zq = (2.0 / 3.0) / chi * delta / (1.0 - delta);
    double f1, f2;
    or_synchrotron(zq, &f1, &f2);
    return sqrt(3.0) / (2.0 * OR_PI) * chi * (1.0 - delta) / delta
           * (f1 + 1.5 * delta * chi * zq * f2);
}

/* P(delta) of Eq. (24): probability density for emitting delta during dt. */
double or_P(double delta, double chi, double gamma, double dt)
{
    return OR_ALPHA * dt * or_G(delta, chi) / gamma;
}

/* Modified event generator, Eq. (25) with f_m(r1) = r1^3 (Sec. IV.G):
 *   P_m(r1) = f_m'(r1) P(f_m(r1)) = 3 r1^2 P(r1^3). */
double or_Pm(double r1, double chi, double gamma, double dt)
{
    double delta = r1 * r1 * r1;
    return 3.0 * r1 * r1 * or_P(delta, chi, gamma, dt);
}

/* The standard event generator (Sec. IV.F): in an interval dt a photon is
 * emitted when r1 < P = W(1), and its energy delta is the root of
 * W(delta)/W(1) = r2, with
 *   W(x) = dt int_{delta_min}^{x} P(delta)/dt d(delta),
 * the emission probability density P of Eq. (24).  delta_min -> 0: the
 * integrand is integrable (~ delta^{-2/3}) and, written in s = delta^{1/3},
 *   W(x) = int_0^{x^{1/3}} 3 s^2 P(s^3) ds,
 * it is finite at s = 0.  The integrals are 8-point Gauss-Legendre over
 * panels of width 1/256 in s (the integrand is smooth in s); the root is
 * found by bisection on s, integrating panel by panel. */
static double or_gl8_x[8], or_gl8_w[8];

/* P_8(x) and P_8'(x): P_8 and P_7 from the three-term recurrence
 * n P_n = (2n - 1) x P_{n-1} - (n - 1) P_{n-2}, and
 * P_8' = 8 (x P_8 - P_7)/(x^2 - 1). */
static void or_legendre8(double x, double *p8, double *dp8)
{
    double p0 = 1.0, p1 = x;
    for (int n = 2; n <= 8; ++n) {
        double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
    }
    *p8 = p1;
    *dp8 = 8.0 * (x * p1 - p0) / (x * x - 1.0);
}

/* The 8-point Gauss-Legendre rule on [-1, 1]: the nodes are the roots of
 * P_8, found by Newton's method from cos(pi (i + 3/4)/(n + 1/2)); the
 * weights are 2/((1 - x^2) P_8'(x)^2).  Filled once when the library is
 * loaded. */
__attribute__((constructor)) static void or_gl8_init(void)
{
    for (int i = 0; i < 4; ++i) {
        double x = cos(OR_PI * (i + 0.75) / 8.5), p8, dp;
        for (int it = 0; it < 10; ++it) {   /* quadratic convergence: 4 would do */
            or_legendre8(x, &p8, &dp);
            x -= p8 / dp;
        }
        or_legendre8(x, &p8, &dp);
        or_gl8_x[7 - i] = x;
        or_gl8_x[i] = -x;
        or_gl8_w[7 - i] = or_gl8_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* The rule, copied out for its pin. */
void or_gauss_legendre8(double x[8], double w[8])
{
    for (int k = 0; k < 8; ++k) { x[k] = or_gl8_x[k]; w[k] = or_gl8_w[k]; }
}

/* int_a^b 3 s^2 G(s^3, chi) ds, Gauss-Legendre on [a, b] */
static double or_W_piece(double a, double b, double chi)
{
    double m = 0.5 * (a + b), r = 0.5 * (b - a), acc = 0.0;
    for (int k = 0; k < 8; ++k) {
        double s = m + r * or_gl8_x[k];
        acc += or_gl8_w[k] * 3.0 * s * s * or_G(s * s * s, chi);
    }
    return r * acc;
}

#define OR_W_PANELS 256
/* W(x)/(alpha dt/gamma) = int_0^{x^{1/3}} 3 s^2 G(s^3, chi) ds */
double or_Wnorm(double x, double chi)
{
    if (!(x > 0.0) || !(chi > 0.0)) return 0.0;
    if (x > 1.0) x = 1.0;
    double sx = cbrt(x), acc = 0.0;
    for (int k = 0; k < OR_W_PANELS; ++k) {
        double a = (double)k / OR_W_PANELS, b = (double)(k + 1) / OR_W_PANELS;
        if (a >= sx) break;
        acc += or_W_piece(a, b < sx ? b : sx, chi);
    }
    return acc;
}

/* Total probability of the standard generator in an interval dt: W(1). */
double or_Pstd(double chi, double gamma, double dt)
{
    return OR_ALPHA * dt / gamma * or_Wnorm(1.0, chi);
}

/* Photon energy of the standard generator: the root delta of
 * W(delta) / W(1) = r2 (inverse transform sampling). */
double or_delta_std(double chi, double r2)
{
    /* the panel integrals depend on chi only: kept for the latest chi */
    static double panel[OR_W_PANELS], total = 0.0, last_chi = -1.0;
    if (chi != last_chi) {
        total = 0.0;
        for (int k = 0; k < OR_W_PANELS; ++k) {
            panel[k] = or_W_piece((double)k / OR_W_PANELS, (double)(k + 1) / OR_W_PANELS, chi);
            total += panel[k];
        }
        last_chi = chi;
    }
    double target = r2 * total, below = 0.0;
    int k = 0;
    while (k < OR_W_PANELS - 1 && below + panel[k] < target) below += panel[k++];
    double a = (double)k / OR_W_PANELS, b = (double)(k + 1) / OR_W_PANELS;
    for (int it = 0; it < 200 && b - a > 1e-16; ++it) {
        double m = 0.5 * (a + b);
        if (below + or_W_piece((double)k / OR_W_PANELS, m, chi) < target) a = m; else b = m;
    }
    double sr = 0.5 * (a + b);
    return sr * sr * sr;
}

/* Pair-production density, Eq. (30), as printed:
 *   P_p(de) = [dt alpha] sqrt(3)/(2 pi) chi_g/eps_g (de-1) de
 *             { F1(z_p) - (3/2) chi_g z_p F2(z_p) },
 *   z_p = (2/3) / (chi_g (1-de) de),   eps_g = hbar omega/(m c^2). */
double or_Pp(double de, double chig, double epsg, double dt)
{
    if (!(de > 0.0) || !(de < 1.0) || !(chig > 0.0) || !(epsg > 0.0)) return 0.0;
    double zp = (2.0 / 3.0) / (chig * (1.0 - de) * de);
    double f1, f2;
    or_synchrotron(zp, &f1, &f2);
    return OR_ALPHA * dt * sqrt(3.0) / (2.0 * OR_PI) * chig / epsg * (de - 1.0) * de
           * (f1 - 1.5 * chig * zp * f2);
}

/* ------------------------------------------------------------------------ */
/* Lorentz-invariant chi of a lepton, Eq. (4), for momentum p (units m c, so
 * eps/c -> gamma) in fields E, B (units E_S):
 *   chi = sqrt( (gamma E + p x B)^2 - (p . E)^2 ). */
double or_chi(const double p[3], const double E[3], const double B[3])
{
    double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double ax = g * E[0] + (p[1] * B[2] - p[2] * B[1]);
    double ay = g * E[1] + (p[2] * B[0] - p[0] * B[2]);
    double az = g * E[2] + (p[0] * B[1] - p[1] * B[0]);
    double pe = p[0] * E[0] + p[1] * E[1] + p[2] * E[2];
    double s = ax * ax + ay * ay + az * az - pe * pe;
    return s > 0.0 ? sqrt(s) : 0.0;
}

/* Effective field, Eq. (3): H_eff = sqrt((E + v x B)^2 - (p_hat . E)^2),
 * with v = p/gamma (c = 1). */
double or_heff(const double p[3], const double E[3], const double B[3])
{
    double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double pm = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double vx = p[0] / g, vy = p[1] / g, vz = p[2] / g;
    double ax = E[0] + (vy * B[2] - vz * B[1]);
    double ay = E[1] + (vz * B[0] - vx * B[2]);
    double az = E[2] + (vx * B[1] - vy * B[0]);
    double pe = pm > 0.0 ? (p[0] * E[0] + p[1] * E[1] + p[2] * E[2]) / pm : 0.0;
    double s = ax * ax + ay * ay + az * az - pe * pe;
    return s > 0.0 ? sqrt(s) : 0.0;
}

/* Photon effective field, Eq. (32), with k_hat = k/|k|:
 * H^g_eff = sqrt((E + k_hat x B)^2 - (k_hat . E)^2). */
double or_heff_photon(const double k[3], const double E[3], const double B[3])
{
    double km = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    if (!(km > 0.0)) return 0.0;
    double nx = k[0] / km, ny = k[1] / km, nz = k[2] / km;
    double ax = E[0] + (ny * B[2] - nz * B[1]);
    double ay = E[1] + (nz * B[0] - nx * B[2]);
    double az = E[2] + (nx * B[1] - ny * B[0]);
    double ke = nx * E[0] + ny * E[1] + nz * E[2];
    double s = ax * ax + ay * ay + az * az - ke * ke;
    return s > 0.0 ? sqrt(s) : 0.0;
}

/* chi_gamma = (hbar omega/m c^2) H^g_eff / E_S, Eq. (31). */
double or_chi_photon(const double k[3], const double E[3], const double B[3])
{
    double km = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    return km * or_heff_photon(k, E, B);
}

/* Time-step bound of the adaptive generator for a lepton, Eq. (28), scaled by
 * kappa (the paper's "<<").  In Compton units lambda_C/c = 2 pi, so
 * (137/2pi)(lambda_C/c) = 137. */
double or_dtq_lepton(double gamma, double heff, double kappa)
{
    if (!(heff > 0.0)) return INFINITY;
    double a = 0.67 * cbrt(gamma) * pow(1.0 / heff, 2.0 / 3.0);
    double b = 2.0 / heff;
    return kappa * 137.0 * (a < b ? a : b);
}

/* Time-step bound for a photon, Eq. (33), scaled by kappa:
 * dt_q = kappa * 130 (lambda_C/c) (E_S/H^g_eff). */
double or_dtq_photon(double heff_g, double kappa)
{
    if (!(heff_g > 0.0)) return INFINITY;
    return kappa * 130.0 * 2.0 * OR_PI / heff_g;
}

/* Number of sub-intervals: the interval t_span is divided into N equal
 * sub-intervals not longer than dt_q (Sec. IV.H), N limited to nmax. */
int or_nsub(double t_span, double dtq, int nmax, int *capped)
{
    double ratio = t_span / dtq;
    *capped = 0;
    if (!(ratio > 1.0)) return 1;
    double n = ceil(ratio);
    if (n > (double)nmax) { *capped = 1; return nmax; }
    return (int)n;
}

/* ------------------------------------------------------------------------ */
/* Boris pusher (Appendix A): half step in E, full rotation in B, half step
 * in E.  Charge q in units of e, mass m in units of m_e, p in m_e c. */
void or_boris(double p[3], const double E[3], const double B[3], double q, double m, double h)
{
    double a = 0.5 * q * h;
    double um[3] = {p[0] + a * E[0], p[1] + a * E[1], p[2] + a * E[2]};
    double gm = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) / (m * m));
    double f = a / (m * gm);
    double t[3] = {f * B[0], f * B[1], f * B[2]};
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
    double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),
                    um[1] + (um[2] * t[0] - um[0] * t[2]),
                    um[2] + (um[0] * t[1] - um[1] * t[0])};
    double uq[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),
                    um[1] + (up[2] * s[0] - up[0] * s[2]),
                    um[2] + (up[0] * s[1] - up[1] * s[0])};
    p[0] = uq[0] + a * E[0];
    p[1] = uq[1] + a * E[1];
    p[2] = uq[2] + a * E[2];
}

/* ------------------------------------------------------------------------ */
/* Analytic external fields for test-particle runs (the paper does not fix
 * them; these are the textbook forms the workloads name).
 *  UNIFORM      fp = {Ex,Ey,Ez,Bx,By,Bz}
 *  GAUSSIAN_LP  linearly polarised paraxial Gaussian pulse travelling along
 *               -x, E along y, B = -E along z:
 *               fp = {E0, omega, w0, tau_fwhm_intensity, xf, yf, zf, tf, phi0}
 *  ROTATING_E   E = E0 (cos wt, sin wt, 0), B = 0: fp = {E0, omega}
 *  STANDING_WAVE  plane standing wave along x of the avalanche cascade
 *               (Sec. V): E_y = E0 sin(omega x) cos(omega t),
 *               B_z = -E0 cos(omega x) sin(omega t) (so that at t = 0 only
 *               E_y = E0 sin(2 pi x / lambda) is present): fp = {E0, omega} */
void or_field(int mode, const double *fp, const double x[3], double t, double E[3], double B[3])
{
    E[0] = E[1] = E[2] = 0.0;
    B[0] = B[1] = B[2] = 0.0;
    if (mode == OR_FIELD_UNIFORM) {
        E[0] = fp[0]; E[1] = fp[1]; E[2] = fp[2];
        B[0] = fp[3]; B[1] = fp[4]; B[2] = fp[5];
    } else if (mode == OR_FIELD_GAUSSIAN_LP) {
        double E0 = fp[0], w = fp[1], w0 = fp[2], tau = fp[3];
        double zeta = fp[4] - x[0];               /* distance past focus along -x */
        double zr = 0.5 * w * w0 * w0;            /* Rayleigh length, k = omega */
        double wz = w0 * sqrt(1.0 + (zeta / zr) * (zeta / zr));
        double dy = x[1] - fp[5], dz = x[2] - fp[6];
        double r2 = dy * dy + dz * dz;
        double invR = zeta / (zeta * zeta + zr * zr);
        double gouy = atan(zeta / zr);
        double eta = (t - fp[7]) - zeta;          /* retarded time */
        double phase = w * eta - 0.5 * w * r2 * invR + gouy + fp[8];
        double env = exp(-2.0 * log(2.0) * eta * eta / (tau * tau));
        double amp = E0 * (w0 / wz) * exp(-r2 / (wz * wz)) * env;
        E[1] = amp * cos(phase);
        B[2] = -E[1];
    } else if (mode == OR_FIELD_ROTATING_E) {
        E[0] = fp[0] * cos(fp[1] * t);
        E[1] = fp[0] * sin(fp[1] * t);
    } else if (mode == OR_FIELD_STANDING_WAVE) {
        E[1] = fp[0] * sin(fp[1] * x[0]) * cos(fp[1] * t);
        B[2] = -fp[0] * cos(fp[1] * x[0]) * sin(fp[1] * t);
    }
}

/* ------------------------------------------------------------------------ */
/* Yee mesh (Appendix C, FDTD; Yee 1966).  Arrays are n0*n1*n2 doubles,
 * x fastest: idx = (k*n1 + j)*n0 + i.  Component positions in cell units:
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)   (J likewise)
 *   Bx (i, j+1/2, k+1/2) By (i+1/2, j, k+1/2) Bz (i+1/2, j+1/2, k)
 * Periodic in all three directions. */
static long or_wrap(long i, long n) { i %= n; return i < 0 ? i + n : i; }
static long or_idx(const int32_t n[3], long i, long j, long k)
{
    return (or_wrap(k, n[2]) * n[1] + or_wrap(j, n[1])) * n[0] + or_wrap(i, n[0]);
}

static void or_curl_e(const int32_t n[3], const double d[3], double *const E[3], double *out[3])
{
    for (long k = 0; k < n[2]; ++k)
        for (long j = 0; j < n[1]; ++j)
            for (long i = 0; i < n[0]; ++i) {
                long c = or_idx(n, i, j, k);
                out[0][c] = (E[2][or_idx(n, i, j + 1, k)] - E[2][c]) / d[1]
                          - (E[1][or_idx(n, i, j, k + 1)] - E[1][c]) / d[2];
                out[1][c] = (E[0][or_idx(n, i, j, k + 1)] - E[0][c]) / d[2]
                          - (E[2][or_idx(n, i + 1, j, k)] - E[2][c]) / d[0];
                out[2][c] = (E[1][or_idx(n, i + 1, j, k)] - E[1][c]) / d[0]
                          - (E[0][or_idx(n, i, j + 1, k)] - E[0][c]) / d[1];
            }
}

static void or_curl_b(const int32_t n[3], const double d[3], double *const B[3], double *out[3])
{
    for (long k = 0; k < n[2]; ++k)
        for (long j = 0; j < n[1]; ++j)
            for (long i = 0; i < n[0]; ++i) {
                long c = or_idx(n, i, j, k);
                out[0][c] = (B[2][c] - B[2][or_idx(n, i, j - 1, k)]) / d[1]
                          - (B[1][c] - B[1][or_idx(n, i, j, k - 1)]) / d[2];
                out[1][c] = (B[0][c] - B[0][or_idx(n, i, j, k - 1)]) / d[2]
                          - (B[2][c] - B[2][or_idx(n, i - 1, j, k)]) / d[0];
                out[2][c] = (B[1][c] - B[1][or_idx(n, i - 1, j, k)]) / d[0]
                          - (B[0][c] - B[0][or_idx(n, i, j - 1, k)]) / d[1];
            }
}

/* One FDTD step, symmetrised in time (Appendix A): B half step, E full step
 * with the current, B half step.  Maxwell in Compton units:
 *   dB/dt = -curl E,   dE/dt = curl B - 4 pi alpha J,
 * with J the number-current density (charge in e, velocity in c, per
 * (hbar/mc)^3).  f = {Ex,Ey,Ez,Bx,By,Bz}, J = {Jx,Jy,Jz}. */
int or_yee_step(const int32_t n[3], const double d[3], double dt, double *f[6], double *const J[3])
{
    long nc = (long)n[0] * n[1] * n[2];
    double *tmp[3];
    for (int c = 0; c < 3; ++c) {
        tmp[c] = (double *)malloc(sizeof(double) * nc);
        if (!tmp[c]) return -1;
    }
    double *E[3] = {f[0], f[1], f[2]};
    double *B[3] = {f[3], f[4], f[5]};
    or_curl_e(n, d, E, tmp);
    for (int c = 0; c < 3; ++c)
        for (long q = 0; q < nc; ++q) B[c][q] -= 0.5 * dt * tmp[c][q];
    or_curl_b(n, d, B, tmp);
    for (int c = 0; c < 3; ++c)
        for (long q = 0; q < nc; ++q) E[c][q] += dt * (tmp[c][q] - 4.0 * OR_PI * OR_ALPHA * J[c][q]);
    or_curl_e(n, d, E, tmp);
    for (int c = 0; c < 3; ++c)
        for (long q = 0; q < nc; ++q) B[c][q] -= 0.5 * dt * tmp[c][q];
    for (int c = 0; c < 3; ++c) free(tmp[c]);
    return 0;
}

/* Linear (CIC) interpolation of one staggered component at index-space
 * position u (cell units from the lattice origin), stagger s in {0, 1/2}. */
static double or_cic_one(const int32_t n[3], const double *a, const double u[3], const double s[3])
{
    double v[3], fr[3];
    long b[3];
    for (int c = 0; c < 3; ++c) {
        v[c] = u[c] - s[c];
        b[c] = (long)floor(v[c]);
        fr[c] = v[c] - (double)b[c];
    }
    double acc = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double wgt = (di ? fr[0] : 1.0 - fr[0]) * (dj ? fr[1] : 1.0 - fr[1])
                           * (dk ? fr[2] : 1.0 - fr[2]);
                acc += wgt * a[or_idx(n, b[0] + di, b[1] + dj, b[2] + dk)];
            }
    return acc;
}

/* CIC gather (Appendix C) of E and B at absolute position x. */
void or_gather(const int32_t n[3], const double d[3], const double x0[3], double *const f[6],
               const double x[3], double E[3], double B[3])
{
    static const double st[6][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},
                                     {0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};
    double u[3] = {(x[0] - x0[0]) / d[0], (x[1] - x0[1]) / d[1], (x[2] - x0[2]) / d[2]};
    for (int c = 0; c < 3; ++c) E[c] = or_cic_one(n, f[c], u, st[c]);
    for (int c = 0; c < 3; ++c) B[c] = or_cic_one(n, f[3 + c], u, st[3 + c]);
}

/* Esirkepov charge-conserving deposit (Appendix C) with the linear shape
 * S(v) = max(0, 1-|v|), for a particle of charge q*w moving from xa to xb
 * (absolute, unwrapped; |xb-xa| below one cell per axis) during dt.
 * Adds the number-current density to J. */
static double or_shape(double v) { double a = fabs(v); return a < 1.0 ? 1.0 - a : 0.0; }

void or_deposit(const int32_t n[3], const double d[3], const double x0[3], double *J[3],
                const double xa[3], const double xb[3], double qw, double dt)
{
    double ua[3], ub[3];
    long base[3];
    double S0[3][4], S1[3][4], dS[3][4];
    for (int c = 0; c < 3; ++c) {
        ua[c] = (xa[c] - x0[c]) / d[c];
        ub[c] = (xb[c] - x0[c]) / d[c];
        base[c] = (long)floor(ua[c]) - 1;
        for (int m = 0; m < 4; ++m) {
            S0[c][m] = or_shape(ua[c] - (double)(base[c] + m));
            S1[c][m] = or_shape(ub[c] - (double)(base[c] + m));
            dS[c][m] = S1[c][m] - S0[c][m];
        }
    }
    double dV = d[0] * d[1] * d[2];
    /* Jx: cumulative along x */
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int i = 0; i < 4; ++i) {
                double W = dS[0][i] * (S0[1][j] * S0[2][k] + 0.5 * dS[1][j] * S0[2][k]
                                       + 0.5 * S0[1][j] * dS[2][k] + dS[1][j] * dS[2][k] / 3.0);
                acc -= qw * d[0] / (dt * dV) * W;
                J[0][or_idx(n, base[0] + i, base[1] + j, base[2] + k)] += acc;
            }
        }
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 4; ++i) {
            double acc = 0.0;
            for (int j = 0; j < 4; ++j) {
                double W = dS[1][j] * (S0[0][i] * S0[2][k] + 0.5 * dS[0][i] * S0[2][k]
                                       + 0.5 * S0[0][i] * dS[2][k] + dS[0][i] * dS[2][k] / 3.0);
                acc -= qw * d[1] / (dt * dV) * W;
                J[1][or_idx(n, base[0] + i, base[1] + j, base[2] + k)] += acc;
            }
        }
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) {
                double W = dS[2][k] * (S0[0][i] * S0[1][j] + 0.5 * dS[0][i] * S0[1][j]
                                       + 0.5 * S0[0][i] * dS[1][j] + dS[0][i] * dS[1][j] / 3.0);
                acc -= qw * d[2] / (dt * dV) * W;
                J[2][or_idx(n, base[0] + i, base[1] + j, base[2] + k)] += acc;
            }
        }
}

/* Charge density rho = sum q w S(x - x_node)/dV at the nodes (for tests of
 * the continuity equation). */
void or_charge_density(const int32_t n[3], const double d[3], const double x0[3], double *rho,
                       const double *x, const double *y, const double *z, const double *qw, long np)
{
    double dV = d[0] * d[1] * d[2];
    for (long p = 0; p < np; ++p) {
        double u[3] = {(x[p] - x0[0]) / d[0], (y[p] - x0[1]) / d[1], (z[p] - x0[2]) / d[2]};
        long b[3];
        double fr[3];
        for (int c = 0; c < 3; ++c) { b[c] = (long)floor(u[c]); fr[c] = u[c] - (double)b[c]; }
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    double wgt = (di ? fr[0] : 1.0 - fr[0]) * (dj ? fr[1] : 1.0 - fr[1])
                               * (dk ? fr[2] : 1.0 - fr[2]);
                    rho[or_idx(n, b[0] + di, b[1] + dj, b[2] + dk)] += qw[p] * wgt / dV;
                }
    }
}

/* ------------------------------------------------------------------------ */
/* The particle step.                                                        */

typedef struct {
    int32_t n[3];            /* lattice (grid) size */
    int32_t periodic[3];     /* 1 periodic, 0 open (particles leaving are removed) */
    int32_t field_mode;      /* OR_FIELD_* */
    int32_t nsub_max;        /* cap on sub-intervals per step */
    int32_t emission_on;
    int32_t pairs_on;
    int32_t same_step_children; /* 1: products evolve for the rest of the step */
    int32_t deposit_on;      /* 1: Esirkepov deposit into J (grid mode) */
    uint32_t seed;
    int32_t nbins;           /* photon spectrum bins (log10 delta) */
    double d[3];             /* cell size */
    double x0[3];            /* lattice origin */
    double kappa;            /* dt_q = kappa * (bound of Eq. (28) / (33)) */
    double lg_lo, lg_hi;     /* log10(delta) range of the spectrum */
    double charge[4], mass[4];
    double fp[16];           /* analytic field parameters */
    /* independent ensembles (OR_FIELD_ENSEMBLE): the top ens_bits bits of an
     * id name the particle's ensemble; products keep their parent's bits */
    int32_t ens_bits;        /* 0..16; 0 = no ensembles */
    int32_t n_ens;
    const double *ens;       /* n_ens x OR_ENS_STRIDE; thin_scale > 0 scales the
                              * thinning limits of the ensemble's group */
    /* tunable generator factors of Sec. VI (values <= 1 mean 1) */
    double emit_fg, pair_fg; /* product kept with probability 1/f_g, weight x f_g */
    int32_t emit_ng, pair_ng;/* N_g product samples per occasion, weight / N_g */
    /* thinning with global even redistribution (Sec. VI) */
    int32_t thin_interval;   /* thin after every step s with (s+1) % interval == 0 */
    int32_t reserved;
    int64_t thin_limit[4];   /* per species: most particles a group keeps (0 = off) */
    int32_t generator;       /* OR_GEN_*: modified (default), alternative, standard */
    int32_t reserved2;
    int32_t schwinger_on;    /* pairs from the vacuum per cell (Sec. V.B) */
    int32_t reserved3;
    double schwinger_weight; /* weight of those electrons and positrons */
} or_params;

typedef struct {
    int64_t n, cap;
    double *x, *y, *z, *px, *py, *pz, *w;
    uint64_t *id;
} or_store;

typedef struct {
    int64_t emissions, pairs, substeps_lepton, substeps_photon;
    int64_t pm_gt1, pp_gt1, capped, absorbed, overflow, nonfinite;
    int64_t photons_created; /* photons made (all N_g samples, after the 1/f_g keep) */
    int64_t pairs_created;   /* pairs made, likewise */
    int64_t thinned;         /* particles removed by thinning */
    int64_t schwinger_pairs; /* pairs created from the vacuum */
    int64_t schwinger_gt1;   /* cells with P_S > 1 */
    double energy_defect;    /* sum of w*(energy before - energy after) over events */
    double *spectrum;        /* nbins, weighted by w, over log10(delta) */
    double *spectrum_energy; /* nbins, weighted by w, over log10(photon energy) with the same range */
    /* optional (test infrastructure): along the realised trajectories, the
     * expected number of photons in each spectrum bin, sum over lepton
     * sub-intervals of w * int_bin P(delta) d delta (Eq. (24)), and the sum of
     * w^2 p (1 - p), its variance (modified generator, trivial factors) */
    double *expected;
    double *expected_var;
} or_diag;

typedef struct {
    const or_params *P;
    or_store *S;
    or_diag *D;
    double *const *f;        /* Yee fields (grid mode) */
    double **J;
    uint32_t step;
    double t, dt;
} or_ctx;

typedef struct {
    double x[3], p[3], w;
    uint64_t id;
    int alive;
} or_particle;

/* Ensemble of a particle: the top ens_bits bits of its id (0 without). */
static uint32_t or_ensemble(const or_params *P, uint64_t id)
{
    return P->ens_bits > 0 ? (uint32_t)(id >> (64 - P->ens_bits)) : 0u;
}

/* Id of a product: or_child_id of the parent, with the parent's ensemble
 * bits kept so that products stay in their parent's ensemble.  kind is the
 * product species plus (sample << 8) for the extra samples of N_g. */
static uint64_t or_product_id(const or_params *P, uint64_t parent, uint32_t step, uint32_t sub,
                              uint32_t kind)
{
    uint64_t mix = or_child_id(parent, step, sub, kind, P->seed);
    if (P->ens_bits <= 0) return mix;
    uint64_t hi = ~(uint64_t)0 << (64 - P->ens_bits);
    return (parent & hi) | (mix & ~hi);
}

/* Field of ensemble e at time t: a uniform part plus a rotating E,
 *   E = Eu + E0 (cos(omega t + phase), sin(omega t + phase), 0),  B = Bu.
 * A particle whose ensemble has no table row sees no field. */
void or_field_ensemble(const or_params *P, uint64_t id, double t, double E[3], double B[3])
{
    uint32_t e = or_ensemble(P, id);
    E[0] = E[1] = E[2] = 0.0;
    B[0] = B[1] = B[2] = 0.0;
    if (!P->ens || e >= (uint32_t)P->n_ens) return;
    const double *q = P->ens + (size_t)OR_ENS_STRIDE * e;
    double ph = q[1] * t + q[2];
    E[0] = q[3] + q[0] * cos(ph);
    E[1] = q[4] + q[0] * sin(ph);
    E[2] = q[5];
    B[0] = q[6]; B[1] = q[7]; B[2] = q[8];
}

/* Generator factor f_g (Sec. VI): a product of an accepted draw is kept
 * with probability 1/f_g.  Draws a uniform only when f_g > 1. */
static int or_keep(const or_params *P, double fg, uint64_t id, uint32_t step, uint32_t sub,
                   uint32_t sample, uint32_t generator)
{
    if (!(fg > 1.0)) return 1;
    double u, unused;
    or_draw(id, step, sub, OR_PURPOSE_KEEP | (sample << 8) | (generator << 16), P->seed, &u, &unused);
    return u < 1.0 / fg;
}

static double or_fg(double fg) { return fg > 1.0 ? fg : 1.0; }
static int or_ng(int32_t ng) { return ng > 1 ? (int)ng : 1; }

/* Probability that the sub-interval of length h emits a photon with delta in
 * each spectrum bin: int_bin P(delta) d delta, by 6-point Gauss-Legendre in
 * ln delta per bin (P = alpha h G / gamma, Eq. (24)); the modified generator
 * emits with exactly this probability when P_m <= 1 (Sec. IV.G). */
static void or_expect_add(or_ctx *C, double chi, double gamma, double h, double w)
{
    static const double x6[6] = {-0.9324695142031521, -0.6612093864662645, -0.2386191860831969,
                                 0.2386191860831969, 0.6612093864662645, 0.9324695142031521};
    static const double w6[6] = {0.1713244923791704, 0.3607615730481386, 0.4679139345726910,
                                 0.4679139345726910, 0.3607615730481386, 0.1713244923791704};
    const or_params *P = C->P;
    const double span = (P->lg_hi - P->lg_lo) / P->nbins;
    for (int b = 0; b < P->nbins; ++b) {
        double ua = (P->lg_lo + b * span) * log(10.0), ub = (P->lg_lo + (b + 1) * span) * log(10.0);
        if (ua >= 0.0) break;                       /* delta < 1 */
        if (ub > 0.0) ub = 0.0;
        double mid = 0.5 * (ua + ub), half = 0.5 * (ub - ua), sum = 0.0;
        for (int k = 0; k < 6; ++k) {
            double delta = exp(mid + half * x6[k]);
            if (delta >= 1.0) continue;
            sum += w6[k] * or_P(delta, chi, gamma, h) * delta;
        }
        double pb = sum * half;
        C->D->expected[b] += w * pb;
        C->D->expected_var[b] += w * w * pb * (1.0 - pb);
    }
}

static void or_spectrum_add(or_ctx *C, double delta, double eps, double w)
{
    const or_params *P = C->P;
    if (P->nbins <= 0 || !C->D->spectrum) return;
    double span = P->lg_hi - P->lg_lo;
    double a = (log10(delta) - P->lg_lo) / span * P->nbins;
    if (a >= 0.0 && a < P->nbins) C->D->spectrum[(long)a] += w;
    if (C->D->spectrum_energy) {
        double b = (log10(eps) - P->lg_lo) / span * P->nbins;
        if (b >= 0.0 && b < P->nbins) C->D->spectrum_energy[(long)b] += w;
    }
}

static int or_append(or_ctx *C, int sp, const or_particle *q)
{
    or_store *s = &C->S[sp];
    if (s->n >= s->cap) { C->D->overflow++; return -1; }
    int64_t i = s->n++;
    s->x[i] = q->x[0]; s->y[i] = q->x[1]; s->z[i] = q->x[2];
    s->px[i] = q->p[0]; s->py[i] = q->p[1]; s->pz[i] = q->p[2];
    s->w[i] = q->w; s->id[i] = q->id;
    return (int)sp;
}

/* End-of-step boundary: periodic wrap, or removal when outside an open box. */
static void or_boundary(or_ctx *C, or_particle *q)
{
    const or_params *P = C->P;
    for (int c = 0; c < 3; ++c) {
        double lo = P->x0[c], L = P->d[c] * (double)P->n[c];
        if (P->periodic[c]) {
            double u = floor((q->x[c] - lo) / L);
            q->x[c] -= u * L;
        } else if (q->x[c] < lo || q->x[c] >= lo + L) {
            q->alive = 0;
        }
    }
    if (!q->alive) C->D->absorbed++;
}

static void or_process(or_ctx *C, int sp, or_particle *q, double t_span,
                       const double E[3], const double B[3], int children_now);

static void or_emit_child(or_ctx *C, int sp, or_particle *child, double t_rem,
                          const double E[3], const double B[3])
{
    const or_params *P = C->P;
    if (P->same_step_children && t_rem > 0.0) {
        or_process(C, sp, child, t_rem, E, B, 1);
    } else {
        or_boundary(C, child);
    }
    if (child->alive) or_append(C, sp, child);
}

/* Lepton: adaptive event generator (Sec. IV.H) around the modified event
 * generator (Sec. IV.G), with the fields frozen over the interval.
 * Photon: the pair event generator of Sec. V.A in the same sub-interval loop.
 * Ion: Boris push only.  The deposit uses the start and end positions. */
static void or_process(or_ctx *C, int sp, or_particle *q, double t_span,
                       const double E[3], const double B[3], int children_now)
{
    const or_params *P = C->P;
    double xs[3] = {q->x[0], q->x[1], q->x[2]};
    (void)children_now;
    if (sp == OR_ELECTRON || sp == OR_POSITRON || sp == OR_ION) {
        double qc = P->charge[sp], m = P->mass[sp];
        int n = 1, capped = 0;
        int qed = (sp != OR_ION) && P->emission_on;
        if (qed) {
            double g0 = sqrt(1.0 + q->p[0] * q->p[0] + q->p[1] * q->p[1] + q->p[2] * q->p[2]);
            double heff = or_heff(q->p, E, B);
            n = or_nsub(t_span, or_dtq_lepton(g0, heff, P->kappa), P->nsub_max, &capped);
            if (capped) C->D->capped++;
        }
        double h = t_span / (double)n;
        for (int s = 0; s < n; ++s) {
            or_boris(q->p, E, B, qc, m, h);
            double g = sqrt(1.0 + (q->p[0] * q->p[0] + q->p[1] * q->p[1] + q->p[2] * q->p[2]) / (m * m));
            for (int c = 0; c < 3; ++c) q->x[c] += q->p[c] / (m * g) * h;
            if (!qed) continue;
            C->D->substeps_lepton++;
            double chi = or_chi(q->p, E, B);
            double r1, r2;
            or_draw(q->id, C->step, (uint32_t)s, OR_PURPOSE_EMIT, P->seed, &r1, &r2);
            if (P->generator == OR_GEN_ALTERNATIVE || P->generator == OR_GEN_STANDARD) {
                /* the unmodified generators of Sec. IV.F */
                double delta, pe;
                int fire;
                if (P->generator == OR_GEN_ALTERNATIVE) {
                    delta = r1;                          /* r2 < P(r1), delta = r1 */
                    pe = or_P(r1, chi, g, h);
                    fire = r2 < pe;
                } else {
                    pe = or_Pstd(chi, g, h);             /* r1 < W(1), W(delta)/W(1) = r2 */
                    fire = r1 < pe;
                    delta = fire ? or_delta_std(chi, r2) : 0.0;
                }
                if (pe > 1.0) C->D->pm_gt1++;
                if (fire) {
                    double p0[3] = {q->p[0], q->p[1], q->p[2]};
                    or_particle ph;
                    for (int c = 0; c < 3; ++c) { ph.x[c] = q->x[c]; ph.p[c] = delta * p0[c]; }
                    ph.w = q->w;
                    ph.id = or_product_id(P, q->id, C->step, (uint32_t)s, OR_PHOTON);
                    ph.alive = 1;
                    double e_before = sqrt(m * m + p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2]);
                    for (int c = 0; c < 3; ++c) q->p[c] = (1.0 - delta) * p0[c];
                    C->D->emissions++;
                    C->D->photons_created++;
                    double eps = sqrt(ph.p[0] * ph.p[0] + ph.p[1] * ph.p[1] + ph.p[2] * ph.p[2]);
                    double e_after = sqrt(m * m + q->p[0] * q->p[0] + q->p[1] * q->p[1] + q->p[2] * q->p[2]);
                    C->D->energy_defect += q->w * (e_before - e_after - eps);
                    or_spectrum_add(C, delta, eps, ph.w);
                    or_emit_child(C, OR_PHOTON, &ph, (double)(n - 1 - s) * h, E, B);
                }
                continue;
            }
            if (C->D->expected && C->D->expected_var && P->nbins > 0) or_expect_add(C, chi, g, h, q->w);
            double pm = or_Pm(r1, chi, g, h);
            if (pm > 1.0) C->D->pm_gt1++;
            /* Products (Sec. VI): N_g samples of the generator, sample 0 being
             * the parent's own draw; each accepted sample makes a photon
             * along p carrying delta = a1^3 of it, kept with probability
             * 1/f_g, with weight w f_g / N_g. */
            double p0[3] = {q->p[0], q->p[1], q->p[2]};
            int ng = or_ng(P->emit_ng);
            double fg = or_fg(P->emit_fg);
            for (int j = 0; j < ng; ++j) {
                double a1 = r1, a2 = r2, pmj = pm;
                if (j > 0) {
                    or_draw(q->id, C->step, (uint32_t)s, OR_PURPOSE_EMIT | ((uint32_t)j << 8), P->seed, &a1, &a2);
                    pmj = or_Pm(a1, chi, g, h);
                    if (pmj > 1.0) C->D->pm_gt1++;
                }
                if (!(a2 < pmj)) continue;
                if (!or_keep(P, fg, q->id, C->step, (uint32_t)s, (uint32_t)j, 0u)) continue;
                double delta = a1 * a1 * a1;
                or_particle ph;
                for (int c = 0; c < 3; ++c) { ph.x[c] = q->x[c]; ph.p[c] = delta * p0[c]; }
                ph.w = q->w * (fg / (double)ng);
                ph.id = or_product_id(P, q->id, C->step, (uint32_t)s, OR_PHOTON | ((uint32_t)j << 8));
                ph.alive = 1;
                C->D->photons_created++;
                double eps = sqrt(ph.p[0] * ph.p[0] + ph.p[1] * ph.p[1] + ph.p[2] * ph.p[2]);
                or_spectrum_add(C, delta, eps, ph.w);
                or_emit_child(C, OR_PHOTON, &ph, (double)(n - 1 - s) * h, E, B);
            }
            if (r2 < pm) {
                /* The parent's event: it keeps (1 - delta) of its momentum. */
                double delta = r1 * r1 * r1;
                double e_before = sqrt(m * m + p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2]);
                for (int c = 0; c < 3; ++c) q->p[c] = (1.0 - delta) * p0[c];
                C->D->emissions++;
                double k[3] = {delta * p0[0], delta * p0[1], delta * p0[2]};
                double eps = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
                double e_after = sqrt(m * m + q->p[0] * q->p[0] + q->p[1] * q->p[1] + q->p[2] * q->p[2]);
                C->D->energy_defect += q->w * (e_before - e_after - eps);
            }
        }
    } else { /* photon */
        double eps = sqrt(q->p[0] * q->p[0] + q->p[1] * q->p[1] + q->p[2] * q->p[2]);
        double hg = or_heff_photon(q->p, E, B);
        double chig = eps * hg;
        int n = 1, capped = 0;
        if (P->pairs_on) {
            n = or_nsub(t_span, or_dtq_photon(hg, P->kappa), P->nsub_max, &capped);
            if (capped) C->D->capped++;
        }
        double h = t_span / (double)n;
        for (int s = 0; s < n; ++s) {
            if (eps > 0.0)
                for (int c = 0; c < 3; ++c) q->x[c] += q->p[c] / eps * h;
            if (!P->pairs_on) continue;
            C->D->substeps_photon++;
            double r1, r2;
            or_draw(q->id, C->step, (uint32_t)s, OR_PURPOSE_PAIR, P->seed, &r1, &r2);
            double pp = or_Pp(r1, chig, eps, h);
            if (pp > 1.0) C->D->pp_gt1++;
            /* Products (Sec. VI): N_g samples, sample 0 being the photon's own
             * draw; each accepted sample makes an electron with a1 of the
             * photon momentum and a positron with 1 - a1, kept with
             * probability 1/f_g, with weight w f_g / N_g. */
            int ng = or_ng(P->pair_ng);
            double fg = or_fg(P->pair_fg);
            double t_rem = (double)(n - 1 - s) * h;
            for (int j = 0; j < ng; ++j) {
                double a1 = r1, a2 = r2, ppj = pp;
                if (j > 0) {
                    or_draw(q->id, C->step, (uint32_t)s, OR_PURPOSE_PAIR | ((uint32_t)j << 8), P->seed, &a1, &a2);
                    ppj = or_Pp(a1, chig, eps, h);
                    if (ppj > 1.0) C->D->pp_gt1++;
                }
                if (!(a2 < ppj)) continue;
                if (!or_keep(P, fg, q->id, C->step, (uint32_t)s, (uint32_t)j, 1u)) continue;
                or_particle el, po;
                for (int c = 0; c < 3; ++c) {
                    el.x[c] = po.x[c] = q->x[c];
                    el.p[c] = a1 * q->p[c];
                    po.p[c] = (1.0 - a1) * q->p[c];
                }
                el.w = po.w = q->w * (fg / (double)ng);
                el.id = or_product_id(P, q->id, C->step, (uint32_t)s, OR_ELECTRON | ((uint32_t)j << 8));
                po.id = or_product_id(P, q->id, C->step, (uint32_t)s, OR_POSITRON | ((uint32_t)j << 8));
                el.alive = po.alive = 1;
                C->D->pairs_created++;
                or_emit_child(C, OR_ELECTRON, &el, t_rem, E, B);
                or_emit_child(C, OR_POSITRON, &po, t_rem, E, B);
            }
            if (r2 < pp) {
                /* The photon's event: it converts and is removed. */
                double ke[3], kp[3];
                for (int c = 0; c < 3; ++c) { ke[c] = r1 * q->p[c]; kp[c] = (1.0 - r1) * q->p[c]; }
                q->alive = 0;
                C->D->pairs++;
                C->D->energy_defect += q->w * (eps
                    - sqrt(1.0 + ke[0] * ke[0] + ke[1] * ke[1] + ke[2] * ke[2])
                    - sqrt(1.0 + kp[0] * kp[0] + kp[1] * kp[1] + kp[2] * kp[2]));
                break;
            }
        }
    }
    if (P->deposit_on && C->J && sp != OR_PHOTON) {
        /* deposit from the start (or birth) position to the final position */
        or_deposit(P->n, P->d, P->x0, C->J, xs, q->x, P->charge[sp] * q->w, C->dt);
    }
    if (q->alive) or_boundary(C, q);
}

/* Advance every particle that is alive at the start of the step by dt.
 * Fields are taken once per particle at its start position and time t
 * (Sec. IV.H: no re-interpolation within the step).  Products are appended
 * to their species stores.  Dead particles are removed at the end, keeping
 * the order of the survivors. */
int or_step(const or_params *P, or_store S[4], or_diag *D, double *const f[6], double *J[3],
            uint32_t step, double t, double dt)
{
    or_ctx C = {P, S, D, f, J, step, t, dt};
    int64_t n0[4];
    for (int sp = 0; sp < OR_NSPECIES; ++sp) n0[sp] = S[sp].n;
    /* keep a liveness mask per species for the initial particles */
    char *alive[4];
    for (int sp = 0; sp < OR_NSPECIES; ++sp) {
        alive[sp] = (char *)malloc((size_t)(S[sp].cap > 0 ? S[sp].cap : 1));
        if (!alive[sp]) return -1;
        memset(alive[sp], 1, (size_t)(S[sp].cap > 0 ? S[sp].cap : 1));
    }
    for (int sp = 0; sp < OR_NSPECIES; ++sp) {
        or_store *s = &S[sp];
        for (int64_t i = 0; i < n0[sp]; ++i) {
            or_particle q;
            q.x[0] = s->x[i]; q.x[1] = s->y[i]; q.x[2] = s->z[i];
            q.p[0] = s->px[i]; q.p[1] = s->py[i]; q.p[2] = s->pz[i];
            q.w = s->w[i]; q.id = s->id[i]; q.alive = 1;
            double E[3], B[3];
            if (P->field_mode == OR_FIELD_GRID)
                or_gather(P->n, P->d, P->x0, f, q.x, E, B);
            else if (P->field_mode == OR_FIELD_ENSEMBLE)
                or_field_ensemble(P, q.id, t, E, B);
            else
                or_field(P->field_mode, P->fp, q.x, t, E, B);
            int finite = 1;
            for (int c = 0; c < 3; ++c) finite &= isfinite(E[c]) && isfinite(B[c]) && isfinite(q.p[c]);
            if (!finite) D->nonfinite++;
            or_process(&C, sp, &q, dt, E, B, 0);
            s->x[i] = q.x[0]; s->y[i] = q.x[1]; s->z[i] = q.x[2];
            s->px[i] = q.p[0]; s->py[i] = q.p[1]; s->pz[i] = q.p[2];
            alive[sp][i] = (char)q.alive;
        }
    }
    for (int sp = 0; sp < OR_NSPECIES; ++sp) {
        or_store *s = &S[sp];
        int64_t o = 0;
        for (int64_t i = 0; i < s->n; ++i) {
            if (i < n0[sp] && !alive[sp][i]) continue;
            s->x[o] = s->x[i]; s->y[o] = s->y[i]; s->z[o] = s->z[i];
            s->px[o] = s->px[i]; s->py[o] = s->py[i]; s->pz[o] = s->pz[i];
            s->w[o] = s->w[i]; s->id[o] = s->id[i];
            ++o;
        }
        s->n = o;
        free(alive[sp]);
    }
    return 0;
}

/* Pairs from the vacuum (Sec. V.B): once per step, in every cell of the
 * lattice, the field E is taken at the cell centre (the Yee mesh's CIC
 * gather there, or the analytic field at the step's start time t) and
 *   P_S = R_S V_cell c dt,   R_S = E^2 exp(-pi E_S/E) / (4 pi^3 lambda_C^4),
 * which in Compton units (lambda_C = c = 1, E in E_S) is
 *   P_S = E^2 exp(-pi/E) d0 d1 d2 dt / (4 pi^3).
 * The magnetic field is neglected, as in the paper's statement.  If
 * r < P_S an electron and a positron at rest are placed at one uniformly
 * drawn point of the cell.  Draws: the cell index keys a Philox stream,
 * counter (step, 0 or 1, SCHWINGER, seed): r, u_x from the first block, u_y,
 * u_z from the second.  Ids: or_child_id of the cell index with the kind
 * flagged OR_SCHWINGER_KIND.  Cells with P_S > 1 are counted. */
int or_schwinger(const or_params *P, or_store S[4], or_diag *D, double *const f[6], uint32_t step, double t,
                 double dt)
{
    const double vol = P->d[0] * P->d[1] * P->d[2];
    for (long k = 0; k < P->n[2]; ++k)
        for (long j = 0; j < P->n[1]; ++j)
            for (long i = 0; i < P->n[0]; ++i) {
                uint64_t cell = (uint64_t)((k * P->n[1] + j) * P->n[0] + i);
                double xc[3] = {P->x0[0] + (i + 0.5) * P->d[0], P->x0[1] + (j + 0.5) * P->d[1],
                                P->x0[2] + (k + 0.5) * P->d[2]};
                double E[3], B[3];
                if (P->field_mode == OR_FIELD_GRID)
                    or_gather(P->n, P->d, P->x0, f, xc, E, B);
                else
                    or_field(P->field_mode, P->fp, xc, t, E, B);
                double Em = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
                if (!(Em > 0.0)) continue;
                double ps = Em * Em * exp(-OR_PI / Em) / (4.0 * OR_PI * OR_PI * OR_PI) * vol * dt;
                if (ps > 1.0) D->schwinger_gt1++;
                double r, ux, uy, uz;
                or_draw(cell, step, 0u, OR_PURPOSE_SCHWINGER, P->seed, &r, &ux);
                if (!(r < ps)) continue;
                or_draw(cell, step, 1u, OR_PURPOSE_SCHWINGER, P->seed, &uy, &uz);
                or_particle el, po;
                el.x[0] = po.x[0] = P->x0[0] + ((double)i + ux) * P->d[0];
                el.x[1] = po.x[1] = P->x0[1] + ((double)j + uy) * P->d[1];
                el.x[2] = po.x[2] = P->x0[2] + ((double)k + uz) * P->d[2];
                for (int c = 0; c < 3; ++c) el.p[c] = po.p[c] = 0.0;
                el.w = po.w = P->schwinger_weight;
                el.id = or_child_id(cell, step, 0u, OR_ELECTRON | OR_SCHWINGER_KIND, P->seed);
                po.id = or_child_id(cell, step, 0u, OR_POSITRON | OR_SCHWINGER_KIND, P->seed);
                el.alive = po.alive = 1;
                or_ctx C = {P, S, D, f, NULL, step, t, dt};
                or_append(&C, OR_ELECTRON, &el);
                or_append(&C, OR_POSITRON, &po);
                D->schwinger_pairs++;
            }
    return 0;
}

/* Limit of species sp in group g: thin_limit[sp], scaled by the ensemble's
 * thin_scale when that is positive (floor of the product). */
static int64_t or_thin_limit(const or_params *P, int sp, uint32_t g)
{
    int64_t L = P->thin_limit[sp];
    if (P->field_mode == OR_FIELD_ENSEMBLE && P->ens_bits > 0 && P->ens && (int64_t)g < (int64_t)P->n_ens) {
        double sc = P->ens[(size_t)OR_ENS_STRIDE * g + 9];
        if (sc > 0.0) L = (int64_t)floor((double)L * sc);
    }
    return L;
}

/* Thinning with global even redistribution (Sec. VI), after step `step`.
 * A group is one ensemble (or the whole species without ensembles).  For
 * each species with a limit L and each group holding N > L particles, every
 * particle survives with probability L/N (its own uniform, purpose THIN),
 * and the survivors' weights are multiplied by (sum of the group's weights)
 * / (sum of the survivors' weights), so the group's total weight is kept.
 * The limit L of a group is thin_limit[sp], times the ensemble's thin_scale
 * when that is positive (an independent instance keeps its own budget).
 * A group in which nothing would survive is left as it is.  Particles whose
 * ensemble has no table row belong to no group.  Survivors keep their order. */
int or_thin(const or_params *P, or_store S[4], or_diag *D, uint32_t step)
{
    /* groups are ensembles only in the ensemble field mode; elsewhere the
     * id bits only record a product's lineage and a species is one group */
    const int by_ens = P->field_mode == OR_FIELD_ENSEMBLE && P->ens_bits > 0;
    int64_t G = by_ens ? (int64_t)P->n_ens : 1;
    if (G <= 0) return 0;
    int64_t *count = (int64_t *)malloc(sizeof(int64_t) * (size_t)G);
    double *wall = (double *)malloc(sizeof(double) * (size_t)G);
    double *wsurv = (double *)malloc(sizeof(double) * (size_t)G);
    if (!count || !wall || !wsurv) { free(count); free(wall); free(wsurv); return -1; }
    for (int sp = 0; sp < OR_NSPECIES; ++sp) {
        if (P->thin_limit[sp] <= 0) continue;
        or_store *s = &S[sp];
        for (int64_t g = 0; g < G; ++g) { count[g] = 0; wall[g] = 0.0; wsurv[g] = 0.0; }
        for (int64_t i = 0; i < s->n; ++i) {
            uint32_t g = by_ens ? or_ensemble(P, s->id[i]) : 0;
            if ((int64_t)g >= G) continue;
            count[g]++;
            wall[g] += s->w[i];
        }
        /* the survivors of a group, and their weight */
        for (int64_t i = 0; i < s->n; ++i) {
            uint32_t g = by_ens ? or_ensemble(P, s->id[i]) : 0;
            if ((int64_t)g >= G) continue;
            int64_t L = or_thin_limit(P, sp, g);
            if (count[g] <= L) continue;
            double u, unused;
            or_draw(s->id[i], step, 0u, OR_PURPOSE_THIN, P->seed, &u, &unused);
            if (u < (double)L / (double)count[g]) wsurv[g] += s->w[i];
        }
        int64_t o = 0;
        for (int64_t i = 0; i < s->n; ++i) {
            uint32_t g = by_ens ? or_ensemble(P, s->id[i]) : 0;
            int keep = 1;
            double w = s->w[i];
            int64_t L = (int64_t)g < G ? or_thin_limit(P, sp, g) : 0;
            if ((int64_t)g < G && count[g] > L && wsurv[g] > 0.0) {
                double u, unused;
                or_draw(s->id[i], step, 0u, OR_PURPOSE_THIN, P->seed, &u, &unused);
                if (u < (double)L / (double)count[g]) w = w * (wall[g] / wsurv[g]);
                else keep = 0;
            }
            if (!keep) { D->thinned++; continue; }
            s->x[o] = s->x[i]; s->y[o] = s->y[i]; s->z[o] = s->z[i];
            s->px[o] = s->px[i]; s->py[o] = s->py[i]; s->pz[o] = s->pz[i];
            s->w[o] = w; s->id[o] = s->id[i];
            ++o;
        }
        s->n = o;
    }
    free(count); free(wall); free(wsurv);
    return 0;
}

/* Frozen-particle sampling of the modified generator (the spectrum test of
 * Sec. IV.G): ndraw independent trials with fixed gamma and chi and no
 * recoil; trial i uses the stream of id = i at step 0, sub-step 0.
 * Accepted delta are histogrammed in log10(delta) over [lo, hi). */
int64_t or_sample_frozen(double chi, double gamma, double h, int64_t ndraw, uint32_t seed,
                         double lo, double hi, int32_t nbins, double *hist, int64_t *pm_gt1)
{
    int64_t acc = 0, viol = 0;
    for (int64_t i = 0; i < ndraw; ++i) {
        double r1, r2;
        or_draw((uint64_t)i, 0u, 0u, OR_PURPOSE_EMIT, seed, &r1, &r2);
        double pm = or_Pm(r1, chi, gamma, h);
        if (pm > 1.0) ++viol;
        if (r2 < pm) {
            ++acc;
            double delta = r1 * r1 * r1;
            double a = (log10(delta) - lo) / (hi - lo) * nbins;
            if (a >= 0.0 && a < nbins) hist[(long)a] += 1.0;
        }
    }
    if (pm_gt1) *pm_gt1 = viol;
    return acc;
}

/* The same frozen-particle test for any of the three generators of
 * Sec. IV.F-G (the paper's Fig. "generators"): modified (P_m, delta =
 * r1^3), alternative (P(r1), delta = r1) or standard (W(1), delta from
 * W(delta)/W(1) = r2).  P > 1 draws are counted in *p_gt1. */
int64_t or_sample_frozen_gen(int32_t generator, double chi, double gamma, double h, int64_t ndraw,
                             uint32_t seed, double lo, double hi, int32_t nbins, double *hist,
                             int64_t *p_gt1)
{
    int64_t acc = 0, viol = 0;
    double pstd = generator == OR_GEN_STANDARD ? or_Pstd(chi, gamma, h) : 0.0;
    for (int64_t i = 0; i < ndraw; ++i) {
        double r1, r2, delta = 0.0, pe;
        int fire;
        or_draw((uint64_t)i, 0u, 0u, OR_PURPOSE_EMIT, seed, &r1, &r2);
        if (generator == OR_GEN_ALTERNATIVE) {
            pe = or_P(r1, chi, gamma, h);
            fire = r2 < pe;
            delta = r1;
        } else if (generator == OR_GEN_STANDARD) {
            pe = pstd;
            fire = r1 < pe;
            if (fire) delta = or_delta_std(chi, r2);
        } else {
            pe = or_Pm(r1, chi, gamma, h);
            fire = r2 < pe;
            delta = r1 * r1 * r1;
        }
        if (pe > 1.0) ++viol;
        if (fire) {
            ++acc;
            double a = (log10(delta) - lo) / (hi - lo) * nbins;
            if (a >= 0.0 && a < nbins) hist[(long)a] += 1.0;
        }
    }
    if (p_gt1) *p_gt1 = viol;
    return acc;
}

/* Draw a block of raw Philox outputs (cross-implementation checks). */
void or_philox_block(uint64_t id, uint32_t step, uint32_t sub0, uint32_t purpose, uint32_t seed,
                     int64_t n, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {step, sub0 + (uint32_t)i, purpose, seed};
        uint32_t key[2] = {(uint32_t)id, (uint32_t)(id >> 32)};
        or_philox4x32_10(ctr, key, out + 4 * i);
    }
}
