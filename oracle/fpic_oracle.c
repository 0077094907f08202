/*
 * FPIC oracle: plain, serial, FP64 CPU restatement of the GRPIC particle
 * path of "FPIC: a new Particle-In-Cell code for stationary and
 * axisymmetric black-hole spacetimes" (Meringolo & Rezzolla, arXiv
 * 2602.07452).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library.  Compiled with -O2 -ffp-contract=off so that every
 * multiply and add rounds separately.
 *
 * Every function names the passage of the paper it restates.  Where the
 * paper is silent, garbled or inconsistent the reading taken is stated at
 * the function ("Reading: ...").
 *
 * Units: geometrised, G = c = 1.  The black-hole mass M and spin a (a
 * length, |a| <= M) are parameters.
 * Particle state z = (r, th, ph, u_r, u_th, u_ph): contravariant position,
 * covariant momentum per unit mass (Sec. 2.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Appendix A: Kerr metric in spherical Kerr-Schild coordinates, 3+1 split. */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s, c;                      /* sin th, cos th */
    double rho2;                      /* rho^2 = r^2 + a^2 cos^2 th */
    double xi;                        /* xi = 1 + 2 M r / rho^2 */
    double alpha;                     /* lapse = xi^{-1/2} */
    double beta;                      /* shift beta^r = (xi - 1)/xi */
    double g_rr, g_rp, g_tt, g_pp;    /* gamma_ij */
    double gu_rr, gu_rp, gu_tt, gu_pp;/* gamma^ij */
    double sqrtg;                     /* sqrt(gamma) = rho^2 sqrt(xi) sin th */
} om_t;

/* Appendix A, Eqs. (gsf), (gsf_2), lapse/shift and (det).
 * Reading: the printed gamma_{r phi} = -a^2 xi sin^2 th is a misprint; the
 * inverse of the printed gamma^{ij} requires gamma_{r phi} = -a xi sin^2 th,
 * which is what is used (and what the inverse-relation test pins). */
static void om_eval(double M, double a, double r, double th, om_t *m)
{
    double s = sin(th), c = cos(th);
    double s2 = s * s, c2 = c * c;
    m->s = s;
    m->c = c;
    m->rho2 = r * r + a * a * c2;
    m->xi = 1.0 + 2.0 * M * r / m->rho2;
    m->alpha = 1.0 / sqrt(m->xi);
    m->beta = (m->xi - 1.0) / m->xi;
    m->g_rr = m->xi;
    m->g_rp = -a * m->xi * s2;
    m->g_tt = m->rho2;
    m->g_pp = s2 * (m->rho2 + a * a * m->xi * s2);
    m->gu_rr = a * a * s2 / m->rho2 + 1.0 / m->xi;
    m->gu_rp = a / m->rho2;
    m->gu_tt = 1.0 / m->rho2;
    m->gu_pp = 1.0 / (m->rho2 * s2);
    m->sqrtg = m->rho2 * sqrt(m->xi) * s;
}

/* Radial and polar derivatives of alpha, beta^r and gamma^{ij}, taken
 * analytically at the particle as Sec. 2.2 prescribes ("both the metric
 * components ... and their derivatives are computed analytically at the
 * position of the particle").  Derived by hand from Appendix A:
 *   d rho^2/dr = 2r,  d rho^2/dth = -2 a^2 s c
 *   d xi = 2M d(r/rho^2)
 *   d alpha = -alpha^3 d xi / 2,  d beta = d xi / xi^2.
 * Layout of d[0..11]: (dr, dth) of alpha, beta, g^rr, g^rp, g^tt, g^pp. */
static void om_deriv(double M, double a, double r, double th, double d[12])
{
    om_t m;
    om_eval(M, a, r, th, &m);
    double s = m.s, c = m.c, s2 = s * s;
    double P = m.rho2, P2 = P * P;
    double dPr = 2.0 * r, dPt = -2.0 * a * a * s * c;
    double dxir = 2.0 * M * (P - r * dPr) / P2;
    double dxit = -2.0 * M * r * dPt / P2;
    double a3 = m.alpha * m.alpha * m.alpha;
    double xi2 = m.xi * m.xi;
    d[0] = -0.5 * a3 * dxir;
    d[1] = -0.5 * a3 * dxit;
    d[2] = dxir / xi2;
    d[3] = dxit / xi2;
    /* g^rr = a^2 s^2 / P + 1/xi */
    d[4] = -a * a * s2 * dPr / P2 - dxir / xi2;
    d[5] = a * a * 2.0 * s * c / P - a * a * s2 * dPt / P2 - dxit / xi2;
    /* g^rp = a / P */
    d[6] = -a * dPr / P2;
    d[7] = -a * dPt / P2;
    /* g^tt = 1 / P */
    d[8] = -dPr / P2;
    d[9] = -dPt / P2;
    /* g^pp = 1 / (P s^2) */
    d[10] = -dPr / (P2 * s2);
    d[11] = -(dPt * s2 + P * 2.0 * s * c) / (P2 * s2 * s2);
}

/* ------------------------------------------------------------------------ */
/* Appendix B.1 and Sec. 3.1.3: the Wald electro-vacuum field (M = 1 units, */
/* as printed).                                                             */
/* ------------------------------------------------------------------------ */

/* A_0 and A_phi as printed in Sec. 3.1.3 (the H and L definitions).
 * Reading: the printed A_phi lacks the overall factor B0 that Eq. (Amu)
 * gives it; the factor is restored.  A_0 is used exactly as printed (no
 * -a B0 gauge constant), so H is defined up to that constant. */
static double wald_A0(double a, double B0, double r, double th)
{
    double c = cos(th);
    double rho2 = r * r + a * a * c * c;
    return B0 * a * r * (1.0 + c * c) / rho2;
}

static double wald_Aph(double a, double B0, double r, double th)
{
    double s = sin(th), c = cos(th);
    double rho2 = r * r + a * a * c * c;
    return 0.5 * B0 * s * s * (r * r + a * a - 2.0 * a * a * r * (1.0 + c * c) / rho2);
}

/* A_r of Eq. (Amu): (B0/2)(g_rph + 2 a g_0r) = (B0/2)(2 a r (1 + c^2)/rho^2 - a s^2)
 * (M = 1).  Sec. 3.1.3's H and L need only A_0 and A_ph; the canonical
 * momentum pi_r = u_r + (q/m) A_r of the discrete-gradient scheme for
 * charged particles needs it too. */
static double wald_Ar(double a, double B0, double r, double th)
{
    double s = sin(th), c = cos(th);
    double rho2 = r * r + a * a * c * c;
    return 0.5 * B0 * (2.0 * a * r * (1.0 + c * c) / rho2 - a * s * s);
}

/* Appendix B.1, Eqs. (wald1)-(wald6): contravariant B^i and covariant E_i.
 * Reading: the printed E_theta carries an extra factor a; the value used,
 * E_theta = 2 B0 a r (a^2 - r^2) sin th cos th / rho^4, is the one that
 * equals dA_0/dth for the printed A_0 (pinned by finite differences of
 * A_0).  Sign convention E_i = F_{i0} = +d_i A_0 (Eq. Ei); Eq. (wald1_0)'s
 * minus sign is taken as a typo because App. B's E_r carries the + sign. */
static void wald_BE(double a, double B0, double r, double th,
                    double B[3], double E[3])
{
    double s = sin(th), c = cos(th);
    double rho2 = r * r + a * a * c * c, rho4 = rho2 * rho2;
    double xi = 1.0 + 2.0 * r / rho2;
    double sqrtg = rho2 * sqrt(xi) * s;
    double a2 = a * a;
    B[0] = B0 / sqrtg * (r * r + a2 - 2.0 * r + 2.0 * r * (r * r * r * r - a2 * a2) / rho4) * s * c;
    B[1] = -B0 / sqrtg * (r + a2 * (1.0 + c * c) * (2.0 * r * r - rho2) / rho4) * s * s;
    B[2] = -B0 / sqrtg * (2.0 * a * r * (a2 - r * r) / rho4 - a) * s * c;
    E[0] = B0 * a * (1.0 + c * c) * (a2 * c * c - r * r) / rho4;
    E[1] = B0 * 2.0 * a * r * (a2 - r * r) / rho4 * s * c;
    E[2] = 0.0;
}

/* FIDO electric field D^i from E_i and B^i via Eq. (Ei):
 * E_i = alpha D_i + sqrt(gamma) eta_ijk beta^j B^k with beta = (beta^r,0,0),
 * i.e. D_r = E_r/alpha, D_th = (E_th + sqrtg beta B^ph)/alpha,
 * D_ph = (E_ph - sqrtg beta B^th)/alpha;  D^i = gamma^ij D_j. */
static void wald_D(double a, double B0, double r, double th, double D[3], double B[3])
{
    double E[3];
    om_t m;
    wald_BE(a, B0, r, th, B, E);
    om_eval(1.0, a, r, th, &m);
    double Dr_ = E[0] / m.alpha;
    double Dt_ = (E[1] + m.sqrtg * m.beta * B[2]) / m.alpha;
    double Dp_ = (E[2] - m.sqrtg * m.beta * B[1]) / m.alpha;
    D[0] = m.gu_rr * Dr_ + m.gu_rp * Dp_;
    D[1] = m.gu_tt * Dt_;
    D[2] = m.gu_rp * Dr_ + m.gu_pp * Dp_;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: Hamiltonian and equations of motion.                           */
/* ------------------------------------------------------------------------ */

/* Eq. (Ham) with the static potential of Sec. 3.1.3:
 * H = alpha Gamma - beta^r u_r - (q/m) A_0,  Gamma = sqrt(1 + g^ij u_i u_j). */
static double gamma_lorentz(const om_t *m, const double *u)
{
    double q = m->gu_rr * u[0] * u[0] + 2.0 * m->gu_rp * u[0] * u[2]
             + m->gu_tt * u[1] * u[1] + m->gu_pp * u[2] * u[2];
    return sqrt(1.0 + q);
}

typedef struct {
    double M, a;
    double B0pot;    /* B0 of the Wald potential entering H and L; 0 = none */
} or_bh;

static double ham(const or_bh *bh, double qm, const double *z)
{
    om_t m;
    om_eval(bh->M, bh->a, z[0], z[1], &m);
    double G = gamma_lorentz(&m, z + 3);
    double h = m.alpha * G - m.beta * z[3];
    if (bh->B0pot != 0.0 && qm != 0.0)
        h -= qm * wald_A0(bh->a, bh->B0pot, z[0], z[1]);
    return h;
}

/* Normaliser of the relative energy error.  Reading: the paper divides by
 * H_0 (Sec. 3.1.2), which for charged particles can be ~0 or negative; the
 * denominator used is |alpha Gamma - beta u_r|_0 + |(q/m) A_0|_0, equal to
 * |H_0| for neutral particles. */
static double ham_norm(const or_bh *bh, double qm, const double *z)
{
    om_t m;
    om_eval(bh->M, bh->a, z[0], z[1], &m);
    double G = gamma_lorentz(&m, z + 3);
    double d = fabs(m.alpha * G - m.beta * z[3]);
    if (bh->B0pot != 0.0 && qm != 0.0)
        d += fabs(qm * wald_A0(bh->a, bh->B0pot, z[0], z[1]));
    return d;
}

/* Conserved angular momentum of Sec. 3.1.3: L = u_ph + (q/m) A_ph. */
static double angmom(const or_bh *bh, double qm, const double *z)
{
    double l = z[5];
    if (bh->B0pot != 0.0 && qm != 0.0)
        l += qm * wald_Aph(bh->a, bh->B0pot, z[0], z[1]);
    return l;
}

/* Eqs. (p1), (p2), (O1), (O2): dz/dt at z given FIDO fields D^i, B^i at the
 * particle.  eta_{r th ph} = +1.  A^(g)_ph = 0 because d_ph = 0. */
static void rhs(double M, double a, double qm, const double *z,
                const double *D, const double *B, double *f)
{
    om_t m;
    double d[12];
    om_eval(M, a, z[0], z[1], &m);
    om_deriv(M, a, z[0], z[1], d);
    double ur = z[3], ut = z[4], up = z[5];
    double Ur = m.gu_rr * ur + m.gu_rp * up;   /* u^r */
    double Ut = m.gu_tt * ut;                  /* u^th */
    double Up = m.gu_rp * ur + m.gu_pp * up;   /* u^ph */
    double G = sqrt(1.0 + ur * Ur + ut * Ut + up * Up);
    f[0] = m.alpha * Ur / G - m.beta;
    f[1] = m.alpha * Ut / G;
    f[2] = m.alpha * Up / G;
    for (int i = 0; i < 2; ++i) {
        double dal = d[0 + i], dbe = d[2 + i];
        double dgrr = d[4 + i], dgrp = d[6 + i], dgtt = d[8 + i], dgpp = d[10 + i];
        double quad = ur * ur * dgrr + 2.0 * ur * up * dgrp + ut * ut * dgtt + up * up * dgpp;
        f[3 + i] = -G * dal + ur * dbe - m.alpha / (2.0 * G) * quad;
    }
    f[5] = 0.0;
    if (qm != 0.0 && D && B) {
        double k = qm * m.alpha;
        double cr = Ut * B[2] - Up * B[1];
        double ct = Up * B[0] - Ur * B[2];
        double cp = Ur * B[1] - Ut * B[0];
        f[3] += k * (m.g_rr * D[0] + m.g_rp * D[2] + m.sqrtg * cr / G);
        f[4] += k * (m.g_tt * D[1] + m.sqrtg * ct / G);
        f[5] += k * (m.g_rp * D[0] + m.g_pp * D[2] + m.sqrtg * cp / G);
    }
}

/* ------------------------------------------------------------------------ */
/* Grid, cell location and field gather.                                    */
/* ------------------------------------------------------------------------ */

/* Yee layout (Sec. 2.1, Fig. 1 caption and the B^r / B^ph example):
 *   D^r (i+1/2, j)   D^th (i, j+1/2)   D^ph (i, j)
 *   B^r (i, j+1/2)   B^th (i+1/2, j)   B^ph (i+1/2, j+1/2)
 * A component array is indexed [i*ld + j]; i counts r nodes (integer or
 * half), j counts th nodes.  ld >= Nth + 1. */
typedef struct {
    int Nr, Nth, ld;
    const double *rn;   /* r_i,        i = 0..Nr   */
    const double *rh;   /* r_{i+1/2},  i = 0..Nr-1 */
    const double *tn;   /* th_j,       j = 0..Nth  */
    const double *th;   /* th_{j+1/2}, j = 0..Nth-1 */
    int full;           /* full-theta domain: th periodic with period tn[Nth] - tn[0] */
} or_grid;

static const int yee_roff[6] = {1, 0, 0, 0, 1, 1};
static const int yee_toff[6] = {0, 1, 0, 1, 0, 1};

/* Cell location against a node list X[0..m-1], m >= 2 (Sec. 2.3: a particle
 * "located between nodes r_ir <= r <= r_ir+1").  Reading: the lower bound is
 * inclusive, the upper exclusive (a point on a node belongs to the upper
 * cell); outside the list the first/last cell is taken. */
static int locate(const double *X, int m, double x)
{
    if (!(x >= X[0])) return 0;
    if (x >= X[m - 1]) return m - 2;
    int lo = 0, hi = m - 1;          /* X[lo] <= x < X[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x >= X[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

/* Linear weight of x in [X[i], X[i+1]], clamped to [0,1] (constant
 * extrapolation beyond the end nodes). */
static double lin_w(const double *X, int i, double x)
{
    double w = (x - X[i]) / (X[i + 1] - X[i]);
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    return w;
}

/* th reduced to one period [tn[0], tn[0] + P) of the full-theta domain
 * (Sec. 2.5: periodic boundaries at th_max = 2 pi + eps). */
static double wrap_theta(const or_grid *g, double t)
{
    const double t0 = g->tn[0], P = g->tn[g->Nth] - g->tn[0];
    while (t < t0) t += P;
    while (t >= t0 + P) t -= P;
    return t;
}

/* Field gather (grid -> particle).  Reading: the paper does not state its
 * gather; each component is interpolated bilinearly in (r, th) on its own
 * staggered sub-grid.  Full-theta domain: th is taken modulo the period;
 * column Nth of every array is the image of column 0, so the node sub-grid
 * interpolates between tn[Nth-1] and tn[Nth] as usual, and the half-node
 * sub-grid's nodes are extended by th[Nth] = th[0] + P: a point below th[0]
 * is taken at th + P, in the cell [th[Nth-1], th[Nth]]. */
static void gather(const or_grid *g, const double *const F[6], double r, double t,
                   double D[3], double B[3])
{
    double v[6], th_ext[2] = {0.0, 0.0};
    if (g->full) t = wrap_theta(g, t);
    for (int k = 0; k < 6; ++k) {
        const double *X = yee_roff[k] ? g->rh : g->rn;
        const double *Y = yee_toff[k] ? g->th : g->tn;
        int mx = yee_roff[k] ? g->Nr : g->Nr + 1;
        int my = yee_toff[k] ? g->Nth : g->Nth + 1;
        int i = locate(X, mx, r), j;
        double wr = lin_w(X, i, r), wt;
        if (g->full && yee_toff[k]) {
            const double P = g->tn[g->Nth] - g->tn[0];
            const double th_top = g->th[0] + P;
            const double tt = t < g->th[0] ? t + P : t;
            if (tt >= g->th[g->Nth - 1]) {
                j = g->Nth - 1;
                th_ext[0] = g->th[g->Nth - 1];
                th_ext[1] = th_top;
                wt = lin_w(th_ext, 0, tt);
            } else {
                j = locate(Y, my, tt);
                wt = lin_w(Y, j, tt);
            }
        } else {
            j = locate(Y, my, t);
            wt = lin_w(Y, j, t);
        }
        const double *f = F[k];
        v[k] = (1.0 - wr) * (1.0 - wt) * f[i * g->ld + j]
             + wr * (1.0 - wt) * f[(i + 1) * g->ld + j]
             + (1.0 - wr) * wt * f[i * g->ld + j + 1]
             + wr * wt * f[(i + 1) * g->ld + j + 1];
    }
    D[0] = v[0]; D[1] = v[1]; D[2] = v[2];
    B[0] = v[3]; B[1] = v[4]; B[2] = v[5];
}

/* ------------------------------------------------------------------------ */
/* Pushers (Sec. 2.2.1-2.2.3) and the hybrid switch (Sec. 3.1.2).           */
/* ------------------------------------------------------------------------ */

enum { OR_FIELD_NONE = 0, OR_FIELD_GRID = 1, OR_FIELD_WALD = 2 };
enum { OR_RK4 = 0, OR_IMR = 1, OR_HAM = 2, OR_HYB1 = 3, OR_HYB2 = 4 };

typedef struct {
    double M, a;
    double B0pot;          /* Wald B0 entering H and L (0: no potential) */
    int field_kind;        /* OR_FIELD_* */
    double B0field;        /* analytic Wald field strength (OR_FIELD_WALD) */
    double dt;
    int scheme;            /* OR_RK4 .. OR_HYB2 */
    int implicit_kind;     /* OR_IMR or OR_HAM: partner of the hybrid */
    double thr;            /* Hyb2: Htilde_max;  Hyb1: (d Htilde/dt)_max */
    double tol;            /* implicit convergence tolerance */
    int max_iter;          /* implicit iteration cap */
    double r_h, r_max;     /* particle removal radii */
    double dg_eps;         /* discrete-gradient increment threshold */
    double dt_imp;         /* step of the implicit partner of a hybrid (0: dt) */
    int imr_newton;        /* IMR solver: 0 the fixed-point map of Eq. (imr2), 1 Newton */
    int imr_substeps;      /* an unconverged IMR solve is redone in up to 2^this substeps (0: never) */
    double substep_tol;    /* |H(end) - H(z^n)| / D_0 a substepped step must meet (0: none) */
    int theta_full;        /* full-theta domain: th periodic on [theta_lo, theta_lo + theta_period) */
    double theta_lo, theta_period;   /* tn[0] and tn[Nth] - tn[0] of the grid (period 2 pi) */
} or_push_params;

typedef struct {
    const or_push_params *p;
    const or_grid *g;
    const double *const *F;
    double qm;
} or_ctx;

static void field_at(const or_ctx *c, const double *z, double D[3], double B[3], int *have)
{
    *have = 0;
    if (c->qm == 0.0) return;
    if (c->p->field_kind == OR_FIELD_GRID) {
        gather(c->g, c->F, z[0], z[1], D, B);
        *have = 1;
    } else if (c->p->field_kind == OR_FIELD_WALD) {
        wald_D(c->p->a, c->p->B0field, z[0], z[1], D, B);
        *have = 1;
    }
}

static void F_eval(const or_ctx *c, const double *z, double *f)
{
    double D[3], B[3];
    int have;
    field_at(c, z, D, B, &have);
    rhs(c->p->M, c->p->a, c->qm, z, have ? D : NULL, have ? B : NULL, f);
}

/* Sec. 2.2.1: classical RK4; fields frozen over the step. */
static void step_rk4(const or_ctx *c, const double *z0, double *z1)
{
    double k1[6], k2[6], k3[6], k4[6], y[6];
    double h = c->p->dt;
    F_eval(c, z0, k1);
    for (int i = 0; i < 6; ++i) y[i] = z0[i] + 0.5 * h * k1[i];
    F_eval(c, y, k2);
    for (int i = 0; i < 6; ++i) y[i] = z0[i] + 0.5 * h * k2[i];
    F_eval(c, y, k3);
    for (int i = 0; i < 6; ++i) y[i] = z0[i] + h * k3[i];
    F_eval(c, y, k4);
    for (int i = 0; i < 6; ++i)
        z1[i] = z0[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Convergence test of the implicit iterations.  Reading: the paper iterates
 * "to machine round-off"; the stop is max_i |dz_i| / (|z_i| + 1) <= tol. */
static int converged(const double *a, const double *b, double tol)
{
    for (int i = 0; i < 6; ++i)
        if (!(fabs(a[i] - b[i]) <= tol * (fabs(a[i]) + 1.0))) return 0;
    return 1;
}

/* Momentum derivatives of the right-hand side at z (Eqs. p1, p2), the
 * blocks kept in the Newton matrix of the IMR solve:
 *   A_il = d(dx^i/dt)/du_l = alpha (g^il / Gamma - u^i u^l / Gamma^3),
 *   J_il = d(du_i/dt)/du_l of the magnetic force qm alpha sqrt(gamma) (u x B)_i / Gamma
 *        = qm alpha sqrt(gamma) ((g^{.l} x B)_i / Gamma - (u x B)_i u^l / Gamma^3),
 * with u^i = g^ij u_j and g^{.l} the l-th column of g^ij (d u^i / du_l).
 * The gravitational part of du/dt depends on u only through Gamma and is
 * left out of J, as are all position derivatives. */
static void cross3(const double *x, const double *y, double *o)
{
    o[0] = x[1] * y[2] - x[2] * y[1];
    o[1] = x[2] * y[0] - x[0] * y[2];
    o[2] = x[0] * y[1] - x[1] * y[0];
}

static void imr_blocks_at(double M, double a, double qm, const double *z, const double *B,
                          double A[3][3], double J[3][3])
{
    om_t m;
    om_eval(M, a, z[0], z[1], &m);
    const double gi[3][3] = {{m.gu_rr, 0.0, m.gu_rp}, {0.0, m.gu_tt, 0.0}, {m.gu_rp, 0.0, m.gu_pp}};
    double U[3];
    for (int i = 0; i < 3; ++i) U[i] = gi[i][0] * z[3] + gi[i][1] * z[4] + gi[i][2] * z[5];
    const double G = sqrt(1.0 + U[0] * z[3] + U[1] * z[4] + U[2] * z[5]);
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) {
            A[i][l] = m.alpha * (gi[i][l] / G - U[i] * U[l] / (G * G * G));
            J[i][l] = 0.0;
        }
    if (!B || qm == 0.0) return;
    const double k = qm * m.alpha * m.sqrtg;
    double cr[3];
    cross3(U, B, cr);
    for (int l = 0; l < 3; ++l) {
        const double col[3] = {gi[0][l], gi[1][l], gi[2][l]};
        double x[3];
        cross3(col, B, x);
        for (int i = 0; i < 3; ++i) J[i][l] = k * (x[i] / G - cr[i] * U[l] / (G * G * G));
    }
}

static void imr_blocks(const or_ctx *c, const double *z, double A[3][3], double J[3][3])
{
    double D[3], B[3];
    int have;
    field_at(c, z, D, B, &have);
    imr_blocks_at(c->p->M, c->p->a, c->qm, z, have ? B : NULL, A, J);
}

/* Solve the 3 x 3 system M x = b by Gaussian elimination with partial
 * pivoting (M is overwritten). */
static void solve3(double M[3][3], double b[3], double x[3])
{
    for (int k = 0; k < 3; ++k) {
        int piv = k;
        for (int i = k + 1; i < 3; ++i)
            if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
        if (piv != k) {
            for (int j = 0; j < 3; ++j) { double t = M[k][j]; M[k][j] = M[piv][j]; M[piv][j] = t; }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < 3; ++i) {
            const double f = M[i][k] / M[k][k];
            for (int j = k; j < 3; ++j) M[i][j] -= f * M[k][j];
            b[i] -= f * b[k];
        }
    }
    for (int i = 2; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < 3; ++j) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
}

/* Sec. 2.2.2, Eqs. (imr1)-(imr2): implicit midpoint rule z1 = z^n + h F((z^n + z1)/2).
 * Reading: Eq. (imr2) prints dt/2 F(z^n + z^[k-1]); the argument is read as
 * the midpoint (Eq. imr1).  Two solvers of the same equation:
 *  - imr_newton = 0: the fixed-point update the equation shows,
 *    z^[k] = z^n + h F((z^n + z^[k-1])/2);
 *  - imr_newton = 1: the Newton iteration the text names, on the residual
 *    R(z) = z - z^n - h F((z^n + z)/2) with the Jacobian dR/dz = 1 - (h/2) dF
 *    in which dF keeps its momentum columns (imr_blocks: A for the
 *    positions, J for the momenta) and drops the position columns.  With
 *    z^p = z^n + h F(y), y = (z^n + z^[k-1])/2, the step solves
 *    (1 - (h/2) J) du = u^[k-1] - u^p, then u^[k] = u^[k-1] - du and
 *    x^[k] = x^p - (h/2) A du.  Only the convergence rate differs: both
 *    stop at the same fixed point.
 * Stop, both forms: the update passes the test of `converged` (the paper
 * iterates to round-off; the successive-update test is that reading and the
 * only stopping rule here, so both forms end on the same solution to within
 * the tolerance).
 * A solve that reaches max_iter without converging (reading: the paper
 * gives no policy) returns the iterate whose update max_i |z^[k]_i - z^[k-1]_i|
 * was the smallest, the earliest on ties: for a locally contracting map
 * that update bounds the iterate's distance to the solution.
 * Returns the iteration count, or -max_iter if the cap was reached. */
static int step_imr(const or_ctx *c, double h, const double *z0, const double *guess, double *z1)
{
    double zk[6], y[6], f[6], zn[6], best[6], best_dz = INFINITY;
    memcpy(zk, guess, sizeof zk);
    for (int k = 1; k <= c->p->max_iter; ++k) {
        for (int i = 0; i < 6; ++i) y[i] = 0.5 * (z0[i] + zk[i]);
        F_eval(c, y, f);
        for (int i = 0; i < 6; ++i) zn[i] = z0[i] + h * f[i];
        if (c->p->imr_newton) {
            double A[3][3], J[3][3], Mx[3][3], b[3], du[3];
            imr_blocks(c, y, A, J);
            for (int i = 0; i < 3; ++i) {
                for (int l = 0; l < 3; ++l) Mx[i][l] = (i == l ? 1.0 : 0.0) - 0.5 * h * J[i][l];
                b[i] = zk[3 + i] - zn[3 + i];
            }
            solve3(Mx, b, du);
            for (int i = 0; i < 3; ++i) {
                zn[3 + i] = zk[3 + i] - du[i];
                zn[i] -= 0.5 * h * (A[i][0] * du[0] + A[i][1] * du[1] + A[i][2] * du[2]);
            }
        }
        const int ok = converged(zn, zk, c->p->tol);
        double dz = 0.0;
        for (int i = 0; i < 6; ++i) dz = fmax(dz, fabs(zn[i] - zk[i]));
        if (dz < best_dz) { best_dz = dz; memcpy(best, zn, sizeof best); }
        memcpy(zk, zn, sizeof zk);
        if (ok) { memcpy(z1, zk, sizeof zk); return k; }
    }
    memcpy(z1, best, sizeof best);
    return -c->p->max_iter;
}

/* sin(h) / h, by its series below |h| = 1e-3 (error < 1e-19 there). */
static double sinc_(double h)
{
    if (fabs(h) < 1e-3) {
        double h2 = h * h;
        return 1.0 - h2 / 6.0 + h2 * h2 / 120.0;
    }
    return sin(h) / h;
}

/* The difference quotient of the geodesic Hamiltonian for a move of the
 * single variable v from zb to za (the other components equal):
 *   G = (H(za) - H(zb)) / (za_v - zb_v),
 * evaluated in closed form with the increment divided out analytically, so
 * that no difference of nearly equal H values is formed (Appendix D writes
 * its quotients in this split form: alpha' Gamma' - alpha Gamma =
 * (alpha' + alpha)/2 (Gamma' - Gamma) + (Gamma' + Gamma)/2 (alpha' - alpha),
 * Gamma' - Gamma = (Gamma'^2 - Gamma^2) / (Gamma' + Gamma)).  The metric
 * differences per unit increment:
 *   r:  d(rho^2) = r + r',  d(2 M r / rho^2) = 2 M (a^2 c^2 - r r') / (rho^2 rho'^2)
 *   th: d(c) = -sin(th_m) sinc(dth/2) (th_m the midpoint), d(c^2) = (c + c') d(c),
 *       d(rho^2) = a^2 d(c^2), d(2 M r / rho^2) = -2 M r d(rho^2) / (rho^2 rho'^2)
 * and then d(1/rho^2) = -d(rho^2) / (rho^2 rho'^2), d(xi) = d(2 M r / rho^2),
 * d(1/xi) = -d(xi) / (xi xi'), d(alpha) = -d(xi) / (sqrt(xi xi')
 * (sqrt(xi) + sqrt(xi'))), d(beta) = d(xi) / (xi xi').  In exact arithmetic
 * G is the plain quotient; it tends to the partial derivative as the
 * increment vanishes, so no switch to the partial is needed. */
static double dg_quot(double M, double a, const double *zb, const double *za, int v)
{
    if (v == 2) return 0.0;                                   /* H does not depend on ph */
    om_t mb, ma;
    om_eval(M, a, zb[0], zb[1], &mb);
    om_eval(M, a, za[0], za[1], &ma);
    const double *ub = zb + 3, *ua = za + 3;
    const double Gb = gamma_lorentz(&mb, ub), Ga = gamma_lorentz(&ma, ua);
    const double Gs = Ga + Gb;
    if (v == 3)
        return mb.alpha * (mb.gu_rr * (ua[0] + ub[0]) + 2.0 * mb.gu_rp * ub[2]) / Gs - mb.beta;
    if (v == 4)
        return mb.alpha * mb.gu_tt * (ua[1] + ub[1]) / Gs;
    if (v == 5)
        return mb.alpha * (2.0 * mb.gu_rp * ub[0] + mb.gu_pp * (ua[2] + ub[2])) / Gs;
    /* position moves: metric differences per unit increment */
    const double a2 = a * a;
    double d_rho2, d_f, d_s2;
    if (v == 0) {
        const double c2 = mb.c * mb.c;
        d_rho2 = zb[0] + za[0];
        d_f = 2.0 * M * (a2 * c2 - zb[0] * za[0]) / (mb.rho2 * ma.rho2);
        d_s2 = 0.0;
    } else {
        const double h = 0.5 * (za[1] - zb[1]);
        const double d_c = -sin(0.5 * (za[1] + zb[1])) * sinc_(h);
        const double d_c2 = (mb.c + ma.c) * d_c;
        d_rho2 = a2 * d_c2;
        d_f = -2.0 * M * zb[0] * d_rho2 / (mb.rho2 * ma.rho2);
        d_s2 = -d_c2;
    }
    const double d_irho2 = -d_rho2 / (mb.rho2 * ma.rho2);
    const double xx = mb.xi * ma.xi, sx = sqrt(xx);
    const double d_ixi = -d_f / xx;
    const double d_alpha = -d_f / (sx * (sqrt(mb.xi) + sqrt(ma.xi)));
    const double d_beta = d_f / xx;
    /* d(s^2 / rho^2) = (d(s^2) rho^2 - s^2 d(rho^2)) / (rho^2 rho'^2) */
    const double s2b = mb.s * mb.s, s2a = ma.s * ma.s;
    const double d_s2irho2 = (d_s2 * mb.rho2 - s2b * d_rho2) / (mb.rho2 * ma.rho2);
    /* d(1 / (rho^2 s^2)) = -(d(rho^2) s'^2 + rho^2 d(s^2)) / (P P'), P = rho^2 s^2 */
    const double d_ipp = -(d_rho2 * s2a + mb.rho2 * d_s2) / (mb.rho2 * s2b * ma.rho2 * s2a);
    const double d_grr = a2 * d_s2irho2 + d_ixi;
    const double d_grp = a * d_irho2;
    const double d_gtt = d_irho2;
    const double u0 = ub[0], u1 = ub[1], u2 = ub[2];         /* momenta unchanged by a position move */
    const double dG2 = d_grr * u0 * u0 + 2.0 * d_grp * u0 * u2 + d_gtt * u1 * u1 + d_ipp * u2 * u2;
    return 0.5 * (ma.alpha + mb.alpha) * dG2 / Gs + 0.5 * Gs * d_alpha - d_beta * u0;
}

/* The same quotient for a charged particle in the static Wald field, in
 * canonical variables w = (r, th, ph, pi_r, pi_th, pi_ph), pi_i = u_i +
 * (q/m) A_i (Eq. Amu, M = 1), of
 *   H_c(x, pi) = alpha Gamma(u) - beta^r u_r - (q/m) A_0,  u = pi - (q/m) A(x)
 * (Sec. 3.1.3's H written in pi).  Momentum moves change u by the same
 * increment, so their quotients are the geodesic ones at u.  A position
 * move changes the metric and u together; with P = r / rho^2 and
 * K = 1 + c^2 (A_0 = a B0 K P, A_ph = (B0/2) s^2 (r^2 + a^2 - 2 a^2 K P),
 * A_r = (B0/2)(2 a K P - a s^2)), the potential differences per unit
 * increment are
 *   r:  dP = (a^2 c^2 - r r') / (rho^2 rho'^2), d(KP) = K dP,
 *       dA_ph = (B0/2) s^2 (r + r' - 2 a^2 d(KP))
 *   th: dP = -r d(rho^2) / (rho^2 rho'^2), d(KP) = d(c^2) P' + K dP,
 *       dA_ph = (B0/2) (d(s^2) (r^2 + a^2 - 2 a^2 K' P') - 2 a^2 s^2 d(KP))
 *   both: dA_0 = a B0 d(KP), dA_r = (B0/2)(2 a d(KP) - a d(s^2)),
 * du_r = -(q/m) dA_r, du_ph = -(q/m) dA_ph, and
 *   Gamma'^2 - Gamma^2 = dg^ij u'_i u'_j + g^ij (du_i u'_j + u_i du_j),
 *   dH = (alpha' + alpha)/2 dGamma + (Gamma' + Gamma)/2 d(alpha)
 *        - (d(beta) u'_r + beta du_r) - (q/m) dA_0. */
static double dg_quot_em(double M, double a, double B0, double qm, const double *wb, const double *wa, int v)
{
    if (v == 2) return 0.0;
    const double rb = wb[0], ra = wa[0], tb = wb[1], ta = wa[1];
    om_t mb, ma;
    om_eval(M, a, rb, tb, &mb);
    om_eval(M, a, ra, ta, &ma);
    double ub[3] = {wb[3] - qm * wald_Ar(a, B0, rb, tb), wb[4], wb[5] - qm * wald_Aph(a, B0, rb, tb)};
    double ua[3] = {wa[3] - qm * wald_Ar(a, B0, ra, ta), wa[4], wa[5] - qm * wald_Aph(a, B0, ra, ta)};
    const double Gb = gamma_lorentz(&mb, ub), Ga = gamma_lorentz(&ma, ua);
    const double Gs = Ga + Gb;
    if (v == 3)
        return mb.alpha * (mb.gu_rr * (ua[0] + ub[0]) + 2.0 * mb.gu_rp * ub[2]) / Gs - mb.beta;
    if (v == 4)
        return mb.alpha * mb.gu_tt * (ua[1] + ub[1]) / Gs;
    if (v == 5)
        return mb.alpha * (2.0 * mb.gu_rp * ub[0] + mb.gu_pp * (ua[2] + ub[2])) / Gs;
    const double a2 = a * a;
    const double s2b = mb.s * mb.s, s2a = ma.s * ma.s, c2b = mb.c * mb.c, c2a = ma.c * ma.c;
    const double Pa = ra / ma.rho2, Kb = 1.0 + c2b, Ka = 1.0 + c2a;
    double d_rho2, d_f, d_s2, dP, dKP, dAph;
    if (v == 0) {
        d_rho2 = rb + ra;
        dP = (a2 * c2b - rb * ra) / (mb.rho2 * ma.rho2);
        d_f = 2.0 * M * dP;
        d_s2 = 0.0;
        dKP = Kb * dP;
        dAph = 0.5 * B0 * s2b * (rb + ra - 2.0 * a2 * dKP);
    } else {
        const double h = 0.5 * (ta - tb);
        const double d_c = -sin(0.5 * (ta + tb)) * sinc_(h);
        const double d_c2 = (mb.c + ma.c) * d_c;
        d_rho2 = a2 * d_c2;
        dP = -rb * d_rho2 / (mb.rho2 * ma.rho2);
        d_f = 2.0 * M * dP;
        d_s2 = -d_c2;
        dKP = d_c2 * Pa + Kb * dP;
        dAph = 0.5 * B0 * (d_s2 * (rb * rb + a2 - 2.0 * a2 * Ka * Pa) - 2.0 * a2 * s2b * dKP);
    }
    const double dA0 = a * B0 * dKP;
    const double dAr = 0.5 * B0 * (2.0 * a * dKP - a * d_s2);
    const double dur = -qm * dAr, dup = -qm * dAph;
    const double d_irho2 = -d_rho2 / (mb.rho2 * ma.rho2);
    const double xx = mb.xi * ma.xi, sx = sqrt(xx);
    const double d_ixi = -d_f / xx;
    const double d_alpha = -d_f / (sx * (sqrt(mb.xi) + sqrt(ma.xi)));
    const double d_beta = d_f / xx;
    const double d_s2irho2 = (d_s2 * mb.rho2 - s2b * d_rho2) / (mb.rho2 * ma.rho2);
    const double d_ipp = -(d_rho2 * s2a + mb.rho2 * d_s2) / (mb.rho2 * s2b * ma.rho2 * s2a);
    const double d_grr = a2 * d_s2irho2 + d_ixi;
    const double d_grp = a * d_irho2;
    const double d_gtt = d_irho2;
    const double dG2 = d_grr * ua[0] * ua[0] + 2.0 * d_grp * ua[0] * ua[2] + d_gtt * ua[1] * ua[1]
                     + d_ipp * ua[2] * ua[2]
                     + mb.gu_rr * (dur * ua[0] + ub[0] * dur)
                     + 2.0 * mb.gu_rp * (dur * ua[2] + ub[0] * dup)
                     + mb.gu_pp * (dup * ua[2] + ub[2] * dup);
    return 0.5 * (ma.alpha + mb.alpha) * dG2 / Gs + 0.5 * Gs * d_alpha - (d_beta * ua[0] + mb.beta * dur)
           - qm * dA0;
}

/* Coordinate-increment discrete gradient along one ordering of the six
 * variables (Sec. 2.2.3, Eq. hh and the displayed quotients): variable
 * ord[k] is moved from z0 to z1 in turn, and its component is the
 * difference quotient of H across that single move (dg_quot), so that the
 * components telescope: sum_v G_v (z1_v - z0_v) = H(z1) - H(z0) (exactly in
 * exact arithmetic, to rounding here).  Appendix D replaces the quotient by
 * the analytic partial when |z1_v - z0_v| < eps, a guard against the 0/0 of
 * the plain quotient; the closed form has no 0/0 (it tends to the partial),
 * so eps is not used. */
static void dg_path(double M, double a, double B0, double qm, const double *z0, const double *z1,
                    const int *ord, double eps, double *G)
{
    (void)eps;
    double zb[6], za[6];
    memcpy(zb, z0, sizeof zb);
    for (int k = 0; k < 6; ++k) {
        int v = ord[k];
        memcpy(za, zb, sizeof za);
        za[v] = z1[v];
        G[v] = (qm != 0.0 && B0 != 0.0) ? dg_quot_em(M, a, B0, qm, zb, za, v) : dg_quot(M, a, zb, za, v);
        memcpy(zb, za, sizeof zb);
    }
}

/* The symmetrised discrete gradient.  Reading: Appendix D prints a 1/6
 * average over update orders that is visibly garbled; the scheme is taken
 * from its principle: the average over all 12 orderings made of the 3! orders
 * of the coordinate pairs (r,u_r), (th,u_th), (ph,u_ph) times the two
 * within-pair orders (coordinate first, or momentum first, for every pair).
 * Each ordering telescopes exactly, so their average conserves H exactly;
 * the set is closed under reversal, which makes the scheme time-symmetric. */
static void dg_grad(double M, double a, double B0, double qm, const double *z0, const double *z1, double eps,
                    double *G)
{
    static const int pairs[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    double acc[6] = {0, 0, 0, 0, 0, 0}, g[6];
    for (int p = 0; p < 6; ++p)
        for (int xf = 0; xf < 2; ++xf) {
            int ord[6];
            for (int q = 0; q < 3; ++q) {
                int x = pairs[p][q], u = 3 + pairs[p][q];
                ord[2 * q] = xf ? x : u;
                ord[2 * q + 1] = xf ? u : x;
            }
            dg_path(M, a, B0, qm, z0, z1, ord, eps, g);
            for (int i = 0; i < 6; ++i) acc[i] += g[i];
        }
    for (int i = 0; i < 6; ++i) G[i] = acc[i] / 12.0;
}

/* Sec. 2.2.3: discrete-gradient Hamiltonian step for geodesics,
 * dx/dt = D_u H, du/dt = -D_x H, solved by fixed-point iteration on z^{n+1}
 * (same stop rule as the IMR). */
/* Kinetic <-> canonical momenta of a charged particle in the Wald field:
 * pi_i = u_i + (q/m) A_i (A_th = 0); sgn = +1 maps u -> pi, -1 pi -> u. */
static void canonical(double a, double B0, double qm, double *z, double sgn)
{
    z[3] += sgn * qm * wald_Ar(a, B0, z[0], z[1]);
    z[5] += sgn * qm * wald_Aph(a, B0, z[0], z[1]);
}

static int step_ham(const or_ctx *c, double h, const double *z0, const double *guess, double *z1)
{
    /* Charged particles in the analytic Wald field (an extension, not in the
     * paper): the same scheme on H_c(x, pi) with the potentials of Eq. (Amu),
     * iterated in canonical variables, which conserves H and L exactly. */
    const double B0 = (c->qm != 0.0 && c->p->field_kind == OR_FIELD_WALD) ? c->p->B0field : 0.0;
    double w0[6], zk[6], G[6], zn[6];
    memcpy(w0, z0, sizeof w0);
    memcpy(zk, guess, sizeof zk);
    if (B0 != 0.0) {
        canonical(c->p->a, B0, c->qm, w0, 1.0);
        canonical(c->p->a, B0, c->qm, zk, 1.0);
    }
    int k, ok = 0;
    for (k = 1; k <= c->p->max_iter; ++k) {
        dg_grad(c->p->M, c->p->a, B0, c->qm, w0, zk, c->p->dg_eps, G);
        for (int i = 0; i < 3; ++i) {
            zn[i] = w0[i] + h * G[3 + i];
            zn[3 + i] = w0[3 + i] - h * G[i];
        }
        ok = converged(zn, zk, c->p->tol);
        memcpy(zk, zn, sizeof zk);
        if (ok) break;
    }
    if (B0 != 0.0) canonical(c->p->a, B0, c->qm, zk, -1.0);
    memcpy(z1, zk, sizeof zk);
    return ok ? k : -c->p->max_iter;
}

/* Particle boundary conditions (Sec. 2.5, closing paragraph), half-th
 * domain.  Reading: crossing a pole maps th -> -th (or 2 pi - th), flips
 * u_th and adds pi to ph (the paper states only the u_th flip).
 * Returns 0 if the particle is removed (r < r_h or r > r_max). */
static int particle_bc(const or_push_params *p, double *z)
{
    if (p->theta_full) {
        /* full-theta domain (Sec. 2.5): periodic in th, no reflection */
        const double P = p->theta_period;
        while (z[1] < p->theta_lo) z[1] += P;
        while (z[1] >= p->theta_lo + P) z[1] -= P;
    } else if (z[1] < 0.0) {
        z[1] = -z[1];
        z[4] = -z[4];
        z[2] += M_PI;
    } else if (z[1] > M_PI) {
        z[1] = 2.0 * M_PI - z[1];
        z[4] = -z[4];
        z[2] += M_PI;
    }
    if (!(z[0] >= p->r_h) || !(z[0] <= p->r_max)) return 0;
    return 1;
}

/* An IMR step whose solve did not converge, or whose end point has
 * |H - H^n| / D_0 > substep_tol (reading: the paper gives no policy; such
 * steps are found within a few 1e-4 rad of the polar axis, where the
 * u_ph^2 / sin^3 th terms change faster than the step resolves and a
 * solve either fails or converges to an inaccurate end point):
 * the step is redone from z^n as m = 2, 4, ..., 2^K substeps of h/m, each
 * an IMR solve of the same form (capped at min(max_iter, 16) iterations: a
 * level whose substeps need more is too coarse) started from the substep's
 * own start state,
 * with the pole reflection of the particle boundaries applied after each
 * substep.  The first level whose solves all converge and whose end state
 * has |H - H(z^n)| / D_0 <= substep_tol (0: no H condition) is taken;
 * failing that, the finest level whose solves all converged; failing that,
 * nothing (the full-step solve's own result stands).  *its accumulates the
 * iterations of every attempt.  Returns 1 if a level was taken. */
static int imr_substeps(const or_ctx *c, double h, const double *z0, double H0ref, double D0, double *z1, int *its);

/* The full-step IMR solve's outcome it (iterations, negative if it did not
 * converge) and end point z1, revised by the substeps when they apply. */
static int imr_revise(const or_ctx *c, double h, const double *z0, double Hn, double D0, double *z1, int it)
{
    const or_push_params *p = c->p;
    or_bh bh = {p->M, p->a, p->B0pot};
    if (p->imr_substeps <= 0) return it;
    if (!(it < 0 || (p->substep_tol > 0.0 && fabs(ham(&bh, c->qm, z1) - Hn) / D0 > p->substep_tol))) return it;
    int sit = 0;
    const int ok = imr_substeps(c, h, z0, ham(&bh, c->qm, z0), D0, z1, &sit);
    const int mag = (it < 0 ? -it : it) + sit;
    return (it >= 0 || ok) ? mag : -mag;
}
static int imr_substeps(const or_ctx *c, double h, const double *z0, double H0ref, double D0, double *z1, int *its)
{
    const or_push_params *p = c->p;
    or_bh bh = {p->M, p->a, p->B0pot};
    or_push_params ps = *p;
    ps.max_iter = p->max_iter < 16 ? p->max_iter : 16;
    const or_ctx cs = {&ps, c->g, c->F, c->qm};
    double best[6];
    int have = 0;
    for (int k = 1; k <= p->imr_substeps; ++k) {
        const int m = 1 << k;
        double zs[6], zn[6];
        memcpy(zs, z0, sizeof zs);
        int ok = 1;
        for (int s = 0; s < m && ok; ++s) {
            const int it = step_imr(&cs, h / m, zs, zs, zn);
            *its += it < 0 ? -it : it;
            if (it < 0) ok = 0;
            particle_bc(p, zn);
            memcpy(zs, zn, sizeof zs);
        }
        if (!ok) continue;
        memcpy(best, zs, sizeof best);
        have = 1;
        if (p->substep_tol <= 0.0 || fabs(ham(&bh, c->qm, zs) - H0ref) / D0 <= p->substep_tol) break;
    }
    if (have) memcpy(z1, best, sizeof best);
    return have;
}

/* One step of one particle.  Hybrid (Sec. 3.1.2): RK4 trial, then
 *   Hyb2: accept iff Ht^{n+1} < Ht_max,
 *   Hyb1: accept iff (Ht^{n+1} - Ht^n)/dt < (dHt/dt)_max,
 * with Ht = |H - H_0| / D_0; otherwise the step is redone from z^n by the
 * implicit scheme (IMR for any particle, or the discrete-gradient scheme
 * for geodesics), started from the rejected trial, and always accepted.
 * A NaN test value rejects.  Returns 1 if the implicit iteration hit its
 * cap, else 0. */
static int push_one(const or_ctx *c, double *z, double H0, double D0, double *Hn,
                    uint8_t *scheme_out, uint8_t *iters_out)
{
    const or_push_params *p = c->p;
    or_bh bh = {p->M, p->a, p->B0pot};
    double z0[6], z1[6], trial[6];
    memcpy(z0, z, sizeof z0);
    int it = 0, implicit = 0;
    if (p->scheme == OR_RK4) {
        step_rk4(c, z0, z1);
    } else if (p->scheme == OR_IMR) {
        it = step_imr(c, p->dt, z0, z0, z1);
        implicit = 1;
        it = imr_revise(c, p->dt, z0, *Hn, D0, z1, it);
    } else if (p->scheme == OR_HAM) {
        it = step_ham(c, p->dt, z0, z0, z1);
        implicit = 1;
    } else {
        step_rk4(c, z0, trial);
        double H1 = ham(&bh, c->qm, trial);
        double Ht1 = fabs(H1 - H0) / D0;
        int accept;
        if (p->scheme == OR_HYB2) {
            accept = Ht1 < p->thr;
        } else {
            double Htn = fabs(*Hn - H0) / D0;
            accept = (Ht1 - Htn) / p->dt < p->thr;
        }
        if (accept) {
            memcpy(z1, trial, sizeof z1);
        } else {
            /* Adaptive step (Sec. 3.1.2, Tab. C.2): the implicit partner
             * takes its own step dt_imp.  Reading: its iteration starts from
             * the trial's increment scaled to that step,
             * z^n + (z_RK4 - z^n) dt_imp / dt (the trial itself when the
             * steps are equal). */
            implicit = 1;
            const double hi = p->dt_imp > 0.0 ? p->dt_imp : p->dt;
            double guess[6];
            if (hi == p->dt) {
                memcpy(guess, trial, sizeof guess);
            } else {
                const double ratio = hi / p->dt;
                for (int i = 0; i < 6; ++i) guess[i] = z0[i] + (trial[i] - z0[i]) * ratio;
            }
            if (p->implicit_kind == OR_HAM) {
                it = step_ham(c, hi, z0, guess, z1);
            } else {
                it = step_imr(c, hi, z0, guess, z1);
                it = imr_revise(c, hi, z0, *Hn, D0, z1, it);
            }
        }
    }
    *Hn = ham(&bh, c->qm, z1);
    memcpy(z, z1, sizeof z1);
    *scheme_out = (uint8_t)implicit;
    int a = it < 0 ? -it : it;
    *iters_out = (uint8_t)(a > 255 ? 255 : a);
    return it < 0;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (called through ctypes by the test-suite).         */
/* ------------------------------------------------------------------------ */

void or_metric(double M, double a, int64_t n, const double *r, const double *th, double *out)
{
    for (int64_t p = 0; p < n; ++p) {
        om_t m;
        om_eval(M, a, r[p], th[p], &m);
        double *o = out + 13 * p;
        o[0] = m.rho2; o[1] = m.xi; o[2] = m.alpha; o[3] = m.beta;
        o[4] = m.g_rr; o[5] = m.g_rp; o[6] = m.g_tt; o[7] = m.g_pp;
        o[8] = m.gu_rr; o[9] = m.gu_rp; o[10] = m.gu_tt; o[11] = m.gu_pp;
        o[12] = m.sqrtg;
    }
}

void or_metric_deriv(double M, double a, int64_t n, const double *r, const double *th, double *out)
{
    for (int64_t p = 0; p < n; ++p) om_deriv(M, a, r[p], th[p], out + 12 * p);
}

void or_wald(double a, double B0, int64_t n, const double *r, const double *th,
             double *B, double *E, double *D, double *A0, double *Aph)
{
    for (int64_t p = 0; p < n; ++p) {
        double Bx[3];
        wald_BE(a, B0, r[p], th[p], B + 3 * p, E + 3 * p);
        wald_D(a, B0, r[p], th[p], D + 3 * p, Bx);
        A0[p] = wald_A0(a, B0, r[p], th[p]);
        Aph[p] = wald_Aph(a, B0, r[p], th[p]);
    }
}

/* H, L and the normaliser D_0 for n states (n x 6). */
void or_hamiltonian(double M, double a, double B0pot, int64_t n, const double *z,
                    const double *qm, double *H, double *L, double *Dn)
{
    or_bh bh = {M, a, B0pot};
    for (int64_t p = 0; p < n; ++p) {
        if (H) H[p] = ham(&bh, qm[p], z + 6 * p);
        if (L) L[p] = angmom(&bh, qm[p], z + 6 * p);
        if (Dn) Dn[p] = ham_norm(&bh, qm[p], z + 6 * p);
    }
}

/* Momentum blocks A, J of the IMR Newton matrix (row-major 3 x 3 each) at
 * n states, B per state (n x 3; NULL = no field). */
void or_imr_blocks(double M, double a, int64_t n, const double *z, const double *qm, const double *B,
                   double *A, double *J)
{
    for (int64_t p = 0; p < n; ++p) {
        double a3[3][3], j3[3][3];
        imr_blocks_at(M, a, qm[p], z + 6 * p, B ? B + 3 * p : NULL, a3, j3);
        memcpy(A + 9 * p, a3, sizeof a3);
        memcpy(J + 9 * p, j3, sizeof j3);
    }
}

/* Right-hand side at n states with fields given per state (D,B n x 3 each;
 * NULL = no field). */
void or_rhs(double M, double a, int64_t n, const double *z, const double *qm,
            const double *D, const double *B, double *f)
{
    for (int64_t p = 0; p < n; ++p)
        rhs(M, a, qm[p], z + 6 * p, D ? D + 3 * p : NULL, B ? B + 3 * p : NULL, f + 6 * p);
}

void or_gather(int Nr, int Nth, int ld, const double *rn, const double *rh,
               const double *tn, const double *th, const double *const *F,
               int64_t n, const double *r, const double *t, double *DB, int full)
{
    or_grid g = {Nr, Nth, ld, rn, rh, tn, th, full};
    for (int64_t p = 0; p < n; ++p) gather(&g, F, r[p], t[p], DB + 6 * p, DB + 6 * p + 3);
}

/* Integer-grid cell index ir * Nth + ith (Sec. 2.3, "located between nodes"). */
void or_cell_index(int Nr, int Nth, const double *rn, const double *tn, int64_t n,
                   const double *r, const double *t, uint32_t *cell)
{
    for (int64_t p = 0; p < n; ++p) {
        int i = locate(rn, Nr + 1, r[p]);
        int j = locate(tn, Nth + 1, t[p]);
        cell[p] = (uint32_t)i * (uint32_t)Nth + (uint32_t)j;
    }
}

/* Discrete gradient between two states (exposed for the conservation pins). */
void or_dg_quot(double M, double a, const double *zb, const double *za, int v, double *G)
{
    *G = dg_quot(M, a, zb, za, v);
}

/* Charged quotient in canonical variables (Wald field B0, q/m = qm). */
void or_dg_quot_em(double M, double a, double B0, double qm, const double *wb, const double *wa, int v, double *G)
{
    *G = dg_quot_em(M, a, B0, qm, wb, wa, v);
}

void or_wald_A(double a, double B0, int64_t n, const double *r, const double *th, double *Ar, double *Aph)
{
    for (int64_t p = 0; p < n; ++p) {
        Ar[p] = wald_Ar(a, B0, r[p], th[p]);
        Aph[p] = wald_Aph(a, B0, r[p], th[p]);
    }
}

void or_dg_grad(double M, double a, const double *z0, const double *z1, double eps, double *G)
{
    dg_grad(M, a, 0.0, 0.0, z0, z1, eps, G);
}

/* One step of n particles.  F: six field arrays (Yee layout) when
 * field_kind == OR_FIELD_GRID.  Returns the number of particles whose
 * implicit iteration reached the cap. */
int64_t or_push(const or_push_params *p, int Nr, int Nth, int ld, const double *rn,
                const double *rh, const double *tn, const double *th,
                const double *const *F, int64_t n, double *z, const double *qm,
                const double *H0, const double *D0, double *Hn, uint8_t *alive,
                uint8_t *scheme_out, uint8_t *iters_out, uint8_t *notconv_out)
{
    or_grid g = {Nr, Nth, ld, rn, rh, tn, th, p->theta_full};
    int64_t notconv = 0;
    for (int64_t k = 0; k < n; ++k) {
        scheme_out[k] = 0;
        iters_out[k] = 0;
        if (notconv_out) notconv_out[k] = 0;
        if (!alive[k]) continue;
        or_ctx c = {p, &g, F, qm[k]};
        const int nc = push_one(&c, z + 6 * k, H0[k], D0[k], Hn + k, scheme_out + k, iters_out + k);
        notconv += nc;
        if (notconv_out) notconv_out[k] = (uint8_t)nc;
        if (!particle_bc(p, z + 6 * k)) alive[k] = 0;
    }
    return notconv;
}

/* Wald field sampled at every Yee point (Appendix B.1; each component at its
 * own staggered location).  F: six arrays of size (Nr+1)*ld. */
void or_wald_on_grid(double a, double B0, int Nr, int Nth, int ld, const double *rn,
                     const double *rh, const double *tn, const double *th, double *const *F)
{
    for (int k = 0; k < 6; ++k) {
        int mx = yee_roff[k] ? Nr : Nr + 1;
        int my = yee_toff[k] ? Nth : Nth + 1;
        for (int i = 0; i < mx; ++i)
            for (int j = 0; j < my; ++j) {
                double r = yee_roff[k] ? rh[i] : rn[i];
                double t = yee_toff[k] ? th[j] : tn[j];
                double D[3], B[3];
                wald_D(a, B0, r, t, D, B);
                F[k][i * ld + j] = k < 3 ? D[k] : B[k - 3];
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Particle initialisation from caller-supplied random draws.               */
/* ------------------------------------------------------------------------ */

/* Bound-orbit seeding (test-particle workload): for each candidate
 * (r, th, E, L, sgn) solve H(r, th, u_r, u_th = 0, u_ph = L) = E for u_r,
 * i.e. alpha^2 (1 + g^rr u_r^2 + 2 g^rp L u_r + g^pp L^2) = (E + beta u_r)^2
 * with E + beta u_r > 0, taking the root picked by sgn.  The first
 * candidate with a valid root is used.  cand: n x K x 5.  Returns the number
 * of particles without a valid candidate (their state is left NaN). */
int64_t or_seed_orbits(double M, double a, int64_t n, int K, const double *cand, double *z)
{
    int64_t bad = 0;
    for (int64_t p = 0; p < n; ++p) {
        int done = 0;
        for (int k = 0; k < K && !done; ++k) {
            const double *c = cand + ((size_t)p * K + k) * 5;
            double r = c[0], th = c[1], E = c[2], L = c[3], sg = c[4];
            om_t m;
            om_eval(M, a, r, th, &m);
            double a2 = m.alpha * m.alpha;
            double A = a2 * m.gu_rr - m.beta * m.beta;
            double Bq = a2 * m.gu_rp * L - E * m.beta;
            double C = a2 * (1.0 + m.gu_pp * L * L) - E * E;
            double disc = Bq * Bq - A * C;
            if (!(disc >= 0.0) || !(A > 0.0)) continue;
            double ur = (-Bq + (sg >= 0.0 ? 1.0 : -1.0) * sqrt(disc)) / A;
            if (!(E + m.beta * ur > 0.0)) continue;
            double *o = z + 6 * p;
            o[0] = r; o[1] = th; o[2] = 0.0; o[3] = ur; o[4] = 0.0; o[5] = L;
            done = 1;
        }
        if (!done) {
            for (int i = 0; i < 6; ++i) z[6 * p + i] = NAN;
            ++bad;
        }
    }
    return bad;
}

/* Thermal seeding: a FIDO-frame momentum uhat (orthonormal triad
 * components) is mapped to covariant u_i = L_ia uhat_a with gamma_ij = L L^T
 * (Cholesky, order r, th, ph), so that g^ij u_i u_j = |uhat|^2.
 * draws: n x 6 = (r, th, ph, uhat_1, uhat_2, uhat_3). */
void or_seed_fido(double M, double a, int64_t n, const double *draws, double *z)
{
    for (int64_t p = 0; p < n; ++p) {
        const double *d = draws + 6 * p;
        om_t m;
        om_eval(M, a, d[0], d[1], &m);
        double L11 = sqrt(m.g_rr);
        double L31 = m.g_rp / L11;
        double L22 = sqrt(m.g_tt);
        double L33 = sqrt(m.g_pp - L31 * L31);
        double *o = z + 6 * p;
        o[0] = d[0]; o[1] = d[1]; o[2] = d[2];
        o[3] = L11 * d[3];
        o[4] = L22 * d[4];
        o[5] = L31 * d[3] + L33 * d[5];
    }
}
