/*
 * FPIC oracle, grid side: charge/current deposition (Sec. 2.3) and the FDTD
 * leapfrog of the Maxwell equations (Sec. 2.1, Sec. 2.5).
 *
 * TEST INFRASTRUCTURE ONLY (see fpic_oracle.c).  Plain serial FP64 loops,
 * compiled with -ffp-contract=off; shares nothing with the CUDA library.
 *
 * Grid conventions as in fpic_oracle.c: arrays [i * ld + j], integer nodes
 * rn (Nr+1), tn (Nth+1), half nodes rh (Nr), th (Nth).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Appendix A metric (restated locally; this file is self-contained) --- */
typedef struct {
    double alpha, beta, sqrtg, g_rr, g_rp, g_tt, g_pp, gu_rr, gu_rp, gu_tt, gu_pp;
} pm_t;

static void pm_eval(double M, double a, double r, double th, pm_t *m)
{
    double s = sin(th), c = cos(th), s2 = s * s;
    double rho2 = r * r + a * a * c * c;
    double xi = 1.0 + 2.0 * M * r / rho2;
    m->alpha = 1.0 / sqrt(xi);
    m->beta = (xi - 1.0) / xi;
    m->sqrtg = rho2 * sqrt(xi) * s;
    m->g_rr = xi;
    m->g_rp = -a * xi * s2;
    m->g_tt = rho2;
    m->g_pp = s2 * (rho2 + a * a * xi * s2);
    m->gu_rr = a * a * s2 / rho2 + 1.0 / xi;
    m->gu_rp = a / rho2;
    m->gu_tt = 1.0 / rho2;
    m->gu_pp = 1.0 / (rho2 * s2);
}

static double sqrtg_at(double M, double a, double r, double th)
{
    double s = sin(th), c = cos(th);
    double rho2 = r * r + a * a * c * c;
    return rho2 * sqrt(1.0 + 2.0 * M * r / rho2) * s;
}

typedef struct {
    int Nr, Nth, ld;
    const double *rn, *rh, *tn, *th;
} pg_t;

static int loc(const double *X, int m, double x)
{
    if (!(x >= X[0])) return 0;
    if (x >= X[m - 1]) return m - 2;
    int lo = 0, hi = m - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x >= X[mid]) lo = mid; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: volume-weighted deposition.                                    */
/* ------------------------------------------------------------------------ */

/* 2D trapezoidal rule of sqrt(gamma) over [x0,x1] x [y0,y1] with 4 x 4
 * points (Sec. 2.3: "discretising each cell into 4 x 4 points").
 * Reading: the 4 x 4 rule is applied to each sub-rectangle. */
static double trap16(double M, double a, double x0, double x1, double y0, double y1, int unit)
{
    static const double wt[4] = {0.5, 1.0, 1.0, 0.5};
    double hx = (x1 - x0) / 3.0, hy = (y1 - y0) / 3.0, acc = 0.0;
    for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) {
            double x = x0 + k * hx, y = y0 + l * hy;
            double f = unit ? 1.0 : sqrtg_at(M, a, x, y);
            acc += wt[k] * wt[l] * f;
        }
    return acc * hx * hy;
}

/* Node weights of a particle at (r, t) on the sub-grid with node lists X, Y
 * (Eqs. v1-v5 and the four q_(.,.) relations): the node (i+a, j+b) receives
 * the subvolume of the opposite corner over V.  Reading: V is the sum of the
 * four subvolumes (so the weights sum to one); the point is clamped into the
 * sub-grid's node range.  Returns i, j and w[b][a] (a = r offset). */
static void vol_weights(double M, double a, const double *X, int mx, const double *Y, int my,
                        double r, double t, int unit, int *io, int *jo, double w[2][2])
{
    if (r < X[0]) r = X[0];
    if (r > X[mx - 1]) r = X[mx - 1];
    if (t < Y[0]) t = Y[0];
    if (t > Y[my - 1]) t = Y[my - 1];
    int i = loc(X, mx, r), j = loc(Y, my, t);
    double r0 = X[i], r1 = X[i + 1], t0 = Y[j], t1 = Y[j + 1];
    double V00 = trap16(M, a, r0, r, t0, t, unit);   /* V_(i,j):     [r_i, r] x [t_j, t]   */
    double V10 = trap16(M, a, r, r1, t0, t, unit);   /* V_(i+1,j):   [r, r_i+1] x [t_j, t] */
    double V01 = trap16(M, a, r0, r, t, t1, unit);   /* V_(i,j+1)                          */
    double V11 = trap16(M, a, r, r1, t, t1, unit);   /* V_(i+1,j+1)                        */
    double V = V00 + V10 + V01 + V11;
    w[0][0] = V11 / V;   /* q_(i,j)     */
    w[0][1] = V01 / V;   /* q_(i+1,j)   */
    w[1][0] = V10 / V;   /* q_(i,j+1)   */
    w[1][1] = V00 / V;   /* q_(i+1,j+1) */
    *io = i;
    *jo = j;
}

/* Dual-cell volume of every node of a sub-grid: 2 pi times the 4 x 4
 * trapezoid of sqrt(gamma) over [X_{i-1/2}, X_{i+1/2}] x [Y_{j-1/2}, Y_{j+1/2}],
 * where the half points are the neighbouring nodes' midpoints in the list
 * (node midpoints of the other staggering), clipped to the list's ends.
 * Reading: the paper does not normalise the deposit; densities per unit
 * (axisymmetric) proper volume need this volume. */
static double dual_edge(const double *X, const double *Xo, int mx, int off, int i, int lo)
{
    /* X: this sub-grid's nodes (mx of them); Xo: the other staggering.
     * off = 1 if this list is the half-node list. */
    if (lo) {
        if (off) return Xo[i];                  /* half node i+1/2: lower edge r_i        */
        return i == 0 ? X[0] : Xo[i - 1];       /* integer node i: lower edge r_{i-1/2}   */
    }
    if (off) return Xo[i + 1];
    return i == mx - 1 ? X[mx - 1] : Xo[i];
}

/* Deposit: rho and the FIDO current j^i = sum Q v^i W / (2 pi V_dual), with
 * Q = w (q/m) and v^j = gamma^ij u_i / Gamma (Sec. 2.3), each on its Yee
 * sub-grid: rho, j^ph at (i, j), j^r at (i+1/2, j), j^th at (i, j+1/2).
 * Outputs are zeroed first.  unit != 0 replaces sqrt(gamma) by 1 in the
 * weights (tests only). */
void or_deposit(double M, double a, int Nr, int Nth, int ld, const double *rn, const double *rh,
                const double *tn, const double *th, int64_t n, const double *z, const double *qm,
                const double *w, const uint8_t *alive, double *rho, double *jr, double *jt, double *jp,
                int unit, int normalise)
{
    size_t sz = (size_t)(Nr + 1) * ld;
    memset(rho, 0, sz * sizeof(double));
    memset(jr, 0, sz * sizeof(double));
    memset(jt, 0, sz * sizeof(double));
    memset(jp, 0, sz * sizeof(double));
    for (int64_t p = 0; p < n; ++p) {
        if (!alive[p]) continue;
        const double *s = z + 6 * p;
        double r = s[0], t = s[1];
        pm_t m;
        pm_eval(M, a, r, t, &m);
        double ur = s[3], ut = s[4], up = s[5];
        double Ur = m.gu_rr * ur + m.gu_rp * up, Ut = m.gu_tt * ut, Up = m.gu_rp * ur + m.gu_pp * up;
        double G = sqrt(1.0 + ur * Ur + ut * Ut + up * Up);
        double Q = w[p] * qm[p];
        double v[3] = {Ur / G, Ut / G, Up / G};
        int i, j;
        double W[2][2];
        /* (i, j): rho and j^ph */
        vol_weights(M, a, rn, Nr + 1, tn, Nth + 1, r, t, unit, &i, &j, W);
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                rho[(i + c) * ld + j + b] += Q * W[b][c];
                jp[(i + c) * ld + j + b] += Q * v[2] * W[b][c];
            }
        /* (i+1/2, j): j^r */
        vol_weights(M, a, rh, Nr, tn, Nth + 1, r, t, unit, &i, &j, W);
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) jr[(i + c) * ld + j + b] += Q * v[0] * W[b][c];
        /* (i, j+1/2): j^th */
        vol_weights(M, a, rn, Nr + 1, th, Nth, r, t, unit, &i, &j, W);
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) jt[(i + c) * ld + j + b] += Q * v[1] * W[b][c];
    }
    if (!normalise) return;
    /* divide by 2 pi V_dual of each node */
    for (int k = 0; k < 4; ++k) {
        int ro = (k == 2), to = (k == 3);     /* rho, j^ph: (0,0); j^r: (1,0); j^th: (0,1) */
        double *f = k == 0 ? rho : k == 1 ? jp : k == 2 ? jr : jt;
        const double *X = ro ? rh : rn, *Xo = ro ? rn : rh;
        const double *Y = to ? th : tn, *Yo = to ? tn : th;
        int mx = ro ? Nr : Nr + 1, my = to ? Nth : Nth + 1;
        for (int ii = 0; ii < mx; ++ii)
            for (int jj = 0; jj < my; ++jj) {
                double x0 = dual_edge(X, Xo, mx, ro, ii, 1), x1 = dual_edge(X, Xo, mx, ro, ii, 0);
                double y0 = dual_edge(Y, Yo, my, to, jj, 1), y1 = dual_edge(Y, Yo, my, to, jj, 0);
                double V = 2.0 * M_PI * trap16(M, a, x0, x1, y0, y1, unit);
                f[ii * ld + jj] /= V;
            }
    }
}

/* Dual volumes (2 pi x trapezoid) of the four sub-grids, exposed for tests:
 * out: 4 arrays (rho/j^ph, j^ph, j^r, j^th layouts). */
void or_dual_volumes(double M, double a, int Nr, int Nth, int ld, const double *rn, const double *rh,
                     const double *tn, const double *th, double *vol00, double *vol10, double *vol01)
{
    double *outs[3] = {vol00, vol10, vol01};
    for (int k = 0; k < 3; ++k) {
        int ro = (k == 1), to = (k == 2);
        const double *X = ro ? rh : rn, *Xo = ro ? rn : rh;
        const double *Y = to ? th : tn, *Yo = to ? tn : th;
        int mx = ro ? Nr : Nr + 1, my = to ? Nth : Nth + 1;
        for (int ii = 0; ii < mx; ++ii)
            for (int jj = 0; jj < my; ++jj) {
                double x0 = dual_edge(X, Xo, mx, ro, ii, 1), x1 = dual_edge(X, Xo, mx, ro, ii, 0);
                double y0 = dual_edge(Y, Yo, my, to, jj, 1), y1 = dual_edge(Y, Yo, my, to, jj, 0);
                outs[k][ii * ld + jj] = 2.0 * M_PI * trap16(M, a, x0, x1, y0, y1, 0);
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: FDTD leapfrog on the Yee grid, Sec. 2.5: boundaries.           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double M, a, dt;
    double chi0, lam, r_abs, r_max;   /* absorbing layer, Eqs. (abs0)-(abs2) */
    int conserving;                   /* j arrays hold coordinate currents J (or_deposit_conserving) */
    int full;                         /* full-theta domain: periodic in th (Sec. 2.5) */
} or_fdtd_params;

typedef struct {
    const or_fdtd_params *p;
    pg_t g;
} fctx;

/* Coordinates of a point of staggering (ro, to) and index (i, j). */
static double R(const fctx *c, int ro, int i) { return ro ? c->g.rh[i] : c->g.rn[i]; }
static double T(const fctx *c, int to, int j) { return to ? c->g.th[j] : c->g.tn[j]; }
static int NR(const fctx *c, int ro) { return ro ? c->g.Nr : c->g.Nr + 1; }
static int NT(const fctx *c, int to) { return to ? c->g.Nth : c->g.Nth + 1; }

/* Full-theta domain (Sec. 2.5: periodic boundaries at th_max = th_0 + 2 pi;
 * reading: the node range is [tn_0, tn_0 + P), P = tn[Nth] - tn[0] = 2 pi,
 * with Nth distinct nodes and Nth distinct half nodes; column Nth of every
 * array holds the image of column 0, the way the gather reads it).  The
 * backward th difference at j = 0 reaches the half node below th_0, i.e.
 * th[Nth-1] - P: its spacing is th_ext - th[Nth-1] with th_ext = th[0] + P. */
static double th_ext(const fctx *c)
{
    return c->g.th[0] + (c->g.tn[c->g.Nth] - c->g.tn[0]);
}

static void theta_images(const fctx *c, double *const F[3])
{
    if (!c->p->full) return;
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i <= c->g.Nr; ++i) F[k][i * c->g.ld + c->g.Nth] = F[k][i * c->g.ld];
}

/* Eq. (abs2): chi(r) = chi0 ((r - r_abs)/(r_max - r_abs))^lambda beyond r_abs.
 * Reading: the damping term -chi F is integrated exactly over the step, i.e.
 * the updated value is multiplied by exp(-chi dt) ("exponentially damp"). */
static double damp(const fctx *c, double r)
{
    const or_fdtd_params *p = c->p;
    if (p->chi0 <= 0.0 || r <= p->r_abs) return 1.0;
    double x = (r - p->r_abs) / (p->r_max - p->r_abs);
    return exp(-p->chi0 * pow(x, p->lam) * p->dt);
}

/* Metric-weighted average of F (staggering (ro,to)) at the point (ro2,to2)
 * displaced by half a cell along one axis (Sec. 2.1, the B^r example):
 * F_target = [(sqrtg F)_a + (sqrtg F)_b] / (2 sqrtg_target); a neighbour
 * outside the array is replaced by the one inside (zero gradient). */
static double avg_r(const fctx *c, const double *F, int ro, int to, int i2, int j)
{
    /* F has r staggering ro; the target has r staggering 1 - ro, index i2.
     * Neighbours in F: if target is half (ro = 0): i2 and i2+1; if target is
     * integer (ro = 1): i2-1 and i2. */
    const fctx *cc = c;
    int ia = ro ? i2 - 1 : i2, ib = ro ? i2 : i2 + 1;
    int m = NR(cc, ro);
    if (ia < 0) ia = ib;
    if (ib > m - 1) ib = ia;
    double t = T(cc, to, j);
    double sa = sqrtg_at(cc->p->M, cc->p->a, R(cc, ro, ia), t);
    double sb = sqrtg_at(cc->p->M, cc->p->a, R(cc, ro, ib), t);
    double st = sqrtg_at(cc->p->M, cc->p->a, R(cc, 1 - ro, i2), t);
    return (sa * F[ia * cc->g.ld + j] + sb * F[ib * cc->g.ld + j]) / (2.0 * st);
}

/* Eq. (Ei): E_i = alpha D_i + sqrtg eta_ijk beta^j B^k, beta = (beta^r,0,0):
 *   E_r  (i+1/2, j)   = alpha (g_rr D^r + g_rp <D^ph>)
 *   E_th (i, j+1/2)   = alpha g_tt D^th - sqrtg beta <B^ph>
 *   E_ph (i, j)       = alpha (g_rp <D^r> + g_pp D^ph) + sqrtg beta <B^th>  */
static void make_E(const fctx *c, const double *const D[3], const double *const B[3], double *const E[3])
{
    const or_fdtd_params *p = c->p;
    int ld = c->g.ld;
    for (int i = 0; i < c->g.Nr; ++i)
        for (int j = 0; j <= c->g.Nth; ++j) {
            pm_t m;
            pm_eval(p->M, p->a, c->g.rh[i], c->g.tn[j], &m);
            double Dp = avg_r(c, D[2], 0, 0, i, j);
            E[0][i * ld + j] = m.alpha * (m.g_rr * D[0][i * ld + j] + m.g_rp * Dp);
        }
    for (int i = 0; i <= c->g.Nr; ++i)
        for (int j = 0; j < c->g.Nth; ++j) {
            pm_t m;
            pm_eval(p->M, p->a, c->g.rn[i], c->g.th[j], &m);
            double Bp = avg_r(c, B[2], 1, 1, i, j);
            E[1][i * ld + j] = m.alpha * m.g_tt * D[1][i * ld + j] - m.sqrtg * m.beta * Bp;
        }
    for (int i = 0; i <= c->g.Nr; ++i)
        for (int j = 0; j <= c->g.Nth; ++j) {
            pm_t m;
            pm_eval(p->M, p->a, c->g.rn[i], c->g.tn[j], &m);
            double Dr = avg_r(c, D[0], 1, 0, i, j);
            double Bt = avg_r(c, B[1], 1, 0, i, j);
            E[2][i * ld + j] = m.alpha * (m.g_rp * Dr + m.g_pp * D[2][i * ld + j]) + m.sqrtg * m.beta * Bt;
        }
    theta_images(c, E);
}

/* H_i = alpha B_i - sqrtg eta_ijk beta^j D^k:
 *   H_r  (i, j+1/2)     = alpha (g_rr B^r + g_rp <B^ph>)
 *   H_th (i+1/2, j)     = alpha g_tt B^th + sqrtg beta <D^ph>
 *   H_ph (i+1/2, j+1/2) = alpha (g_rp <B^r> + g_pp B^ph) - sqrtg beta <D^th> */
static void make_H(const fctx *c, const double *const D[3], const double *const B[3], double *const H[3])
{
    const or_fdtd_params *p = c->p;
    int ld = c->g.ld;
    for (int i = 0; i <= c->g.Nr; ++i)
        for (int j = 0; j < c->g.Nth; ++j) {
            pm_t m;
            pm_eval(p->M, p->a, c->g.rn[i], c->g.th[j], &m);
            double Bp = avg_r(c, B[2], 1, 1, i, j);
            H[0][i * ld + j] = m.alpha * (m.g_rr * B[0][i * ld + j] + m.g_rp * Bp);
        }
    for (int i = 0; i < c->g.Nr; ++i)
        for (int j = 0; j <= c->g.Nth; ++j) {
            pm_t m;
            pm_eval(p->M, p->a, c->g.rh[i], c->g.tn[j], &m);
            double Dp = avg_r(c, D[2], 0, 0, i, j);
            H[1][i * ld + j] = m.alpha * m.g_tt * B[1][i * ld + j] + m.sqrtg * m.beta * Dp;
        }
    for (int i = 0; i < c->g.Nr; ++i)
        for (int j = 0; j < c->g.Nth; ++j) {
            pm_t m;
            pm_eval(p->M, p->a, c->g.rh[i], c->g.th[j], &m);
            double Br = avg_r(c, B[0], 0, 1, i, j);
            double Dt = avg_r(c, D[1], 0, 1, i, j);
            H[2][i * ld + j] = m.alpha * (m.g_rp * Br + m.g_pp * B[2][i * ld + j]) - m.sqrtg * m.beta * Dt;
        }
    theta_images(c, H);
}

/* Eq. (m4) with Eq. (abs0): B_out = (B_in - dt curl E / sqrtg) exp(-chi dt),
 *   (curl E)^r = d_th E_ph,  (curl E)^th = -d_r E_ph,  (curl E)^ph = d_r E_th - d_th E_r,
 * every component by its own two-point differences (no boundary rows). */
static void update_B(const fctx *c, const double *const Bin[3], const double *const E[3], double *const Bout[3])
{
    const or_fdtd_params *p = c->p;
    int ld = c->g.ld;
    for (int i = 0; i <= c->g.Nr; ++i)              /* B^r (i, j+1/2) */
        for (int j = 0; j < c->g.Nth; ++j) {
            double r = c->g.rn[i], t = c->g.th[j];
            double sg = sqrtg_at(p->M, p->a, r, t);
            double curl = (E[2][i * ld + j + 1] - E[2][i * ld + j]) / (c->g.tn[j + 1] - c->g.tn[j]);
            Bout[0][i * ld + j] = (Bin[0][i * ld + j] - p->dt * curl / sg) * damp(c, r);
        }
    for (int i = 0; i < c->g.Nr; ++i)               /* B^th (i+1/2, j) */
        for (int j = 0; j <= c->g.Nth; ++j) {
            double r = c->g.rh[i], t = c->g.tn[j];
            double sg = sqrtg_at(p->M, p->a, r, t);
            double curl = -(E[2][(i + 1) * ld + j] - E[2][i * ld + j]) / (c->g.rn[i + 1] - c->g.rn[i]);
            Bout[1][i * ld + j] = (Bin[1][i * ld + j] - p->dt * curl / sg) * damp(c, r);
        }
    for (int i = 0; i < c->g.Nr; ++i)               /* B^ph (i+1/2, j+1/2) */
        for (int j = 0; j < c->g.Nth; ++j) {
            double r = c->g.rh[i], t = c->g.th[j];
            double sg = sqrtg_at(p->M, p->a, r, t);
            double dEt = (E[1][(i + 1) * ld + j] - E[1][i * ld + j]) / (c->g.rn[i + 1] - c->g.rn[i]);
            double dEr = (E[0][i * ld + j + 1] - E[0][i * ld + j]) / (c->g.tn[j + 1] - c->g.tn[j]);
            Bout[2][i * ld + j] = (Bin[2][i * ld + j] - p->dt * (dEt - dEr) / sg) * damp(c, r);
        }
    theta_images(c, Bout);
}

/* Source J = alpha j - rho beta (Sec. 2.1, below Eq. m4) at the J^i points;
 * rho enters J^r through its metric-weighted average to (i+1/2, j). */
static double Jsrc(const fctx *c, int k, int i, int j, const double *const jv[3], const double *rho)
{
    const or_fdtd_params *p = c->p;
    pm_t m;
    int ld = c->g.ld;
    if (p->conserving) return jv[k][i * ld + j];   /* already J = alpha j - rho beta, per coordinate time */
    if (k == 0) {
        pm_eval(p->M, p->a, c->g.rh[i], c->g.tn[j], &m);
        double rb = avg_r(c, rho, 0, 0, i, j);
        return m.alpha * jv[0][i * ld + j] - rb * m.beta;
    }
    if (k == 1) {
        pm_eval(p->M, p->a, c->g.rn[i], c->g.th[j], &m);
        return m.alpha * jv[1][i * ld + j];
    }
    pm_eval(p->M, p->a, c->g.rn[i], c->g.tn[j], &m);
    return m.alpha * jv[2][i * ld + j];
}

/* Eq. (m3) with Eq. (abs1):
 *   D_out = (D_in + dt [curl H / sqrtg - 4 pi J]) exp(-chi dt),
 *   (curl H)^r = d_th H_ph,  (curl H)^th = -d_r H_ph,  (curl H)^ph = d_r H_th - d_th H_r,
 * J = w0 J(j0, rho0) + w1 J(j1, rho1).  Boundaries (Sec. 2.5, reading):
 * components without a two-sided stencil copy their neighbour (zero
 * gradient) -- D^th, D^ph at i = 0 and i = Nr, D^r at j = 0 and j = Nth --
 * and D^ph = 0 on the axis rows j = 0, Nth.  In the full-theta domain there
 * are no axis rows: D^r and D^ph at j = 0 take their th difference across
 * the seam (half node Nth-1, one period below), and column Nth is the image
 * of column 0. */
static void update_D(const fctx *c, const double *const Din[3], const double *const H[3],
                     const double *const j0[3], const double *rho0, double w0,
                     const double *const j1[3], const double *rho1, double w1, double *const Dout[3])
{
    const or_fdtd_params *p = c->p;
    int ld = c->g.ld, Nr = c->g.Nr, Nth = c->g.Nth, j_lo = p->full ? 0 : 1;
    for (int i = 0; i < Nr; ++i)                    /* D^r (i+1/2, j) */
        for (int j = j_lo; j < Nth; ++j) {
            double r = c->g.rh[i], t = c->g.tn[j];
            double sg = sqrtg_at(p->M, p->a, r, t);
            int jm = j > 0 ? j - 1 : Nth - 1;
            double dth = j > 0 ? c->g.th[j] - c->g.th[j - 1] : th_ext(c) - c->g.th[Nth - 1];
            double curl = (H[2][i * ld + j] - H[2][i * ld + jm]) / dth;
            double J = 0.0;
            if (w0 != 0.0) J += w0 * Jsrc(c, 0, i, j, j0, rho0);
            if (w1 != 0.0) J += w1 * Jsrc(c, 0, i, j, j1, rho1);
            Dout[0][i * ld + j] = (Din[0][i * ld + j] + p->dt * (curl / sg - 4.0 * M_PI * J)) * damp(c, r);
        }
    for (int i = 1; i < Nr; ++i)                    /* D^th (i, j+1/2) */
        for (int j = 0; j < Nth; ++j) {
            double r = c->g.rn[i], t = c->g.th[j];
            double sg = sqrtg_at(p->M, p->a, r, t);
            double curl = -(H[2][i * ld + j] - H[2][(i - 1) * ld + j]) / (c->g.rh[i] - c->g.rh[i - 1]);
            double J = 0.0;
            if (w0 != 0.0) J += w0 * Jsrc(c, 1, i, j, j0, rho0);
            if (w1 != 0.0) J += w1 * Jsrc(c, 1, i, j, j1, rho1);
            Dout[1][i * ld + j] = (Din[1][i * ld + j] + p->dt * (curl / sg - 4.0 * M_PI * J)) * damp(c, r);
        }
    for (int i = 1; i < Nr; ++i)                    /* D^ph (i, j) */
        for (int j = j_lo; j < Nth; ++j) {
            double r = c->g.rn[i], t = c->g.tn[j];
            double sg = sqrtg_at(p->M, p->a, r, t);
            int jm = j > 0 ? j - 1 : Nth - 1;
            double dth = j > 0 ? c->g.th[j] - c->g.th[j - 1] : th_ext(c) - c->g.th[Nth - 1];
            double dHt = (H[1][i * ld + j] - H[1][(i - 1) * ld + j]) / (c->g.rh[i] - c->g.rh[i - 1]);
            double dHr = (H[0][i * ld + j] - H[0][i * ld + jm]) / dth;
            double J = 0.0;
            if (w0 != 0.0) J += w0 * Jsrc(c, 2, i, j, j0, rho0);
            if (w1 != 0.0) J += w1 * Jsrc(c, 2, i, j, j1, rho1);
            Dout[2][i * ld + j] = (Din[2][i * ld + j] + p->dt * ((dHt - dHr) / sg - 4.0 * M_PI * J)) * damp(c, r);
        }
    /* boundaries */
    if (!p->full)
        for (int i = 0; i < Nr; ++i) {
            Dout[0][i * ld + 0] = Dout[0][i * ld + 1];
            Dout[0][i * ld + Nth] = Dout[0][i * ld + Nth - 1];
        }
    for (int j = 0; j < Nth; ++j) {
        Dout[1][0 * ld + j] = Dout[1][1 * ld + j];
        Dout[1][Nr * ld + j] = Dout[1][(Nr - 1) * ld + j];
    }
    for (int j = j_lo; j < Nth; ++j) {
        Dout[2][0 * ld + j] = Dout[2][1 * ld + j];
        Dout[2][Nr * ld + j] = Dout[2][(Nr - 1) * ld + j];
    }
    if (!p->full)
        for (int i = 0; i <= Nr; ++i) {
            Dout[2][i * ld + 0] = 0.0;
            Dout[2][i * ld + Nth] = 0.0;
        }
    theta_images(c, Dout);
}

/* The ten sub-steps of Sec. 2.1, split around the particle push:
 *   stage 1:  E <- alpha <D> + beta x B1           (<D> = (D0 + D1)/2)     [1]
 *             Bh <- (B0 + B1)/2 - dt curl E          -> B^{n+3/2}         [2]
 *             E <- alpha D1 + beta x Bh                                   [3]
 *             B0 <- B1 - dt curl E                   -> B^{n+2}            [4]
 *   (push with D1, Bh; deposit j1, rho1)                                [5,6]
 *   stage 2:  H <- alpha Bh - beta x D1                                   [7]
 *             Dw <- <D> + dt [curl H - 4 pi (J0 + J1)/2] -> D^{n+2}       [8]
 *             H <- alpha B0 - beta x Dw                                   [9]
 *             D0 <- D1 + dt [curl H - 4 pi J1]       -> D^{n+5/2}         [10]
 * On entry B0 = B^n, B1 = B^{n+1}, D0 = D^{n+1/2}, D1 = D^{n+3/2}, (j0, rho0)
 * at n+1 and (j1, rho1) at n+2.  After stage 2 the caller swaps B0/B1,
 * D0/D1 and (j0,rho0)/(j1,rho1) for the next step.  E, H, Bh, Dw are work
 * arrays (3 each).  Every array is (Nr+1) * ld. */
void or_fdtd(const or_fdtd_params *p, int Nr, int Nth, int ld, const double *rn, const double *rh,
             const double *tn, const double *th, int stage, double *const B0[3], double *const B1[3],
             double *const D0[3], double *const D1[3], double *const j0[3], double *rho0,
             double *const j1[3], double *rho1, double *const E[3], double *const H[3],
             double *const Bh[3], double *const Dw[3])
{
    fctx c = {p, {Nr, Nth, ld, rn, rh, tn, th}};
    size_t sz = (size_t)(Nr + 1) * ld;
    double *avg[3];
    for (int k = 0; k < 3; ++k) avg[k] = (double *)malloc(sz * sizeof(double));
    if (stage == 1) {
        for (int k = 0; k < 3; ++k)
            for (size_t q = 0; q < sz; ++q) avg[k][q] = 0.5 * (D0[k][q] + D1[k][q]);
        make_E(&c, (const double *const *)avg, (const double *const *)B1, E);
        for (int k = 0; k < 3; ++k)
            for (size_t q = 0; q < sz; ++q) avg[k][q] = 0.5 * (B0[k][q] + B1[k][q]);
        update_B(&c, (const double *const *)avg, (const double *const *)E, Bh);
        make_E(&c, (const double *const *)D1, (const double *const *)Bh, E);
        update_B(&c, (const double *const *)B1, (const double *const *)E, B0);
    } else {
        make_H(&c, (const double *const *)D1, (const double *const *)Bh, H);
        for (int k = 0; k < 3; ++k)
            for (size_t q = 0; q < sz; ++q) avg[k][q] = 0.5 * (D0[k][q] + D1[k][q]);
        update_D(&c, (const double *const *)avg, (const double *const *)H, (const double *const *)j0, rho0,
                 0.5, (const double *const *)j1, rho1, 0.5, Dw);
        make_H(&c, (const double *const *)Dw, (const double *const *)B0, H);
        update_D(&c, (const double *const *)D1, (const double *const *)H, (const double *const *)j0, rho0,
                 0.0, (const double *const *)j1, rho1, 1.0, D0);
    }
    for (int k = 0; k < 3; ++k) free(avg[k]);
}

/* Discrete divergences (tests): div B at cell centres (i+1/2, j+1/2) and
 * div D at interior integer nodes, both as sqrtg-weighted two-point
 * differences (the Yee forms of Eqs. m1-m2), times sqrtg at the point. */
void or_div(double M, double a, int Nr, int Nth, int ld, const double *rn, const double *rh,
            const double *tn, const double *th, const double *const B[3], const double *const D[3],
            double *divB, double *divD, int full)
{
    for (int i = 0; i < Nr; ++i)
        for (int j = 0; j < Nth; ++j) {
            double fr1 = sqrtg_at(M, a, rn[i + 1], th[j]) * B[0][(i + 1) * ld + j];
            double fr0 = sqrtg_at(M, a, rn[i], th[j]) * B[0][i * ld + j];
            double ft1 = sqrtg_at(M, a, rh[i], tn[j + 1]) * B[1][i * ld + j + 1];
            double ft0 = sqrtg_at(M, a, rh[i], tn[j]) * B[1][i * ld + j];
            divB[i * ld + j] = (fr1 - fr0) / (rn[i + 1] - rn[i]) + (ft1 - ft0) / (tn[j + 1] - tn[j]);
        }
    /* full-theta domain: div D at j = 0 too, across the seam (half node
     * Nth-1 one period below; spacing th[0] + P - th[Nth-1]) */
    for (int i = 1; i < Nr; ++i)
        for (int j = full ? 0 : 1; j < Nth; ++j) {
            int jm = j > 0 ? j - 1 : Nth - 1;
            double dth = j > 0 ? th[j] - th[j - 1] : (th[0] + (tn[Nth] - tn[0])) - th[Nth - 1];
            double fr1 = sqrtg_at(M, a, rh[i], tn[j]) * D[0][i * ld + j];
            double fr0 = sqrtg_at(M, a, rh[i - 1], tn[j]) * D[0][(i - 1) * ld + j];
            double ft1 = sqrtg_at(M, a, rn[i], th[j]) * D[1][i * ld + j];
            double ft0 = sqrtg_at(M, a, rn[i], th[jm]) * D[1][i * ld + jm];
            divD[i * ld + j] = (fr1 - fr0) / (rh[i] - rh[i - 1]) + (ft1 - ft0) / dth;
        }
}

/* Split-monopole initial field (Sec. 3.4; App. B.2): B^r = d_th Psi / sqrtg
 * with the flux function Psi = 4 M^2 B0 zeta(th) (1 - cos th) and the
 * smoothed equatorial step zeta = (2/pi) arctan[zeta0 (th - pi/2)], at the
 * B^r Yee points (r_i, th_{j+1/2}); every other component is zero (the
 * paper starts from this vacuum field).
 *   d_th Psi = 4 M^2 B0 [zeta'(th) (1 - cos th) + zeta(th) sin th],
 *   zeta' = (2/pi) zeta0 / (1 + zeta0^2 (th - pi/2)^2).
 * F[0..5] = D^r, D^th, D^ph, B^r, B^th, B^ph (size (Nr + 1) ld each). */
void or_split_monopole_on_grid(double M, double a, double B0, double zeta0, int Nr, int Nth, int ld,
                               const double *rn, const double *rh, const double *tn, const double *th,
                               double *const F[6])
{
    (void)rh;
    (void)tn;
    const size_t sz = (size_t)(Nr + 1) * ld;
    for (int k = 0; k < 6; ++k)
        for (size_t o = 0; o < sz; ++o) F[k][o] = 0.0;
    for (int i = 0; i <= Nr; ++i)
        for (int j = 0; j < Nth; ++j) {
            const double t = th[j], x = t - M_PI / 2.0;
            const double zeta = 2.0 / M_PI * atan(zeta0 * x);
            const double dzeta = 2.0 / M_PI * zeta0 / (1.0 + zeta0 * zeta0 * x * x);
            const double dpsi = 4.0 * M * M * B0 * (dzeta * (1.0 - cos(t)) + zeta * sin(t));
            F[3][i * ld + j] = dpsi / sqrtg_at(M, a, rn[i], t);
        }
}

/* Eq. (Pbz): P_BZ = 2 pi int S^r sqrtg dth with S^r = (E_th H_ph - E_ph
 * H_th) / (4 pi sqrtg), i.e. (1/2) int (E_th H_ph - E_ph H_th) dth, on the
 * sphere r = rh[i] (half-r index i).  Each product is formed at the cell
 * centres (rh[i], th_{j+1/2}): H_ph lives there; E_th (i, j+1/2) and
 * (i+1, j+1/2) are averaged in r; H_th (i+1/2, j), (i+1/2, j+1) in th; E_ph
 * at the four surrounding nodes.  Midpoint rule over the th cells. */
double or_bz_power(int Nr, int Nth, int ld, const double *tn, const double *const E[3],
                   const double *const H[3], int i)
{
    double P = 0.0;
    if (i < 0 || i >= Nr) return 0.0;
    for (int j = 0; j < Nth; ++j) {
        const double Eth = 0.5 * (E[1][i * ld + j] + E[1][(i + 1) * ld + j]);
        const double Hph = H[2][i * ld + j];
        const double Eph = 0.25 * (E[2][i * ld + j] + E[2][i * ld + j + 1] + E[2][(i + 1) * ld + j] +
                                   E[2][(i + 1) * ld + j + 1]);
        const double Hth = 0.5 * (H[1][i * ld + j] + H[1][i * ld + j + 1]);
        P += (Eth * Hph - Eph * Hth) * (tn[j + 1] - tn[j]);
    }
    return 0.5 * P;
}

/* Divergence cleaning (Sec. 2.4, Eq. phi).  Solve
 *   (1/sqrtg) d_k (sqrtg gamma^kl d_l phi) = (1/sqrtg) d_j (sqrtg D^j) - 4 pi rho
 * at the integer nodes (rn[i], tn[j]), i = 1 .. Nr-1, j = 0 .. Nth, by
 * n_iter Jacobi sweeps from phi = 0, then correct D^i -= gamma^ij d_j phi.
 * Discretisation: d_r phi at the D^r points (i+1/2, j), d_th phi at the D^th
 * points (i, j+1/2); both sides are multiplied by sqrtg at the node, so the
 * left side is the sum over the four faces of (sqrtg gamma^kk d_k phi)
 * differences over the dual widths rh[i] - rh[i-1] and th[j] - th[j-1] —
 * the same fluxes as the Yee divergence of D, so at convergence the
 * corrected field satisfies the discrete Gauss law exactly.  Boundaries:
 * phi = 0 on the radial end rows; the faces at the poles (th = 0, pi) carry
 * no flux (sqrtg = 0 there), the end dual widths reaching the pole.
 * (d_ph = 0; gamma^{r th} = 0.)  The correction of D^ph uses gamma^{ph r}
 * times d_r phi at the node, the mean of the two adjacent half-point
 * derivatives (one-sided on the end rows).  phi_out: nullable, size
 * (Nr + 1) ld. */
void or_div_clean(double M, double a, int Nr, int Nth, int ld, const double *rn, const double *rh,
                  const double *tn, const double *th, double *const D[3], const double *rho, int n_iter,
                  double *phi_out)
{
    const size_t sz = (size_t)(Nr + 1) * ld;
    double *phi = calloc(sz, sizeof(double)), *nxt = calloc(sz, sizeof(double));
    double *rhs = calloc(sz, sizeof(double));
    double *c_r1 = calloc(sz, sizeof(double)), *c_r0 = calloc(sz, sizeof(double));
    double *c_t1 = calloc(sz, sizeof(double)), *c_t0 = calloc(sz, sizeof(double));
    pm_t m;
    for (int i = 1; i < Nr; ++i)
        for (int j = 0; j <= Nth; ++j) {
            const size_t o = (size_t)i * ld + j;
            const double dr = rh[i] - rh[i - 1];
            const double dth = (j < Nth ? th[j] : M_PI) - (j > 0 ? th[j - 1] : 0.0);
            /* right side: sqrtg-weighted divergence of D minus 4 pi sqrtg rho */
            const double fr1 = sqrtg_at(M, a, rh[i], tn[j]) * D[0][o];
            const double fr0 = sqrtg_at(M, a, rh[i - 1], tn[j]) * D[0][o - ld];
            const double ft1 = j < Nth ? sqrtg_at(M, a, rn[i], th[j]) * D[1][o] : 0.0;
            const double ft0 = j > 0 ? sqrtg_at(M, a, rn[i], th[j - 1]) * D[1][o - 1] : 0.0;
            rhs[o] = (fr1 - fr0) / dr + (ft1 - ft0) / dth - 4.0 * M_PI * sqrtg_at(M, a, rn[i], tn[j]) * rho[o];
            /* face coefficients sqrtg gamma^kk / (spacing x dual width) */
            pm_eval(M, a, rh[i], tn[j], &m);
            c_r1[o] = m.sqrtg * m.gu_rr / ((rn[i + 1] - rn[i]) * dr);
            pm_eval(M, a, rh[i - 1], tn[j], &m);
            c_r0[o] = m.sqrtg * m.gu_rr / ((rn[i] - rn[i - 1]) * dr);
            if (j < Nth) {
                pm_eval(M, a, rn[i], th[j], &m);
                c_t1[o] = m.sqrtg * m.gu_tt / ((tn[j + 1] - tn[j]) * dth);
            }
            if (j > 0) {
                pm_eval(M, a, rn[i], th[j - 1], &m);
                c_t0[o] = m.sqrtg * m.gu_tt / ((tn[j] - tn[j - 1]) * dth);
            }
        }
    for (int it = 0; it < n_iter; ++it) {
        for (int i = 1; i < Nr; ++i)
            for (int j = 0; j <= Nth; ++j) {
                const size_t o = (size_t)i * ld + j;
                double s = c_r1[o] * phi[o + ld] + c_r0[o] * phi[o - ld];
                if (j < Nth) s += c_t1[o] * phi[o + 1];
                if (j > 0) s += c_t0[o] * phi[o - 1];
                nxt[o] = (s - rhs[o]) / (c_r1[o] + c_r0[o] + c_t1[o] + c_t0[o]);
            }
        double *t = phi;
        phi = nxt;
        nxt = t;
    }
    /* D^i -= gamma^ij d_j phi */
    for (int i = 0; i < Nr; ++i)
        for (int j = 0; j <= Nth; ++j) {
            pm_eval(M, a, rh[i], tn[j], &m);
            D[0][(size_t)i * ld + j] -= m.gu_rr * (phi[(size_t)(i + 1) * ld + j] - phi[(size_t)i * ld + j]) /
                                        (rn[i + 1] - rn[i]);
        }
    for (int i = 0; i <= Nr; ++i)
        for (int j = 0; j < Nth; ++j) {
            pm_eval(M, a, rn[i], th[j], &m);
            D[1][(size_t)i * ld + j] -= m.gu_tt * (phi[(size_t)i * ld + j + 1] - phi[(size_t)i * ld + j]) /
                                        (tn[j + 1] - tn[j]);
        }
    for (int i = 0; i <= Nr; ++i)
        for (int j = 0; j <= Nth; ++j) {
            double dr_up = 0.0, dr_dn = 0.0;
            int k = 0;
            if (i < Nr) { dr_up = (phi[(size_t)(i + 1) * ld + j] - phi[(size_t)i * ld + j]) / (rn[i + 1] - rn[i]); ++k; }
            if (i > 0) { dr_dn = (phi[(size_t)i * ld + j] - phi[(size_t)(i - 1) * ld + j]) / (rn[i] - rn[i - 1]); ++k; }
            pm_eval(M, a, rn[i], tn[j], &m);
            D[2][(size_t)i * ld + j] -= m.gu_rp * (dr_up + dr_dn) / k;
        }
    if (phi_out) memcpy(phi_out, phi, sz * sizeof(double));
    free(phi); free(nxt); free(rhs); free(c_r1); free(c_r0); free(c_t1); free(c_t0);
}

/* ------------------------------------------------------------------------ */
/* Pair injection (Sec. 3.3 and Sec. 3.4).                                   */
/* ------------------------------------------------------------------------ */

/* In every cell whose centre radius rh[i] lies in [r_lo, r_hi], an e-/e+
 * pair is added when the plasma density is below the multiplicity times
 * the Goldreich-Julian density, n < mult n_GJ, n_GJ = |Omega . B| / (4 pi e)
 * with Omega the horizon's angular velocity a / (2 M r_h) along the spin
 * axis.  Readings (the paper is silent on them):
 *   - densities are charge-number densities: e n = sum of w |q/m| over the
 *     cell's alive particles (in particle-index order) / V, V = 2 pi x the
 *     4 x 4 trapezoid of sqrt(gamma) over the cell (the Sec. 2.3 volume);
 *   - Omega . B = Omega (B^r cos th - r sin th B^th) at the cell centre,
 *     B^r averaged over the cell's two r faces, B^th over its two th faces
 *     (the flat-space z component of B with the coordinate r, th);
 *   - the pair is placed at one point, drawn uniformly in the cell's
 *     coordinate box, ph uniform in [0, 2 pi), each particle with its own
 *     FIDO-frame momentum (Maxwell-Juttner draws supplied by the caller),
 *     mapped to u_i as in the FIDO seeding (gamma = L L^T);
 *   - both particles get the weight that makes the pair's density n0 n_GJ
 *     (the "effective density" conferred by one injection), w |q/m| / V =
 *     n0 e n_GJ / 2;
 *   - pairs are appended in cell order (c = i Nth + j), e- then e+, while
 *     they fit in the capacity.
 * draws: 9 numbers per cell c (u_r, u_th, u_ph uniform in [0,1), e- FIDO
 * momentum, e+ FIDO momentum).  z (cap x 6), qm, w, alive hold n particles.
 * flags (nullable, Nr Nth bytes) receives the decisions.  Returns the
 * number of pairs wanted; *n_out = the new particle count. */
int64_t or_inject_pairs(double M, double a, int Nr, int Nth, int ld, const double *rn, const double *rh,
                        const double *tn, const double *th, const double *Br, const double *Bth, double r_lo,
                        double r_hi, double mult, double n0, double qm_e, const double *draws, int64_t n,
                        int64_t cap, double *z, double *qm, double *w, uint8_t *alive, uint8_t *flags,
                        int64_t *n_out)
{
    const int64_t C = (int64_t)Nr * Nth;
    double *S = calloc((size_t)C, sizeof(double));
    for (int64_t p = 0; p < n; ++p) {
        if (!alive[p]) continue;
        int i = loc(rn, Nr + 1, z[6 * p]), j = loc(tn, Nth + 1, z[6 * p + 1]);
        S[(int64_t)i * Nth + j] += w[p] * fabs(qm[p]);
    }
    const double r_h = M + sqrt(M * M - a * a);
    const double Om = a / (2.0 * M * r_h);
    int64_t K = 0, m = n;
    for (int i = 0; i < Nr; ++i)
        for (int j = 0; j < Nth; ++j) {
            const int64_t c = (int64_t)i * Nth + j;
            int inj = 0;
            double V = 0.0, gj = 0.0;
            if (rh[i] >= r_lo && rh[i] <= r_hi) {
                V = 2.0 * M_PI * trap16(M, a, rn[i], rn[i + 1], tn[j], tn[j + 1], 0);
                double br = 0.5 * (Br[(size_t)i * ld + j] + Br[(size_t)(i + 1) * ld + j]);
                double bt = 0.5 * (Bth[(size_t)i * ld + j] + Bth[(size_t)i * ld + j + 1]);
                double Bz = br * cos(th[j]) - rh[i] * sin(th[j]) * bt;
                gj = fabs(Om * Bz) / (4.0 * M_PI);
                inj = S[c] / V < mult * gj;
            }
            if (flags) flags[c] = (uint8_t)inj;
            if (!inj) continue;
            ++K;
            if (m + 2 > cap) continue;
            const double *d = draws + 9 * c;
            const double r = rn[i] + d[0] * (rn[i + 1] - rn[i]);
            const double t = tn[j] + d[1] * (tn[j + 1] - tn[j]);
            const double ph = 2.0 * M_PI * d[2];
            pm_t g;
            pm_eval(M, a, r, t, &g);
            const double L11 = sqrt(g.g_rr), L31 = g.g_rp / L11, L22 = sqrt(g.g_tt);
            const double L33 = sqrt(g.g_pp - L31 * L31);
            const double wp = n0 * gj * V / (2.0 * qm_e);
            for (int s = 0; s < 2; ++s) {
                const double *u = d + 3 + 3 * s;
                double *o = z + 6 * m;
                o[0] = r; o[1] = t; o[2] = ph;
                o[3] = L11 * u[0];
                o[4] = L22 * u[1];
                o[5] = L31 * u[0] + L33 * u[2];
                qm[m] = s == 0 ? -qm_e : qm_e;
                w[m] = wp;
                alive[m] = 1;
                ++m;
            }
        }
    free(S);
    *n_out = m;
    return K;
}


/* ------------------------------------------------------------------------ */
/* Charge-conserving deposit (an extension: the paper's deposit is not, and  */
/* relies on the cleaning of Sec. 2.4).                                      */
/* ------------------------------------------------------------------------ */

/* Yee dual widths of integer node i (r) and j (th): the spans between the
 * neighbouring half nodes, reaching the grid ends / the poles. */
static double ydual_r(const pg_t *g, int i)
{
    double lo = i == 0 ? g->rn[0] : g->rh[i - 1], hi = i == g->Nr ? g->rn[g->Nr] : g->rh[i];
    return hi - lo;
}

static double ydual_t(const pg_t *g, int j)
{
    double lo = j == 0 ? 0.0 : g->th[j - 1], hi = j == g->Nth ? M_PI : g->th[j];
    return hi - lo;
}

/* A particle's move from x^n to x^{n+1} deposited so that charge is
 * conserved node by node (Esirkepov's construction, which needs node weights
 * that are a product S(r, th) = S_r(r) S_th(th); the volume weights of
 * Sec. 2.3 are not, so the variant takes the linear (area) weights in r and
 * in th between the integer nodes).  With a = old, b = new:
 *   W_r (i, j) = (S_r^b(i) - S_r^a(i)) (S_th^a(j) + S_th^b(j)) / 2,
 *   W_th(i, j) = (S_r^a(i) + S_r^b(i)) (S_th^b(j) - S_th^a(j)) / 2,
 *   W_r + W_th = S^b - S^a,  sum_i W_r(i, j) = 0 = sum_j W_th(i, j),
 * on the union of the two stencils (3 x 3 for a move of at most one cell);
 * the charge crossing the dual face between nodes (i, j) and (i+1, j) in +r
 * is -Q sum_{i' <= i} W_r(i', j) (and alike in th).  Outputs, zeroed first:
 *   rho  (i, j)       = Q S^b / (2 pi sqrtg dr_dual dth_dual)  (the Yee cell of the node)
 *   J^r  (i+1/2, j)   = flux / (dt 2 pi sqrtg dth_dual)
 *   J^th (i, j+1/2)   = flux / (dt 2 pi sqrtg dr_dual)
 *   J^ph (i, j)       = Q (S^a + S^b)/2 (dph/dt)_mid / (2 pi sqrtg dr_dual dth_dual),
 *     (dph/dt)_mid the mean of alpha gamma^{ph j} u_j / Gamma at both states,
 * the J being coordinate currents (alpha j - rho beta), which the FDTD takes
 * as they are in its conserving mode.  Then
 *   sqrtg (rho^{n+1} - rho^n) + dt Yee-div(sqrtg J) = 0
 * at every node to rounding, so Ampere's law (sub-step 10) keeps
 * Yee-div(sqrtg D) - 4 pi sqrtg rho unchanged.  alive: particles alive
 * before the move (their new state is deposited even if it left the
 * domain; positions are clamped into the node range).  Returns the number
 * of moves longer than one cell (skipped). */
static void lin_weights(const double *X, int m, double x, int *i, double wgt[2])
{
    if (x < X[0]) x = X[0];
    if (x > X[m - 1]) x = X[m - 1];
    int k = loc(X, m, x);
    double f = (x - X[k]) / (X[k + 1] - X[k]);
    *i = k;
    wgt[0] = 1.0 - f;
    wgt[1] = f;
}

int64_t or_deposit_conserving(double M, double a, int Nr, int Nth, int ld, const double *rn, const double *rh,
                              const double *tn, const double *th, int64_t n, const double *z0,
                              const double *z1, const double *qm, const double *w, const uint8_t *alive,
                              double dt, double *rho, double *Jr, double *Jt, double *Jp)
{
    pg_t g = {Nr, Nth, ld, rn, rh, tn, th};
    size_t sz = (size_t)(Nr + 1) * ld;
    memset(rho, 0, sz * sizeof(double));
    memset(Jr, 0, sz * sizeof(double));
    memset(Jt, 0, sz * sizeof(double));
    memset(Jp, 0, sz * sizeof(double));
    double *Ir = calloc(sz, sizeof(double)), *It = calloc(sz, sizeof(double));
    double *Qn = calloc(sz, sizeof(double)), *Pn = calloc(sz, sizeof(double));
    int64_t skipped = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (!alive[p]) continue;
        const double *a0 = z0 + 6 * p, *a1 = z1 + 6 * p;
        const double Q = w[p] * qm[p];
        int ia, ib, ja, jb;
        double ra[2], rb[2], ta[2], tb[2];
        lin_weights(rn, Nr + 1, a0[0], &ia, ra);
        lin_weights(rn, Nr + 1, a1[0], &ib, rb);
        lin_weights(tn, Nth + 1, a0[1], &ja, ta);
        lin_weights(tn, Nth + 1, a1[1], &jb, tb);
        int i0 = ia < ib ? ia : ib, j0 = ja < jb ? ja : jb;
        if (abs(ia - ib) > 1 || abs(ja - jb) > 1) { ++skipped; continue; }
        double Sra[3] = {0, 0, 0}, Srb[3] = {0, 0, 0}, Sta[3] = {0, 0, 0}, Stb[3] = {0, 0, 0};
        for (int c = 0; c < 2; ++c) {
            Sra[ia - i0 + c] = ra[c];
            Srb[ib - i0 + c] = rb[c];
            Sta[ja - j0 + c] = ta[c];
            Stb[jb - j0 + c] = tb[c];
        }
        double Wn[2][2][3][3], Wr[3][3], Wt[3][3];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                Wn[0][0][x][y] = Sra[x] * Sta[y];
                Wn[1][1][x][y] = Srb[x] * Stb[y];
                Wr[x][y] = 0.5 * (Srb[x] - Sra[x]) * (Sta[y] + Stb[y]);
                Wt[x][y] = 0.5 * (Sra[x] + Srb[x]) * (Stb[y] - Sta[y]);
            }
        /* fluxes through the faces inside the window */
        for (int y = 0; y < 3; ++y) {
            double acc = 0.0;
            for (int x = 0; x < 2; ++x) {
                acc += Wr[x][y];
                int gi = i0 + x, gj = j0 + y;
                if (gi < Nr && gj <= Nth) Ir[(size_t)gi * ld + gj] += -Q * acc;
            }
        }
        for (int x = 0; x < 3; ++x) {
            double acc = 0.0;
            for (int y = 0; y < 2; ++y) {
                acc += Wt[x][y];
                int gi = i0 + x, gj = j0 + y;
                if (gi <= Nr && gj < Nth) It[(size_t)gi * ld + gj] += -Q * acc;
            }
        }
        /* coordinate dph/dt at both states */
        double phd = 0.0;
        for (int k = 0; k < 2; ++k) {
            const double *s_ = k ? a1 : a0;
            pm_t m;
            pm_eval(M, a, s_[0], s_[1], &m);
            double G = sqrt(1.0 + m.gu_rr * s_[3] * s_[3] + 2.0 * m.gu_rp * s_[3] * s_[5]
                            + m.gu_tt * s_[4] * s_[4] + m.gu_pp * s_[5] * s_[5]);
            phd += 0.5 * m.alpha * (m.gu_rp * s_[3] + m.gu_pp * s_[5]) / G;
        }
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                int gi = i0 + x, gj = j0 + y;
                if (gi > Nr || gj > Nth) continue;
                Qn[(size_t)gi * ld + gj] += Q * Wn[1][1][x][y];
                Pn[(size_t)gi * ld + gj] += Q * 0.5 * (Wn[0][0][x][y] + Wn[1][1][x][y]) * phd;
            }
    }
    for (int i = 0; i <= Nr; ++i)
        for (int j = 0; j <= Nth; ++j) {
            size_t o = (size_t)i * ld + j;
            double vol = 2.0 * M_PI * sqrtg_at(M, a, rn[i], tn[j]) * ydual_r(&g, i) * ydual_t(&g, j);
            rho[o] = vol > 0.0 ? Qn[o] / vol : 0.0;
            Jp[o] = vol > 0.0 ? Pn[o] / vol : 0.0;
            if (i < Nr) {
                double d = 2.0 * M_PI * sqrtg_at(M, a, rh[i], tn[j]) * ydual_t(&g, j) * dt;
                Jr[o] = d != 0.0 ? Ir[o] / d : 0.0;
            }
            if (j < Nth) {
                double d = 2.0 * M_PI * sqrtg_at(M, a, rn[i], th[j]) * ydual_r(&g, i) * dt;
                Jt[o] = d != 0.0 ? It[o] / d : 0.0;
            }
        }
    free(Ir); free(It); free(Qn); free(Pn);
    return skipped;
}
