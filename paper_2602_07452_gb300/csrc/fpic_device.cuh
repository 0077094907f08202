// Device-side building blocks of the GRPIC push: closed-form Kerr-Schild
// metric and derivatives (Appendix A), the equations of motion (Eqs. p1, p2,
// O1, O2), the Hamiltonian (Eq. Ham) and the staggered-grid field gather.
//
// GB300 note: FP64 issues at a small fraction of the FP32 rate, so these
// helpers are written to minimise FP64-pipe instructions: one sincos, one
// reciprocal and two reciprocal square roots per evaluation, fused
// multiply-adds throughout, and cell location by integer comparison of the
// IEEE bit patterns (order-preserving) instead of FP64 compares.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fpic {

struct BH {
    double M, a, a2, twoM;
};

// 1/x from the hardware approximation y refined by one third-order step:
// with e = 1 - x y, 1/x = y / (1 - e) = y (1 + e + e^2 + ...), so
// y (1 + e + e^2) triples the correct bits of the estimate (its relative
// error e^3); fpic_probe_math measures the result against correctly
// rounded reciprocals.
__device__ __forceinline__ double rcp_nr(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for a positive normal x from the hardware estimate y: with
// e = 1 - x y^2 (one rounded product, then a fused multiply-add),
// 1/sqrt(x) = y (1 - e)^(-1/2) = y (1 + e/2 + 3 e^2/8 + ...), taken to
// second order; the omitted terms are of order e^3, far below double
// rounding for the estimate's error, so the result is within about an ulp
// (fpic_probe_math measures it against an extended-precision reference).
// Five FP64 operations and no special-case branches: the push only takes
// it of xi = 1 + 2 M r / rho^2 and Gamma^2, both at least 1.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x * y, y, 1.0);
    return fma(y * e, fma(e, 0.375, 0.5), y);
}

// Square root of a positive normal x (the deposit's trapezoid sums): the
// hardware reciprocal-square-root estimate y refined by one coupled Newton
// step on (g, h) = (x y, y / 2) (Goldschmidt's iteration, e.g. Markstein,
// IA-64 and Elementary Functions, 2000): g (1 + r), r = 1/2 - g h, squares
// the estimate's relative error; fpic_probe_math measures at most 1.3e-12
// (2^-39.6) against correctly rounded square roots, far inside the deposit's
// 1e-10 bound.  Each particle's shares still sum to its charge to rounding:
// they are ratios of the same subvolumes.
// sqrt2_dep returns 2 sqrt(x) in the same step written as g (3 - g y) with
// g = x y: three FP64 operations after the estimate; the deposit only uses
// ratios of sums of these values, so the factor 2 cancels.
__device__ __forceinline__ double sqrt2_dep(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double g = x * y;
    return g * fma(-g, y, 3.0);
}

__device__ __forceinline__ double sqrt_dep(double x)
{
    return 0.5 * sqrt2_dep(x);
}

// sin h and cos h - 1 for a step h inside one cell: Maclaurin series through
// h^5 / h^6 when |h| < 2^-10 (the first omitted terms are below 2^-62 of
// sin h and 2^-63 of cos h - 1), through h^7 / h^8 when |h| < 2^-7 (below
// 1e-22 relative), else libm.
// |x| < 2^e for a power of two 2^e whose double has high word hi_pow2 (and
// low word 0): the same result as the FP64 compare (false for a NaN), from
// the high word by one integer compare, off the FP64 pipe.
__device__ __forceinline__ bool abs_below_pow2(double x, unsigned hi_pow2)
{
    return ((unsigned)__double2hiint(x) & 0x7fffffffu) < hi_pow2;
}
constexpr unsigned HI_2M10 = 0x3f500000u, HI_2M7 = 0x3f800000u;   // 2^-10, 2^-7

__device__ __forceinline__ void sincos_step(double h, double& sh, double& cm)
{
    if (abs_below_pow2(h, HI_2M10)) {
        const double h2 = h * h;
        sh = h * fma(h2, fma(h2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
        cm = h2 * fma(h2, fma(h2, -1.0 / 720.0, 1.0 / 24.0), -0.5);
    } else if (abs_below_pow2(h, HI_2M7)) {
        const double h2 = h * h;
        sh = h * fma(h2, fma(h2, fma(h2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), 1.0);
        cm = h2 * fma(h2, fma(h2, fma(h2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5);
    } else {
        double s, c;
        sincos(h, &s, &c);
        sh = s;
        cm = c - 1.0;
    }
}

// sin and cos of t from those of a nearby t0 by the angle-addition formula,
// with sin d and cos d - 1 of d = t - t0 by their Taylor series (the first
// omitted terms are below 1e-23 for |d| < 2^-7); farther away, sincos.
__device__ __forceinline__ void sincos_near(double t0, double s0, double c0, double t, double& s, double& c)
{
    const double d = t - t0;
    if (abs_below_pow2(d, HI_2M7)) {
        double sd, cm;
        sincos_step(d, sd, cm);
        s = fma(s0, cm, fma(c0, sd, s0));
        c = fma(c0, cm, fma(-s0, sd, c0));
    } else {
        sincos(t, &s, &c);
    }
}

// Metric at a point (r, th) given sin/cos th.
struct Geo {
    double s, c, s2, c2, r2, rho2, irho2, t;  // t = 1/(rho^2 sin^2 th)
    double twoMr, a2s2;               // 2 M r, a^2 sin^2 th
    double xi, alpha, ixi, beta;
    double gurr, gurp, gutt, gupp;
    double grr, grp, gtt, gpp, sqrtg;
};

// With xi = 1 + 2 M r / rho^2: alpha = xi^(-1/2), beta^r = 2 M r / (rho^2 xi)
// = 1 - 1/xi, g^rr = a^2 s^2 / rho^2 + 1/xi, g^rp = a / rho^2,
// g^tt = 1 / rho^2, g^pp = 1 / (rho^2 s^2) (App. A).
__device__ __forceinline__ void geo_eval(const BH& bh, double r, double s, double c, Geo& g)
{
    const double s2 = s * s, c2 = c * c;
    g.s = s;
    g.c = c;
    g.s2 = s2;
    g.c2 = c2;
    g.r2 = r * r;
    g.rho2 = fma(bh.a2, c2, g.r2);
    g.t = rcp_nr(g.rho2 * s2);
    g.irho2 = g.t * s2;
    g.twoMr = bh.twoM * r;
    g.a2s2 = bh.a2 * s2;
    g.xi = fma(g.twoMr, g.irho2, 1.0);
    g.alpha = rsqrt_nr(g.xi);
    g.ixi = g.alpha * g.alpha;
    g.beta = 1.0 - g.ixi;
    g.gurr = fma(g.a2s2, g.irho2, g.ixi);
    g.gurp = bh.a * g.irho2;
    g.gutt = g.irho2;
    g.gupp = g.t;
    g.grr = g.xi;
    g.grp = -bh.a * g.xi * s2;
    g.gtt = g.rho2;
    g.gpp = s2 * fma(bh.a2 * g.xi, s2, g.rho2);
    g.sqrtg = g.rho2 * g.xi * g.alpha * s;
}

// d_r and d_th of the three functions the momentum equations need: xi,
// g^tt = 1/rho^2 (g^rp = a g^tt, and g^rr, alpha, beta^r follow from xi and
// g^tt, see eval_rhs_sc) and g^pp; plus q = 2 a^2 sin cos = -d_th rho^2.
struct GeoD {
    double xi[2], tt[2], pp[2];
    double q;
};

// With P = rho^2 (d_r P = 2 r, d_th P = -q) and u = 1/P^2: d g^tt = -dP u,
// d_r xi = 2M (P - 2 r^2) u, d_th xi = 2 M r q u, d_r g^pp = -2 r t / P,
// d_th g^pp = -2 s c t^2 (P - a^2 s^2)  (t = g^pp = 1 / (P s^2)).
__device__ __forceinline__ void geo_deriv(const BH& bh, double r, const Geo& g, GeoD& d)
{
    const double sc = g.s * g.c;
    d.q = 2.0 * bh.a2 * sc;
    const double u = g.irho2 * g.irho2;
    const double mr2 = -2.0 * r;
    d.tt[0] = mr2 * u;
    d.tt[1] = d.q * u;
    d.xi[0] = fma(bh.a2, g.c2, -g.r2) * (bh.twoM * u);   // rho^2 - 2 r^2 = a^2 cos^2 - r^2
    d.xi[1] = g.twoMr * d.tt[1];
    d.pp[0] = mr2 * (g.t * g.irho2);
    d.pp[1] = (-2.0 * sc) * (g.t * g.t) * (g.rho2 - g.a2s2);
}

// FP32 value of a double from its high word (20 of its 52 mantissa bits,
// truncated), by integer operations only, for the index estimates of
// locate: no FP64 conversion instruction.  Exact enough for normal floats;
// any other input still ends in the right cell, since the walk in locate
// corrects any start.
__device__ __forceinline__ float f32_est(double x)
{
    const int hi = __double2hiint(x);
    const int e = ((hi >> 20) & 0x7ff) - 896;
    return __int_as_float((hi & (int)0x80000000) | (e << 23) | ((hi & 0xfffff) << 3));
}

// For a, b >= 0 or NaN (update sizes, tolerances): a <= b and a < b as the
// FP64 compares give them (false when either is a NaN), and fmax(m, a) for a
// running maximum m >= 0 (a NaN a is ignored), by integer compares of the
// bit patterns -- non-negative doubles order like their bits -- off the
// FP64 pipe.
constexpr long long F64_INF_BITS = 0x7ff0000000000000LL;
__device__ __forceinline__ bool le_nonneg(double a, double b)
{
    const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
    return ba <= bb && bb <= F64_INF_BITS;
}
__device__ __forceinline__ bool lt_nonneg(double a, double b)
{
    const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
    return ba < bb && bb <= F64_INF_BITS;
}
__device__ __forceinline__ double fmax_nonneg(double m, double a)
{
    const long long bm = __double_as_longlong(m), ba = __double_as_longlong(a);
    return (ba > F64_INF_BITS || ba <= bm) ? m : a;
}

// Order-preserving integer key of a double (monotone for all non-NaN values).
__device__ __forceinline__ long long okey(double x)
{
    long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// Grid as seen by the kernels.  Node tables and their inverse spacings
// 1/(X[i+1]-X[i]) live in library-owned device memory.
struct GridDev {
    int Nr, Nth, ld;
    const double *rn, *rh, *tn, *th;   // th: Nth half nodes + th[Nth] = th[0] + (tn[Nth] - tn[0])
    const double *irn, *irh, *itn, *ith;
    const double *brn, *brh, *btn, *bth;   // -X[i] / (X[i+1] - X[i]) (locate_fma)
    float lr0, lrh0, ilr;        // FP32 index estimate in ln r
    float t0, th0, it;           // FP32 index estimate in th
    int full;                    // full-theta domain (periodic th), else half-theta
    double tlo, tper, thlo;      // tn[0], the period tn[Nth] - tn[0], th[0]
};

// The th a gather sees.  Half-theta domain: th itself on both sub-grids,
// Nth half nodes.  Full-theta domain (Sec. 2.5: periodic boundaries): th
// wrapped into [tn[0], tn[0] + P) on the node sub-grid; on the half-node
// sub-grid a point below th[0] is taken at th + P, in the wrap cell
// [th[Nth-1], th[Nth] = th[0] + P] whose upper column (Nth) holds the image
// of column 0, so that sub-grid has Nth + 1 nodes.  One wrap suffices:
// particle states stay in the period and the RK4 stages and IMR midpoints
// stay within a step of it.
// The full-theta wrap is kept out of line behind a warp-uniform branch: if
// it were if-converted, its FP64 compares and adds would be issued in the
// half-theta domain too, on an FP64-bound push.
static __device__ __noinline__ double2 theta_wrap_full(double th, double tlo, double tper, double thlo)
{
    double t = th < tlo ? th + tper : th;
    t = t >= tlo + tper ? t - tper : t;
    return make_double2(t, t < thlo ? t + tper : t);
}

__device__ __forceinline__ void theta_views(const GridDev& G, double th, double& tn_view, double& th_view, int& mh)
{
    if (G.full) {
        const double2 v = theta_wrap_full(th, G.tlo, G.tper, G.thlo);
        tn_view = v.x;
        th_view = v.y;
        mh = G.Nth + 1;
    } else {
        tn_view = th_view = th;
        mh = G.Nth;
    }
}

// Locate x in node list X[0..m-1]: X[i] <= x < X[i+1], clamped to
// [0, m-2]; w is the clamped linear weight.  est: FP32 index estimate.
__device__ __forceinline__ int locate_walk(const double* __restrict__ X, int m, long long kx, float est)
{
    int k = __float2int_rd(est);
    k = max(0, min(k, m - 2));
    // walk to the right cell (the estimate is within one cell on uniform grids)
    for (int it = 0; it < m && k > 0 && kx < okey(__ldg(X + k)); ++it) --k;
    for (int it = 0; it < m && k < m - 2 && kx >= okey(__ldg(X + k + 1)); ++it) ++k;
    return k;
}

__device__ __forceinline__ void locate(const double* __restrict__ X, const double* __restrict__ iX,
                                       int m, double x, float est, int& i, double& w)
{
    const long long kx = okey(x);
    const int k = locate_walk(X, m, kx, est);
    i = k;
    const double x0 = __ldg(X + k);
    double ww = (x - x0) * __ldg(iX + k);
    const bool below = kx < okey(x0);
    const bool above = kx >= okey(__ldg(X + k + 1));
    ww = below ? 0.0 : ww;
    ww = above ? 1.0 : ww;
    w = ww;
}

// The same with the weight as one fused multiply-add, x iX[i] + BX[i]
// (BX[i] = -X[i] iX[i]): an absolute error of about X[i] iX[i] ulps of 1
// (~1e-13 on grids of a few hundred cells per e-fold) against one rounding
// for (x - X[i]) iX[i]; the field gathers take it (one FP64 instruction
// fewer per weight, four per gather).
__device__ __forceinline__ void locate_fma(const double* __restrict__ X, const double* __restrict__ iX,
                                           const double* __restrict__ BX, int m, double x, float est, int& i,
                                           double& w)
{
    const long long kx = okey(x);
    const int k = locate_walk(X, m, kx, est);
    i = k;
    double ww = fma(x, __ldg(iX + k), __ldg(BX + k));
    const bool below = kx < okey(__ldg(X + k));
    const bool above = kx >= okey(__ldg(X + k + 1));
    ww = below ? 0.0 : ww;
    ww = above ? 1.0 : ww;
    w = ww;
}

struct Fields {
    const double* f[6];   // D^r, D^th, D^ph, B^r, B^th, B^ph (Yee layout)
};

// Bilinear (r, th) gather of the six components at (r, th).
__device__ __forceinline__ void gather(const GridDev& G, const Fields& F, double r, double th,
                                       double D[3], double B[3])
{
    const float lr = __logf(f32_est(r));
    int i0, i1, j0, j1;
    double wr0, wr1, wt0, wt1;
    locate_fma(G.rn, G.irn, G.brn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i0, wr0);
    locate_fma(G.rh, G.irh, G.brh, G.Nr, r, (lr - G.lrh0) * G.ilr, i1, wr1);
    double tnv, thv;
    int mh;
    theta_views(G, th, tnv, thv, mh);
    const float tfn = f32_est(tnv), tfh = G.full ? f32_est(thv) : tfn;
    locate_fma(G.tn, G.itn, G.btn, G.Nth + 1, tnv, (tfn - G.t0) * G.it, j0, wt0);
    locate_fma(G.th, G.ith, G.bth, mh, thv, (tfh - G.th0) * G.it, j1, wt1);
    const int ld = G.ld;
    // component k sits at (roff, toff): D^r (1,0) D^th (0,1) D^ph (0,0)
    //                                    B^r (0,1) B^th (1,0) B^ph (1,1)
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool ro = (k == 0 || k == 4 || k == 5);
        const bool to = (k == 1 || k == 3 || k == 5);
        const int i = ro ? i1 : i0, j = to ? j1 : j0;
        const double wr = ro ? wr1 : wr0, wt = to ? wt1 : wt0;
        const double* p = F.f[k] + i * ld + j;
        const double f00 = __ldg(p), f01 = __ldg(p + 1);
        const double f10 = __ldg(p + ld), f11 = __ldg(p + ld + 1);
        const double lo = fma(wt, f01 - f00, f00);
        const double hi = fma(wt, f11 - f10, f10);
        v[k] = fma(wr, hi - lo, lo);
    }
    D[0] = v[0]; D[1] = v[1]; D[2] = v[2];
    B[0] = v[3]; B[1] = v[4]; B[2] = v[5];
}

// The same bilinear interpolant from per-cell coefficients: component k's
// cell (i, j) holds (a, b, c, d) = (f00, f10 - f00, f01 - f00,
// f11 - f10 - f01 + f00) at 4 (i ld + j) (r index first), so that
// f = a + b w_r + c w_th + d w_r w_th costs 3 FMA instead of 3 subtractions
// and 3 FMA (built by k_field_coef before each push).
struct FieldsC {
    const double* c[6];
};

__device__ __forceinline__ void gather_c(const GridDev& G, const FieldsC& F, double r, double th, double D[3],
                                         double B[3])
{
    const float lr = __logf(f32_est(r));
    int i0, i1, j0, j1;
    double wr0, wr1, wt0, wt1;
    locate_fma(G.rn, G.irn, G.brn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i0, wr0);
    locate_fma(G.rh, G.irh, G.brh, G.Nr, r, (lr - G.lrh0) * G.ilr, i1, wr1);
    double tnv, thv;
    int mh;
    theta_views(G, th, tnv, thv, mh);
    const float tfn = f32_est(tnv), tfh = G.full ? f32_est(thv) : tfn;
    locate_fma(G.tn, G.itn, G.btn, G.Nth + 1, tnv, (tfn - G.t0) * G.it, j0, wt0);
    locate_fma(G.th, G.ith, G.bth, mh, thv, (tfh - G.th0) * G.it, j1, wt1);
    const int ld = G.ld;
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool ro = (k == 0 || k == 4 || k == 5);
        const bool to = (k == 1 || k == 3 || k == 5);
        const int i = ro ? i1 : i0, j = to ? j1 : j0;
        const double wr = ro ? wr1 : wr0, wt = to ? wt1 : wt0;
        const double2* q = reinterpret_cast<const double2*>(F.c[k] + 4 * ((size_t)i * ld + j));
        const double2 ab = __ldg(q), cd = __ldg(q + 1);
        v[k] = fma(wt, fma(cd.y, wr, cd.x), fma(ab.y, wr, ab.x));
    }
    D[0] = v[0]; D[1] = v[1]; D[2] = v[2];
    B[0] = v[3]; B[1] = v[4]; B[2] = v[5];
}

// Field tile staged in shared memory for a block of cell-sorted particles:
// STAGE_TI coefficient rows (r cells) x STAGE_TJ coefficient cells (th) of
// each of the six components, starting at coefficient cell (i0, j0).  A
// gather whose cell lies in the tile reads shared memory, any other the
// global coefficients (so staging never changes a result).
constexpr int STAGE_TI = 5, STAGE_TJ = 16;
struct StageTile {
    const double* s;    // shared: [6][STAGE_TI][4 * STAGE_TJ]; nullptr = nothing staged
    int i0, j0;
};

__device__ __forceinline__ void gather_c(const GridDev& G, const FieldsC& F, double r, double th, double D[3],
                                         double B[3], const StageTile& T)
{
    const float lr = __logf(f32_est(r));
    int i0, i1, j0, j1;
    double wr0, wr1, wt0, wt1;
    locate_fma(G.rn, G.irn, G.brn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i0, wr0);
    locate_fma(G.rh, G.irh, G.brh, G.Nr, r, (lr - G.lrh0) * G.ilr, i1, wr1);
    double tnv, thv;
    int mh;
    theta_views(G, th, tnv, thv, mh);
    const float tfn = f32_est(tnv), tfh = G.full ? f32_est(thv) : tfn;
    locate_fma(G.tn, G.itn, G.btn, G.Nth + 1, tnv, (tfn - G.t0) * G.it, j0, wt0);
    locate_fma(G.th, G.ith, G.bth, mh, thv, (tfh - G.th0) * G.it, j1, wt1);
    const int ld = G.ld;
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool ro = (k == 0 || k == 4 || k == 5);
        const bool to = (k == 1 || k == 3 || k == 5);
        const int i = ro ? i1 : i0, j = to ? j1 : j0;
        const double wr = ro ? wr1 : wr0, wt = to ? wt1 : wt0;
        const unsigned ti = (unsigned)(i - T.i0), tj = (unsigned)(j - T.j0);
        double2 ab, cd;
        if (T.s && ti < (unsigned)STAGE_TI && tj < (unsigned)STAGE_TJ) {
            const double2* q = reinterpret_cast<const double2*>(T.s + ((k * STAGE_TI + ti) * STAGE_TJ + tj) * 4);
            ab = q[0];
            cd = q[1];
        } else {
            const double2* q = reinterpret_cast<const double2*>(F.c[k] + 4 * ((size_t)i * ld + j));
            ab = __ldg(q);
            cd = __ldg(q + 1);
        }
        v[k] = fma(wt, fma(cd.y, wr, cd.x), fma(ab.y, wr, ab.x));
    }
    D[0] = v[0]; D[1] = v[1]; D[2] = v[2];
    B[0] = v[3]; B[1] = v[4]; B[2] = v[5];
}

// What the Newton form of the implicit-midpoint solve needs from one
// right-hand side: u^i = g^ij u_j, 1 / Gamma, alpha / Gamma, g^ij, the
// magnetic-force factor qm alpha sqrt(gamma) / Gamma (0 without a field),
// B^i and u x B.
struct RhsJ {
    double U[3], iG, aiG;
    double gurr, gurp, gutt, gupp;
    double ks;
    double B[3], cx[3];
};

// Equations of motion at y (Eqs. p1, p2, O1, O2) and, as a by-product, the
// Hamiltonian H(y) = alpha Gamma - beta u_r - (q/m) A_0 (Eq. Ham with the
// Wald A_0 when B0pot != 0).  D, B: FIDO fields at y (ignored if !em).
// JAC: also fill *J (RhsJ) for the Newton iteration.
template <bool JAC>
__device__ __forceinline__ void eval_rhs_sc_t(const BH& bh, const double y[6], double s, double c, double qm,
                                              bool em, const double D[3], const double B[3], double B0pot,
                                              double f[6], double& H, RhsJ* J)
{
    Geo g;
    geo_eval(bh, y[0], s, c, g);
    GeoD d;
    geo_deriv(bh, y[0], g, d);
    const double ur = y[3], ut = y[4], up = y[5];
    const double Ur = fma(g.gurr, ur, g.gurp * up);
    const double Ut = g.gutt * ut;
    const double Up = fma(g.gurp, ur, g.gupp * up);
    const double G2 = fma(ur, Ur, fma(ut, Ut, fma(up, Up, 1.0)));
    const double iG = rsqrt_nr(G2);
    const double aiG = g.alpha * iG;
    f[0] = fma(aiG, Ur, -g.beta);
    f[1] = aiG * Ut;
    f[2] = aiG * Up;
    // du_i/dt = -Gamma d_i alpha + u_r d_i beta^r - (alpha / 2 Gamma) u_j u_k d_i g^jk
    // (Eq. p2).  With d alpha = -(alpha^3 / 2) d xi, d beta^r = d xi / xi^2,
    // d g^rr = a^2 s^2 d g^tt - d xi / xi^2 (+ q / rho^2 in th), d g^rp = a d g^tt:
    //   u_j u_k d_i g^jk = W d_i g^tt + u_ph^2 d_i g^pp - u_r^2 d_i xi / xi^2 (+ u_r^2 q / rho^2)
    //   with W = a^2 s^2 u_r^2 + 2 a u_r u_ph + u_th^2, so
    //   du_i/dt = h (W d_i g^tt + u_ph^2 d_i g^pp [+ u_r^2 q / rho^2])
    //             + d_i xi (u_r (1 - h u_r) / xi^2 + Gamma alpha^3 / 2),  h = -alpha / (2 Gamma).
    //   In r: W d_r g^tt + u_ph^2 d_r g^pp = -2 r (W / rho^4 + u_ph^2 / (rho^4 s^2))
    //   = -2 r / rho^2 (W / rho^2 + u_ph^2 t), t = 1 / (rho^2 s^2), so that
    //   h (...) = (alpha / Gamma) m0 with m0 = (r / rho^2) (W / rho^2 + u_ph^2 t).
    //   With alpha^2 = 1/xi the d_i xi factor is
    //   kap = (1/xi) ((1/xi) u_r (1 - h u_r) + alpha Gamma / 2), alpha Gamma / 2 = -h Gamma^2.
    const double h = -0.5 * aiG;
    const double urur = ur * ur, upup = up * up;
    const double W = fma(urur, g.a2s2, fma(2.0 * bh.a * ur, up, ut * ut));
    const double haG = -h * G2;                       // alpha Gamma / 2
    const double kap = g.ixi * fma(g.ixi * ur, fma(-h, ur, 1.0), haG);
    const double m0 = (y[0] * g.irho2) * fma(W, g.irho2, upup * g.t);
    f[3] = fma(aiG, m0, d.xi[0] * kap);
    f[4] = fma(h, fma(W, d.tt[1], fma(upup, d.pp[1], urur * d.q * g.irho2)), d.xi[1] * kap);
    f[5] = 0.0;
    if (JAC) {
        J->U[0] = Ur; J->U[1] = Ut; J->U[2] = Up;
        J->iG = iG; J->aiG = aiG;
        J->gurr = g.gurr; J->gurp = g.gurp; J->gutt = g.gutt; J->gupp = g.gupp;
        // no field: the force terms of the Newton matrix vanish (set, not left undefined)
        J->ks = 0.0;
        J->B[0] = J->B[1] = J->B[2] = 0.0;
        J->cx[0] = J->cx[1] = J->cx[2] = 0.0;
    }
    if (em) {
        // (q/m) alpha gamma_ij D^j with gamma_rr = xi, gamma_rph = -a xi s^2,
        // gamma_thth = rho^2, gamma_phph = s^2 (rho^2 + a^2 xi s^2):
        //   r:  k xi X,  X = D^r - a s^2 D^ph
        //   ph: k s^2 (rho^2 D^ph - a xi X)
        const double k = qm * g.alpha;
        const double kxi = k * g.xi, kr = k * g.rho2;
        const double ks = (qm * g.rho2) * (g.s * iG);    // k sqrt(gamma) / Gamma, alpha^2 xi = 1
        const double cr = fma(Ut, B[2], -Up * B[1]);
        const double ct = fma(Up, B[0], -Ur * B[2]);
        const double cp = fma(Ur, B[1], -Ut * B[0]);
        const double X = fma(-bh.a * g.s2, D[2], D[0]);
        f[3] = fma(kxi, X, fma(ks, cr, f[3]));
        f[4] = fma(kr, D[1], fma(ks, ct, f[4]));
        f[5] = fma(g.s2, fma(kr, D[2], -(bh.a * kxi) * X), ks * cp);
        if (JAC) {
            J->ks = ks;
            J->B[0] = B[0]; J->B[1] = B[1]; J->B[2] = B[2];
            J->cx[0] = cr; J->cx[1] = ct; J->cx[2] = cp;
        }
    }
    H = fma(-g.beta, ur, haG + haG);                  // alpha Gamma - beta^r u_r
    if (B0pot != 0.0 && qm != 0.0) {
        // A_0 = B0 a r (1 + cos^2 th) / rho^2   (Sec. 3.1.3)
        H = fma(-qm * B0pot * bh.a * y[0], (1.0 + g.c2) * g.irho2, H);
    }
}

__device__ __forceinline__ void eval_rhs_sc(const BH& bh, const double y[6], double s, double c, double qm,
                                            bool em, const double D[3], const double B[3], double B0pot,
                                            double f[6], double& H)
{
    eval_rhs_sc_t<false>(bh, y, s, c, qm, em, D, B, B0pot, f, H, nullptr);
}

__device__ __forceinline__ void eval_rhs(const BH& bh, const double y[6], double qm, bool em,
                                         const double D[3], const double B[3], double B0pot,
                                         double f[6], double& H)
{
    double s, c;
    sincos(y[1], &s, &c);
    eval_rhs_sc(bh, y, s, c, qm, em, D, B, B0pot, f, H);
}

// Hamiltonian only (no derivatives, no force), given sin/cos of y[1].
__device__ __forceinline__ double eval_H_sc(const BH& bh, const double y[6], double s, double c, double qm,
                                            double B0pot)
{
    Geo g;
    geo_eval(bh, y[0], s, c, g);
    const double ur = y[3], ut = y[4], up = y[5];
    const double Ur = fma(g.gurr, ur, g.gurp * up);
    const double Ut = g.gutt * ut;
    const double Up = fma(g.gurp, ur, g.gupp * up);
    const double G = sqrt(fma(ur, Ur, fma(ut, Ut, fma(up, Up, 1.0))));
    double H = fma(g.alpha, G, -g.beta * ur);
    if (B0pot != 0.0 && qm != 0.0) H = fma(-qm * B0pot * bh.a * y[0], (1.0 + c * c) * g.irho2, H);
    return H;
}

// The two parts of H at z (Sec. 3.1.2): kin = alpha Gamma - beta^r u_r and
// pot = (q/m) A_0 of the Wald potential (B0pot = 0: none); H = kin - pot and
// the error normaliser D0 = |kin| + |pot|.
__device__ __forceinline__ void h_parts(const BH& bh, const double z[6], double qm, double B0pot, double& kin,
                                        double& pot)
{
    double s, c;
    sincos(z[1], &s, &c);
    Geo g;
    geo_eval(bh, z[0], s, c, g);
    const double ur = z[3], ut = z[4], up = z[5];
    const double G2 = fma(ur, fma(g.gurr, ur, g.gurp * up),
                          fma(ut, g.gutt * ut, fma(up, fma(g.gurp, ur, g.gupp * up), 1.0)));
    kin = fma(g.alpha, sqrt(G2), -g.beta * ur);
    pot = 0.0;
    if (B0pot != 0.0 && qm != 0.0) pot = qm * B0pot * bh.a * z[0] * (1.0 + c * c) * g.irho2;
}

__device__ __forceinline__ double eval_H(const BH& bh, const double y[6], double qm, double B0pot)
{
    double s, c;
    sincos(y[1], &s, &c);
    return eval_H_sc(bh, y, s, c, qm, B0pot);
}

// The Wald field (App. B.1) at (r, th) with sin/cos of th given: B^i =
// eta^ijk d_j A_k / sqrt(gamma) from the potentials of Eq. (Amu), E_i =
// d_i A_0, D^i raised from Eq. (Ei) with beta = (beta^r, 0, 0).
__device__ __forceinline__ void wald_point_sc(const BH& bh, double B0, double r, double s, double c, double D[3],
                                              double B[3])
{
    Geo g;
    geo_eval(bh, r, s, c, g);
    const double M = bh.M, a = bh.a, a2 = bh.a2;
    const double P = g.rho2, iP = g.irho2, iP2 = iP * iP;
    const double sc = s * c, s2 = s * s, c2p1 = 1.0 + c * c;
    const double q = a2 * c2p1 - P;                 // enters d_th[(1+c^2)/rho^2]
    const double isg = 1.0 / g.sqrtg;
    const double dAph_t = B0 * sc * (r * r + a2 - 2.0 * M * a2 * r * c2p1 * iP - 2.0 * M * a2 * r * s2 * q * iP2);
    const double dAph_r = 0.5 * B0 * s2 * (2.0 * r - 2.0 * M * a2 * c2p1 * (P - 2.0 * r * r) * iP2);
    const double dAr_t = B0 * a * sc * (-1.0 + 2.0 * M * r * q * iP2);
    B[0] = dAph_t * isg;
    B[1] = -dAph_r * isg;
    B[2] = -dAr_t * isg;
    const double Er = B0 * a * M * c2p1 * (P - 2.0 * r * r) * iP2;
    const double Et = 2.0 * B0 * a * M * r * sc * q * iP2;
    // D_i from Eq. (Ei) with beta = (beta^r, 0, 0), then raised
    const double Dr_ = Er / g.alpha;
    const double Dt_ = (Et + g.sqrtg * g.beta * B[2]) / g.alpha;
    const double Dp_ = -g.sqrtg * g.beta * B[1] / g.alpha;
    D[0] = fma(g.gurr, Dr_, g.gurp * Dp_);
    D[1] = g.gutt * Dt_;
    D[2] = fma(g.gurp, Dr_, g.gupp * Dp_);
}

}  // namespace fpic
