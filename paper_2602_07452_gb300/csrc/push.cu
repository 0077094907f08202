// Particle push (Sec. 2.2) and the hybrid RK4 <-> implicit switch (Sec. 3.1.2).
//
// Two kernels per hybrid step:
//   k_explicit  one thread per particle: RK4 trial (4 right-hand sides), H of
//               the trial, the Hyb1/Hyb2 test.  Accepted particles are
//               finished in place; rejected ones append their index to a
//               queue and park the trial as the implicit initial guess.
//   k_imr       persistent, lane-refilling implicit-midpoint solver over the
//               queue: every loop trip performs exactly one right-hand-side
//               evaluation per lane, and a lane whose particle converged
//               fetches the next queue entry, so the spread of iteration
//               counts does not idle the FP64 pipe.
//   k_dg        discrete-gradient Hamiltonian scheme (geodesics), one thread
//               per queued particle.
#include <math.h>

#include "fpic_internal.h"

namespace fpic {

struct PartDev {
    double *r, *th, *ph, *ur, *uth, *uph, *qm, *H0, *D0, *Hn;
    uint8_t *alive, *scheme, *iters;
    uint32_t* cell;
};

struct PushK {
    BH bh;
    GridDev G;
    Fields F;
    int has_fields;
    int has_grid;
    double dt, thr, tol, dg_eps, B0pot, r_h, r_max;
    int scheme, max_iter;
    long long n;
    PartDev P;
    double* guess;          // 6 x n (SoA) implicit initial guesses
    uint32_t* queue;        // indices of particles for the implicit solver
    long long* cnt;
    const float* learned;   // n x 8 learned guess (nullable)
};

__device__ __forceinline__ void load_state(const PartDev& P, long long p, double z[6])
{
    z[0] = P.r[p]; z[1] = P.th[p]; z[2] = P.ph[p];
    z[3] = P.ur[p]; z[4] = P.uth[p]; z[5] = P.uph[p];
}

__device__ __forceinline__ void store_state(const PartDev& P, long long p, const double z[6])
{
    P.r[p] = z[0]; P.th[p] = z[1]; P.ph[p] = z[2];
    P.ur[p] = z[3]; P.uth[p] = z[4]; P.uph[p] = z[5];
}

__device__ __forceinline__ uint32_t cell_of(const GridDev& G, double r, double th)
{
    int i, j;
    double w;
    const float lr = __logf((float)r);
    locate(G.rn, G.irn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i, w);
    locate(G.tn, G.itn, G.Nth + 1, th, ((float)th - G.t0) * G.it, j, w);
    return (uint32_t)i * (uint32_t)G.Nth + (uint32_t)j;
}

// Right-hand side at y: gathers the fields when the particle is charged.
__device__ __forceinline__ void F_at(const PushK& k, const double y[6], double qm, bool em,
                                     double f[6], double& H)
{
    double D[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    if (em) gather(k.G, k.F, y[0], y[1], D, B);
    eval_rhs(k.bh, y, qm, em, D, B, k.B0pot, f, H);
}

// Particle boundaries (Sec. 2.5) and write-back of a finished step.
__device__ __forceinline__ bool finish(const PushK& k, long long p, double z[6], double H,
                                       int implicit, int iters)
{
    if (z[1] < 0.0) {
        z[1] = -z[1];
        z[4] = -z[4];
        z[2] += M_PI;
    } else if (z[1] > M_PI) {
        z[1] = 2.0 * M_PI - z[1];
        z[4] = -z[4];
        z[2] += M_PI;
    }
    const bool alive = (z[0] >= k.r_h) && (z[0] <= k.r_max);
    store_state(k.P, p, z);
    k.P.Hn[p] = H;
    k.P.scheme[p] = (uint8_t)implicit;
    k.P.iters[p] = (uint8_t)min(iters, 255);
    k.P.alive[p] = alive ? 1 : 0;
    if (k.P.cell) k.P.cell[p] = k.has_grid ? cell_of(k.G, z[0], z[1]) : 0u;
    return alive;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-aggregated add of a per-lane value to a device counter.
__device__ __forceinline__ void warp_add(long long* c, long long v, unsigned mask)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o);
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && v) atomicAdd((unsigned long long*)c, (unsigned long long)v);
}

// MODE 0: RK4 only.  MODE 1: hybrid (RK4 trial + test + enqueue).
template <int MODE>
__global__ void __launch_bounds__(128) k_explicit(PushK k)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= k.n) return;
    if (!k.P.alive[p]) {
        k.P.scheme[p] = 0;
        k.P.iters[p] = 0;
        return;
    }
    double z0[6], kk[6], acc[6], y[6];
    load_state(k.P, p, z0);
    const double qm = k.P.qm[p];
    const bool em = k.has_fields && qm != 0.0;
    const double dt = k.dt, hdt = 0.5 * k.dt;
    double Hd;
    F_at(k, z0, qm, em, kk, Hd);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = kk[i]; y[i] = fma(hdt, kk[i], z0[i]); }
    F_at(k, y, qm, em, kk, Hd);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = fma(2.0, kk[i], acc[i]); y[i] = fma(hdt, kk[i], z0[i]); }
    F_at(k, y, qm, em, kk, Hd);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = fma(2.0, kk[i], acc[i]); y[i] = fma(dt, kk[i], z0[i]); }
    F_at(k, y, qm, em, kk, Hd);
    const double d6 = dt / 6.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = fma(d6, acc[i] + kk[i], z0[i]);
    const double H1 = eval_H(k.bh, y, qm, k.B0pot);
    bool accept = true;
    if (MODE == 1) {
        const double H0 = k.P.H0[p], D0 = k.P.D0[p];
        const double Ht1 = fabs(H1 - H0) / D0;
        if (k.scheme == FPIC_HYB2) {
            accept = Ht1 < k.thr;
        } else {
            const double Htn = fabs(k.P.Hn[p] - H0) / D0;
            accept = (Ht1 - Htn) / dt < k.thr;
        }
    }
    const unsigned act = __activemask();
    const unsigned rej = __ballot_sync(act, !accept);
    if (accept && !finish(k, p, y, H1, 0, 0))
        atomicAdd((unsigned long long*)&k.cnt[CNT_REMOVED], 1ull);
    if (rej) {
        const int leader = __ffs(act) - 1;
        unsigned long long base = 0;
        if ((int)(threadIdx.x & 31) == leader)
            base = atomicAdd((unsigned long long*)&k.cnt[CNT_QUEUE], (unsigned long long)__popc(rej));
        base = __shfl_sync(act, base, leader);
        if (!accept) {
            const unsigned long long idx = base + __popc(rej & lanemask_lt());
            k.queue[idx] = (uint32_t)p;
#pragma unroll
            for (int i = 0; i < 6; ++i) k.guess[(size_t)i * k.n + p] = y[i];
        }
    }
}

__device__ __forceinline__ bool conv6(const double a[6], const double b[6], double tol)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) ok = ok && (fabs(a[i] - b[i]) <= tol * (fabs(a[i]) + 1.0));
    return ok;
}

// Persistent lane-refilling implicit-midpoint solver (Sec. 2.2.2):
// z^[k] = z^n + dt F((z^n + z^[k-1]) / 2), then one evaluation at the
// converged point for H.  all_mode: the queue is every particle (pure IMR,
// guess z^n); otherwise entries come from k_explicit with their trial.
__global__ void __launch_bounds__(128) k_imr(PushK k, int all_mode)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long qn = all_mode ? k.n : k.cnt[CNT_QUEUE];
    long long p = -1;
    bool exhausted = false, fin = false;
    double z0[6], zk[6];
    double qm = 0.0;
    bool em = false;
    int it = 0;
    long long n_it = 0, n_nc = 0, n_ev = 0, n_rm = 0;
    for (;;) {
        const bool need = (p < 0) && !exhausted;
        const unsigned nm = __ballot_sync(FULL, need);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader)
                base = atomicAdd((unsigned long long*)&k.cnt[CNT_HEAD], (unsigned long long)__popc(nm));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                const long long idx = (long long)(base + __popc(nm & lanemask_lt()));
                if (idx < qn) {
                    const long long q = all_mode ? idx : (long long)k.queue[idx];
                    if (all_mode && !k.P.alive[q]) {
                        k.P.scheme[q] = 0;
                        k.P.iters[q] = 0;
                    } else {
                        p = q;
                        load_state(k.P, p, z0);
                        if (all_mode) {
#pragma unroll
                            for (int i = 0; i < 6; ++i) zk[i] = z0[i];
                        } else {
#pragma unroll
                            for (int i = 0; i < 6; ++i) zk[i] = k.guess[(size_t)i * k.n + p];
                        }
                        qm = k.P.qm[p];
                        em = k.has_fields && qm != 0.0;
                        it = 0;
                        fin = false;
                    }
                } else {
                    exhausted = true;
                }
            }
        }
        const unsigned busy = __ballot_sync(FULL, p >= 0);
        if (!busy) {
            if (!__ballot_sync(FULL, !exhausted)) break;
            continue;
        }
        if (p >= 0) {
            double y[6], f[6], H;
            if (fin) {
#pragma unroll
                for (int i = 0; i < 6; ++i) y[i] = zk[i];
            } else {
#pragma unroll
                for (int i = 0; i < 6; ++i) y[i] = 0.5 * (z0[i] + zk[i]);
            }
            F_at(k, y, qm, em, f, H);
            ++n_ev;
            if (!fin) {
                double zn[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) zn[i] = fma(k.dt, f[i], z0[i]);
                const bool ok = conv6(zn, zk, k.tol);
#pragma unroll
                for (int i = 0; i < 6; ++i) zk[i] = zn[i];
                ++it;
                if (ok || it >= k.max_iter) {
                    fin = true;
                    if (!ok) ++n_nc;
                }
            } else {
                if (!finish(k, p, zk, H, 1, it)) ++n_rm;
                n_it += it;
                p = -1;
            }
        }
    }
    warp_add(&k.cnt[CNT_ITERS], n_it, FULL);
    warp_add(&k.cnt[CNT_NOTCONV], n_nc, FULL);
    warp_add(&k.cnt[CNT_EVALS], n_ev, FULL);
    warp_add(&k.cnt[CNT_REMOVED], n_rm, FULL);
}

// ---------------------------------------------------------------------------
// Discrete-gradient Hamiltonian scheme for geodesics (Sec. 2.2.3, App. D).
// The symmetrised gradient averages the coordinate-increment gradients of
// the 12 update orders (3! pair orders x {coordinate-first, momentum-first});
// since H does not depend on ph and u_ph never changes, they reduce to four
// distinct orders over (r, u_r, th, u_th), each of weight 1/4, and the
// u_ph component to the analytic dH/du_ph averaged over the states where
// u_ph is visited (weights 2,1,1,2 / 6).  H needs the metric at only four
// (r, th) combinations per iteration.
// ---------------------------------------------------------------------------
struct GH {
    double alpha, beta, gurr, gurp, gutt, gupp;
};

__device__ __forceinline__ GH gh_at(const BH& bh, double r, double th)
{
    double s, c;
    sincos(th, &s, &c);
    Geo g;
    geo_eval(bh, r, s, c, g);
    return GH{g.alpha, g.beta, g.gurr, g.gurp, g.gutt, g.gupp};
}

__device__ __forceinline__ double gh_G(const GH& g, double ur, double ut, double up)
{
    return sqrt(fma(g.gurr * ur, ur, fma(2.0 * g.gurp * ur, up, fma(g.gutt * ut, ut, fma(g.gupp * up, up, 1.0)))));
}

__device__ __forceinline__ double gh_H(const GH& g, double ur, double ut, double up)
{
    return fma(g.alpha, gh_G(g, ur, ut, up), -g.beta * ur);
}

__device__ __forceinline__ double gh_dHdup(const GH& g, double ur, double ut, double up)
{
    return g.alpha * fma(g.gurp, ur, g.gupp * up) / gh_G(g, ur, ut, up);
}

// Analytic partial dH/dz_v (v: 0 r, 1 th, 3 u_r, 4 u_th) at a state.
__device__ double dg_partial(const BH& bh, double r, double th, double ur, double ut, double up, int v)
{
    double y[6] = {r, th, 0.0, ur, ut, up}, f[6], H;
    const double D[3] = {0, 0, 0};
    eval_rhs(bh, y, 0.0, false, D, D, 0.0, f, H);
    switch (v) {
        case 0: return -f[3];
        case 1: return -f[4];
        case 3: return f[0];
        default: return f[1];
    }
}

__device__ __forceinline__ double dgq(const BH& bh, double Hn, double Ho, double dz, double eps,
                                      double r, double th, double ur, double ut, double up, int v)
{
    if (fabs(dz) < eps) return dg_partial(bh, r, th, ur, ut, up, v);
    return (Hn - Ho) / dz;
}

__global__ void __launch_bounds__(128) k_dg(PushK k, int all_mode)
{
    const long long qn = all_mode ? k.n : k.cnt[CNT_QUEUE];
    long long n_it = 0, n_nc = 0, n_rm = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < qn;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long p = all_mode ? idx : (long long)k.queue[idx];
        if (all_mode && !k.P.alive[p]) {
            k.P.scheme[p] = 0;
            k.P.iters[p] = 0;
            continue;
        }
        double z0[6], zk[6];
        load_state(k.P, p, z0);
        if (all_mode) {
            for (int i = 0; i < 6; ++i) zk[i] = z0[i];
        } else {
            for (int i = 0; i < 6; ++i) zk[i] = k.guess[(size_t)i * k.n + p];
        }
        const double R0 = z0[0], T0 = z0[1], U0 = z0[3], V0 = z0[4], P = z0[5];
        const GH m00 = gh_at(k.bh, R0, T0);
        const double Hz0 = gh_H(m00, U0, V0, P);
        const double f00 = gh_dHdup(m00, U0, V0, P);
        const double eps = k.dg_eps;
        int it = 0;
        bool ok = false;
        while (it < k.max_iter) {
            const double R1 = zk[0], T1 = zk[1], U1 = zk[3], V1 = zk[4];
            const GH m10 = gh_at(k.bh, R1, T0), m01 = gh_at(k.bh, R0, T1), m11 = gh_at(k.bh, R1, T1);
            const double dR = R1 - R0, dT = T1 - T0, dU = U1 - U0, dV = V1 - V0;
            const double Rm = 0.5 * (R0 + R1), Tm = 0.5 * (T0 + T1);
            const double Um = 0.5 * (U0 + U1), Vm = 0.5 * (V0 + V1);
            const double Hz1 = gh_H(m11, U1, V1, P);
            const double A1 = gh_H(m10, U0, V0, P), A2 = gh_H(m10, U1, V0, P), A3 = gh_H(m11, U1, V0, P);
            const double B1 = gh_H(m00, U1, V0, P), B3 = gh_H(m10, U1, V1, P);
            const double C1 = gh_H(m01, U0, V0, P), C2 = gh_H(m01, U0, V1, P), C3 = gh_H(m11, U0, V1, P);
            const double D1 = gh_H(m00, U0, V1, P), D3 = gh_H(m01, U1, V1, P);
            const BH& bh = k.bh;
            // order A: r, u_r, th, u_th
            const double rA = dgq(bh, A1, Hz0, dR, eps, Rm, T0, U0, V0, P, 0);
            const double uA = dgq(bh, A2, A1, dU, eps, R1, T0, Um, V0, P, 3);
            const double tA = dgq(bh, A3, A2, dT, eps, R1, Tm, U1, V0, P, 1);
            const double vA = dgq(bh, Hz1, A3, dV, eps, R1, T1, U1, Vm, P, 4);
            // order B: u_r, r, u_th, th
            const double uB = dgq(bh, B1, Hz0, dU, eps, R0, T0, Um, V0, P, 3);
            const double rB = dgq(bh, A2, B1, dR, eps, Rm, T0, U1, V0, P, 0);
            const double vB = dgq(bh, B3, A2, dV, eps, R1, T0, U1, Vm, P, 4);
            const double tB = dgq(bh, Hz1, B3, dT, eps, R1, Tm, U1, V1, P, 1);
            // order C: th, u_th, r, u_r
            const double tC = dgq(bh, C1, Hz0, dT, eps, R0, Tm, U0, V0, P, 1);
            const double vC = dgq(bh, C2, C1, dV, eps, R0, T1, U0, Vm, P, 4);
            const double rC = dgq(bh, C3, C2, dR, eps, Rm, T1, U0, V1, P, 0);
            const double uC = dgq(bh, Hz1, C3, dU, eps, R1, T1, Um, V1, P, 3);
            // order D: u_th, th, u_r, r
            const double vD = dgq(bh, D1, Hz0, dV, eps, R0, T0, U0, Vm, P, 4);
            const double tD = dgq(bh, C2, D1, dT, eps, R0, Tm, U0, V1, P, 1);
            const double uD = dgq(bh, D3, C2, dU, eps, R0, T1, Um, V1, P, 3);
            const double rD = dgq(bh, Hz1, D3, dR, eps, Rm, T1, U1, V1, P, 0);
            const double Gr = 0.25 * (rA + rB + rC + rD);
            const double Gt = 0.25 * (tA + tB + tC + tD);
            const double Gu = 0.25 * (uA + uB + uC + uD);
            const double Gv = 0.25 * (vA + vB + vC + vD);
            const double Gp = (2.0 * f00 + gh_dHdup(m10, U1, V0, P) + gh_dHdup(m01, U0, V1, P) +
                               2.0 * gh_dHdup(m11, U1, V1, P)) / 6.0;
            double zn[6];
            zn[0] = fma(k.dt, Gu, z0[0]);
            zn[1] = fma(k.dt, Gv, z0[1]);
            zn[2] = fma(k.dt, Gp, z0[2]);
            zn[3] = fma(-k.dt, Gr, z0[3]);
            zn[4] = fma(-k.dt, Gt, z0[4]);
            zn[5] = z0[5];
            ok = conv6(zn, zk, k.tol);
            for (int i = 0; i < 6; ++i) zk[i] = zn[i];
            ++it;
            if (ok) break;
        }
        if (!ok) ++n_nc;
        n_it += it;
        const double H1 = eval_H(k.bh, zk, 0.0, 0.0);
        if (!finish(k, p, zk, H1, 1, it)) ++n_rm;
    }
    const unsigned m = __activemask();
    warp_add(&k.cnt[CNT_ITERS], n_it, m);
    warp_add(&k.cnt[CNT_NOTCONV], n_nc, m);
    warp_add(&k.cnt[CNT_EVALS], n_it, m);
    warp_add(&k.cnt[CNT_REMOVED], n_rm, m);
}

__global__ void k_count_alive(PartDev P, long long n, long long* cnt)
{
    long long v = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v += P.alive[i] ? 1 : 0;
    warp_add(&cnt[CNT_ALIVE], v, 0xffffffffu);
}

}  // namespace fpic

using namespace fpic;

extern "C" int fpic_push(fpic_ctx* c, fpic_particles* p, const double* const fields[6],
                         const fpic_push_params* prm, fpic_push_stats* stats, void* stream)
{
    if (!c || !p || !prm) return set_error(FPIC_EINVAL, "fpic_push: NULL ctx/particles/params");
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_push: n out of range [0, 2^31)");
    if (!particles_ok(p, true)) return set_error(FPIC_EINVAL, "fpic_push: a particle array is NULL");
    if (!(std::isfinite(prm->dt)) || prm->dt == 0.0) return set_error(FPIC_EINVAL, "fpic_push: dt must be finite and nonzero");
    if (prm->scheme < FPIC_RK4 || prm->scheme > FPIC_HYB2) return set_error(FPIC_EINVAL, "fpic_push: unknown scheme %d", prm->scheme);
    if (prm->scheme >= FPIC_HYB1 && prm->implicit != FPIC_IMR && prm->implicit != FPIC_HAM)
        return set_error(FPIC_EINVAL, "fpic_push: implicit partner must be FPIC_IMR or FPIC_HAM");
    if (prm->max_iter < 1 || prm->max_iter > 255) return set_error(FPIC_EINVAL, "fpic_push: max_iter must be in [1, 255]");
    if (!(prm->tol >= 0.0)) return set_error(FPIC_EINVAL, "fpic_push: tol must be >= 0");
    bool has_fields = fields != nullptr;
    if (has_fields) {
        for (int i = 0; i < 6; ++i)
            if (!fields[i]) return set_error(FPIC_EINVAL, "fpic_push: fields[%d] is NULL", i);
        if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_push: fields given but no grid set");
    }
    if (prm->guess) return set_error(FPIC_EINVAL, "fpic_push: learned guesses need fpic_push_learned");
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    FPIC_CUDA(cudaSetDevice(c->device));
    const size_t need = (size_t)n * (6 * sizeof(double) + sizeof(uint32_t)) + 256;
    int rc = ensure_scratch(c, need);
    if (rc) return rc;
    PushK k{};
    k.bh = c->bh;
    k.G = c->G;
    k.has_grid = c->has_grid;
    k.has_fields = has_fields;
    for (int i = 0; i < 6; ++i) k.F.f[i] = has_fields ? fields[i] : nullptr;
    k.dt = prm->dt;
    k.thr = prm->thr;
    k.tol = prm->tol;
    k.dg_eps = prm->dg_eps;
    k.B0pot = prm->B0pot;
    k.r_h = c->r_h;
    k.r_max = prm->r_max;
    k.scheme = prm->scheme;
    k.max_iter = prm->max_iter;
    k.n = n;
    k.P = PartDev{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                  p->alive, p->scheme, p->iters, p->cell};
    k.guess = (double*)c->d_scratch;
    k.queue = (uint32_t*)((char*)c->d_scratch + (size_t)n * 6 * sizeof(double));
    k.cnt = c->d_cnt;
    k.learned = nullptr;
    FPIC_CUDA(cudaMemsetAsync(c->d_cnt, 0, CNT_N * sizeof(long long), s));
    if (n == 0) {
        if (stats) *stats = fpic_push_stats{};
        return FPIC_OK;
    }
    const int TB = 128;
    const unsigned nb = (unsigned)((n + TB - 1) / TB);
    const unsigned persist = (unsigned)c->sm_count * 8u;
    cudaEvent_t* ev = prm->events ? (cudaEvent_t*)prm->events : nullptr;
    if (stats) k_count_alive<<<persist, 256, 0, s>>>(k.P, n, c->d_cnt);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[0], s));
    if (prm->scheme == FPIC_RK4) k_explicit<0><<<nb, TB, 0, s>>>(k);
    else if (prm->scheme >= FPIC_HYB1) k_explicit<1><<<nb, TB, 0, s>>>(k);
    if (ev) {
        FPIC_CUDA(cudaEventRecord(ev[1], s));
        FPIC_CUDA(cudaEventRecord(ev[2], s));
    }
    if (prm->scheme == FPIC_IMR) k_imr<<<persist, TB, 0, s>>>(k, 1);
    else if (prm->scheme == FPIC_HAM) k_dg<<<nb, TB, 0, s>>>(k, 1);
    else if (prm->scheme >= FPIC_HYB1 && prm->implicit == FPIC_IMR) k_imr<<<persist, TB, 0, s>>>(k, 0);
    else if (prm->scheme >= FPIC_HYB1) k_dg<<<nb, TB, 0, s>>>(k, 0);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[3], s));
    FPIC_CUDA(cudaGetLastError());
    if (stats) {
        FPIC_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, CNT_N * sizeof(long long), cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        const long long* h = c->h_cnt;
        const bool explicit_pass = prm->scheme == FPIC_RK4 || prm->scheme >= FPIC_HYB1;
        stats->n_alive_before = h[CNT_ALIVE];
        stats->n_implicit = prm->scheme == FPIC_RK4 ? 0 : (prm->scheme >= FPIC_HYB1 ? h[CNT_QUEUE] : h[CNT_ALIVE]);
        stats->n_iter_total = h[CNT_ITERS];
        stats->n_notconv = h[CNT_NOTCONV];
        stats->n_removed = h[CNT_REMOVED];
        stats->n_rhs_evals = h[CNT_EVALS] + (explicit_pass ? 4 * h[CNT_ALIVE] : 0);
        if (h[CNT_NOTCONV] > 0) return FPIC_ENOTCONVERGED;
    }
    return FPIC_OK;
}

extern "C" int fpic_push_host(fpic_ctx* c, fpic_particles* hp, const double* const fields[6],
                              const fpic_push_params* prm, fpic_push_stats* stats, void* stream)
{
    if (!c || !hp || !prm) return set_error(FPIC_EINVAL, "fpic_push_host: NULL ctx/particles/params");
    if (hp->n < 0 || hp->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_push_host: n out of range");
    if (!particles_ok(hp, true)) return set_error(FPIC_EINVAL, "fpic_push_host: a particle array is NULL");
    const long long n = hp->n;
    cudaStream_t s = (cudaStream_t)stream;
    FPIC_CUDA(cudaSetDevice(c->device));
    // device mirror: 11 double arrays, 3 byte arrays, 1 u32 array
    const size_t nd = (size_t)n * sizeof(double), nb = (size_t)n, n4 = (size_t)n * 4;
    int rc = ensure_scratch2(c, 11 * nd + 3 * nb + n4 + 64);
    if (rc) return rc;
    char* base = (char*)c->d_scratch2;
    fpic_particles d{};
    d.n = n;
    double** dd[] = {&d.r, &d.th, &d.ph, &d.ur, &d.uth, &d.uph, &d.qm, &d.w, &d.H0, &d.D0, &d.Hn};
    double* const hd[] = {hp->r, hp->th, hp->ph, hp->ur, hp->uth, hp->uph, hp->qm, hp->w, hp->H0, hp->D0, hp->Hn};
    for (int i = 0; i < 11; ++i) *dd[i] = (double*)(base + i * nd);
    d.alive = (uint8_t*)(base + 11 * nd);
    d.scheme = d.alive + nb;
    d.iters = d.scheme + nb;
    d.cell = (uint32_t*)(((uintptr_t)(d.iters + nb) + 15) & ~(uintptr_t)15);
    for (int i = 0; i < 11; ++i)
        if (hd[i] && n) FPIC_CUDA(cudaMemcpyAsync(*dd[i], hd[i], nd, cudaMemcpyHostToDevice, s));
    if (n) FPIC_CUDA(cudaMemcpyAsync(d.alive, hp->alive, nb, cudaMemcpyHostToDevice, s));
    rc = fpic_push(c, &d, fields, prm, stats, stream);
    if (rc < 0) return rc;
    const int back[] = {0, 1, 2, 3, 4, 5, 10};
    for (int i : back)
        if (n) FPIC_CUDA(cudaMemcpyAsync(hd[i], *dd[i], nd, cudaMemcpyDeviceToHost, s));
    if (n) {
        FPIC_CUDA(cudaMemcpyAsync(hp->alive, d.alive, nb, cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaMemcpyAsync(hp->scheme, d.scheme, nb, cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaMemcpyAsync(hp->iters, d.iters, nb, cudaMemcpyDeviceToHost, s));
        if (hp->cell) FPIC_CUDA(cudaMemcpyAsync(hp->cell, d.cell, n4, cudaMemcpyDeviceToHost, s));
    }
    FPIC_CUDA(cudaStreamSynchronize(s));
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free geodesic push.
//
// For callers that must not allocate device memory themselves or through
// this library: code that runs where the process's device memory is owned
// by someone else (a host framework or a custom allocator that forbids
// direct cudaMalloc), real-time loops in which an allocation (and the
// device synchronisation a cudaFree implies) is not allowed, and embedded
// or plugin builds linked without an allocator.  The scratch that
// fpic_push keeps in the context (implicit-solver guesses, the queue of
// rejected particles, counters) lives here in one file-scope device array
// of fixed size instead, so no context and no allocation are needed.
// ---------------------------------------------------------------------------

namespace fpic {

constexpr long long kNoAllocMax = FPIC_NOALLOC_MAX_PARTICLES;
constexpr size_t kNoAllocCountersBytes = 256;   // CNT_N counters, padded for alignment
constexpr size_t kNoAllocBytes = kNoAllocCountersBytes + (size_t)kNoAllocMax * (6 * sizeof(double) + sizeof(uint32_t));

// Shared by every call on a device and held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Per-device set-up cache: the device address of g_noalloc_scratch (the host
// symbol is only a stand-in and must never be passed to a kernel) and the
// SM count.  Filled by the first call on each device.
constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_dev_ptr[kNoAllocMaxDevices];
static int g_noalloc_sms[kNoAllocMaxDevices];

static int noalloc_setup(int dev)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(FPIC_EINVAL, "fpic_push_noalloc: device id %d out of range", dev);
    if (g_noalloc_dev_ptr[dev]) return 0;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
        return set_error(FPIC_ECUDA, "fpic_push_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int sms = 0;
    FPIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g_noalloc_sms[dev] = sms;
    g_noalloc_dev_ptr[dev] = ptr;
    return 0;
}

}  // namespace fpic

extern "C" int fpic_push_noalloc(double M, double a, fpic_particles* p, const fpic_push_params* prm,
                                 fpic_push_stats* stats, void* stream)
{
    if (!p || !prm) return set_error(FPIC_EINVAL, "fpic_push_noalloc: NULL particles/params");
    if (!(M > 0.0) || !std::isfinite(M) || !(fabs(a) <= M))
        return set_error(FPIC_EINVAL, "fpic_push_noalloc: need M > 0 and |a| <= M");
    if (p->n < 0) return set_error(FPIC_EINVAL, "fpic_push_noalloc: n < 0");
    if (p->n > kNoAllocMax)
        return set_error(FPIC_EINVAL, "fpic_push_noalloc: n = %lld exceeds the fixed scratch capacity of %lld particles",
                         (long long)p->n, (long long)kNoAllocMax);
    if (!particles_ok(p, true)) return set_error(FPIC_EINVAL, "fpic_push_noalloc: a particle array is NULL");
    if (!(std::isfinite(prm->dt)) || prm->dt == 0.0) return set_error(FPIC_EINVAL, "fpic_push_noalloc: dt must be finite and nonzero");
    if (prm->scheme < FPIC_RK4 || prm->scheme > FPIC_HYB2) return set_error(FPIC_EINVAL, "fpic_push_noalloc: unknown scheme %d", prm->scheme);
    if (prm->scheme >= FPIC_HYB1 && prm->implicit != FPIC_IMR && prm->implicit != FPIC_HAM)
        return set_error(FPIC_EINVAL, "fpic_push_noalloc: implicit partner must be FPIC_IMR or FPIC_HAM");
    if (prm->max_iter < 1 || prm->max_iter > 255) return set_error(FPIC_EINVAL, "fpic_push_noalloc: max_iter must be in [1, 255]");
    if (!(prm->tol >= 0.0)) return set_error(FPIC_EINVAL, "fpic_push_noalloc: tol must be >= 0");
    if (prm->guess) return set_error(FPIC_EINVAL, "fpic_push_noalloc: learned guesses are not supported here");
    int dev = 0;
    FPIC_CUDA(cudaGetDevice(&dev));
    int rc = noalloc_setup(dev);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    unsigned char* base = (unsigned char*)g_noalloc_dev_ptr[dev];
    PushK k{};
    k.bh = BH{M, a, a * a, 2.0 * M};
    k.has_grid = 0;
    k.has_fields = 0;
    k.dt = prm->dt;
    k.thr = prm->thr;
    k.tol = prm->tol;
    k.dg_eps = prm->dg_eps;
    k.B0pot = prm->B0pot;
    k.r_h = M + sqrt(M * M - a * a);
    k.r_max = prm->r_max;
    k.scheme = prm->scheme;
    k.max_iter = prm->max_iter;
    k.n = n;
    k.P = PartDev{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                  p->alive, p->scheme, p->iters, p->cell};
    k.cnt = (long long*)base;
    k.guess = (double*)(base + kNoAllocCountersBytes);
    k.queue = (uint32_t*)(base + kNoAllocCountersBytes + (size_t)n * 6 * sizeof(double));
    k.learned = nullptr;
    // the counters (queue length and head among them) must start at zero
    FPIC_CUDA(cudaMemsetAsync(k.cnt, 0, CNT_N * sizeof(long long), s));
    if (n == 0) {
        if (stats) *stats = fpic_push_stats{};
        return FPIC_OK;
    }
    const int TB = 128;
    const unsigned nb = (unsigned)((n + TB - 1) / TB);
    const unsigned persist = (unsigned)g_noalloc_sms[dev] * 8u;
    cudaEvent_t* ev = prm->events ? (cudaEvent_t*)prm->events : nullptr;
    if (stats) k_count_alive<<<persist, 256, 0, s>>>(k.P, n, k.cnt);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[0], s));
    if (prm->scheme == FPIC_RK4) k_explicit<0><<<nb, TB, 0, s>>>(k);
    else if (prm->scheme >= FPIC_HYB1) k_explicit<1><<<nb, TB, 0, s>>>(k);
    if (ev) {
        FPIC_CUDA(cudaEventRecord(ev[1], s));
        FPIC_CUDA(cudaEventRecord(ev[2], s));
    }
    if (prm->scheme == FPIC_IMR) k_imr<<<persist, TB, 0, s>>>(k, 1);
    else if (prm->scheme == FPIC_HAM) k_dg<<<nb, TB, 0, s>>>(k, 1);
    else if (prm->scheme >= FPIC_HYB1 && prm->implicit == FPIC_IMR) k_imr<<<persist, TB, 0, s>>>(k, 0);
    else if (prm->scheme >= FPIC_HYB1) k_dg<<<nb, TB, 0, s>>>(k, 0);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[3], s));
    FPIC_CUDA(cudaGetLastError());
    if (stats) {
        long long h[CNT_N];
        FPIC_CUDA(cudaMemcpyAsync(h, k.cnt, sizeof h, cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        const bool explicit_pass = prm->scheme == FPIC_RK4 || prm->scheme >= FPIC_HYB1;
        stats->n_alive_before = h[CNT_ALIVE];
        stats->n_implicit = prm->scheme == FPIC_RK4 ? 0 : (prm->scheme >= FPIC_HYB1 ? h[CNT_QUEUE] : h[CNT_ALIVE]);
        stats->n_iter_total = h[CNT_ITERS];
        stats->n_notconv = h[CNT_NOTCONV];
        stats->n_removed = h[CNT_REMOVED];
        stats->n_rhs_evals = h[CNT_EVALS] + (explicit_pass ? 4 * h[CNT_ALIVE] : 0);
        if (h[CNT_NOTCONV] > 0) return FPIC_ENOTCONVERGED;
    }
    return FPIC_OK;
}
