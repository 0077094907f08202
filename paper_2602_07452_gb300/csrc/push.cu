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
#include <cuda.h>
#include <limits.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "fpic_internal.h"
#include "mlp_dev.cuh"

namespace fpic {

struct PartDev {
    double *r, *th, *ph, *ur, *uth, *uph, *qm, *H0, *D0, *Hn;
    uint8_t *alive, *scheme, *iters;
    uint32_t* cell;
};

// Parameters of one spacetime / grid / field set (one run of a batch).
struct RunK {
    BH bh;
    GridDev G;
    Fields F;
    int has_fields;
    int has_grid;
    double B0pot, r_h, r_max;
    double B0field;           // analytic Wald field (no grid fields): its B0, else 0
    FieldsC FC;               // per-cell interpolation coefficients of F (has_coef)
    int has_coef;
    long long begin, end;     // particle range of the run (batched push)
};

struct PushK {
    RunK run;
    const RunK* runs;       // batched push: run table (nruns > 0), particle ranges [begin, end)
    int nruns;
    double dt, thr, tol, dg_eps;
    double d6, thr_dt, imp_ratio;   // dt / 6, thr dt and dt_imp / dt, formed once on the host
    double dt_imp;          // step of the implicit solves (the hybrid's partner: fpic_push_params.dt_implicit)
    int imr_newton;         // IMR iteration: Newton form (fpic_push_params.imr_newton)
    double* t;              // nullable per-particle time, advanced by the step each particle took
    // particle arrays in host memory (read over the link): the implicit pass
    // works from device copies by queue slot of z^n, q/m, H^n and D_0 (9 x n)
    // and of the iteration counts (n bytes); both null for device-resident
    // particles
    double* z0s;
    uint8_t* its;
    int count_alive;        // the explicit pass also counts the alive particles (stats)
    int scheme, max_iter;
    long long n;
    long long p_begin, p_end;   // explicit pass over [p_begin, p_end) (p_end 0: all n)
    PartDev P;
    PartDev before;         // fpic_push_params.before: r, th, ur, uth, uph, alive at the step's start (r null: off)
    double* guess;          // 6 x n (SoA) implicit initial guesses, then the implicit results
    double* sc0;            // 2 x n: sin, cos of th^n of the implicit particles
    uint32_t* queue;        // indices of particles for the implicit solver
    uint32_t* order;        // nullable: processing order of the queue slots (k_order)
    long long* cnt;
    const float* learned;   // n x 16 MLP outputs (nullable)
    // learned / sampling extensions
    uint32_t* work;         // explicit-pass work list (nullable: all particles)
    int record;             // sampling mode: write targets, leave the particles unchanged
    float* recT;            // n x 16 targets (sampling)
    float* recS;            // n labels (sampling)
    double inc_scale[6];    // scale of the implicit-step increments
    // corrector form of the learned guess (per implicit-queue slot)
    float* featX;           // 16 floats: trial features (network input)
    float* featS;           // 16 floats: scales s_i (0-5), leading-order gaps g_i (8-13)
    double* stg;            // STG_ROWS x n, by queue slot: see STG_* (corrector form)
    float fmean[14], fistd[14];
    float oscale[6];        // corrector outputs 0-5 are residual / (s_i oscale_i)
    int restart_after;      // corrector: restart from the trial after this many iterations (0: never)
    // field-tile staging (FPIC_TUNE_STAGE_FIELDS): six 2-D tensor maps of the
    // coefficient arrays (device memory, 64-byte aligned); null = off
    const uint8_t* stage_maps;
    // substeps of unconverged IMR solves (fpic_push_params.imr_substeps):
    // levels K (0 = off), H condition, and the list of the solves' queue
    // slots (particle indices in all_mode), CNT_STRAG entries
    int substeps;
    double substep_tol;
    uint32_t* strag;
    uint8_t* strag_flag;    // by queue slot: k_imr's solve did not converge
    // slope reuse (FPIC_TUNE_REUSE_SLOPE): SLOPE_ROWS x n, see SLOPE_*; null = off
    double* slope;
    int slope_cold;         // the cache holds nothing for these particles: do not look
};

// Per-push constants the kernels would otherwise divide for per particle
// (the same IEEE quotients, once).
static void push_constants(PushK& k)
{
    k.d6 = k.dt / 6.0;
    k.thr_dt = k.thr * k.dt;
    k.imp_ratio = k.dt_imp / k.dt;
}

// Rows of the slope cache: the state z^{n+1} and q/m it was computed for
// (the validity tag, compared bit for bit), F(z^{n+1}), sin and cos th^{n+1}.
enum { SLOPE_Z = 0, SLOPE_QM = 6, SLOPE_F = 7, SLOPE_S = 13, SLOPE_C = 14, SLOPE_ROWS = 15 };

__device__ __forceinline__ bool slope_valid(const PushK& k, long long p, const double z[6], double qm)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i)
        ok = ok && __double_as_longlong(__ldcs(k.slope + (size_t)(SLOPE_Z + i) * k.n + p)) == __double_as_longlong(z[i]);
    return ok && __double_as_longlong(__ldcs(k.slope + (size_t)SLOPE_QM * k.n + p)) == __double_as_longlong(qm);
}

__device__ __forceinline__ void slope_store(const PushK& k, long long p, const double z[6], double qm,
                                            const double f[6], double s, double c)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        __stcs(k.slope + (size_t)(SLOPE_Z + i) * k.n + p, z[i]);
        __stcs(k.slope + (size_t)(SLOPE_F + i) * k.n + p, f[i]);
    }
    __stcs(k.slope + (size_t)SLOPE_QM * k.n + p, qm);
    __stcs(k.slope + (size_t)SLOPE_S * k.n + p, s);
    __stcs(k.slope + (size_t)SLOPE_C * k.n + p, c);
}

// Invalidates a particle's cache entry (its tag can no longer match a state).
__device__ __forceinline__ void slope_drop(const PushK& k, long long p)
{
    __stcs(k.slope + (size_t)SLOPE_Z * k.n + p, __longlong_as_double(0x7ff8dead0000dead));
}

// Run of particle p in a batched push (runs sorted by begin).
__device__ __forceinline__ int run_of(const RunK* __restrict__ runs, int nruns, long long p)
{
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (runs[mid].begin <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

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
    const float lr = __logf(f32_est(r));
    double tnv, thv;
    int mh;
    theta_views(G, th, tnv, thv, mh);
    locate(G.rn, G.irn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i, w);
    locate(G.tn, G.itn, G.Nth + 1, tnv, (f32_est(tnv) - G.t0) * G.it, j, w);
    return (uint32_t)i * (uint32_t)G.Nth + (uint32_t)j;
}

// Right-hand side at y: gathers the fields when the particle is charged.
__device__ __forceinline__ void F_at(const RunK& R, const double y[6], double qm, bool em,
                                     double f[6], double& H)
{
    double D[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    if (em) {
        if (R.has_coef) gather_c(R.G, R.FC, y[0], y[1], D, B);
        else gather(R.G, R.F, y[0], y[1], D, B);
    }
    eval_rhs(R.bh, y, qm, em, D, B, R.B0pot, f, H);
}

// Same, with sin/cos of y[1] supplied (from sincos_near).  STAGED: the
// coefficient gather looks in the block's staged field tile T first.
template <bool JAC = false, bool STAGED = false>
__device__ __forceinline__ void F_at_sc(const RunK& R, const double y[6], double s, double c, double qm, bool em,
                                        double f[6], double& H, RhsJ* J = nullptr, const StageTile* T = nullptr)
{
    double D[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    if (em) {
        if (R.B0field != 0.0) wald_point_sc(R.bh, R.B0field, y[0], s, c, D, B);
        else if (STAGED && R.has_coef) gather_c(R.G, R.FC, y[0], y[1], D, B, *T);
        else if (R.has_coef) gather_c(R.G, R.FC, y[0], y[1], D, B);
        else gather(R.G, R.F, y[0], y[1], D, B);
    }
    eval_rhs_sc_t<JAC>(R.bh, y, s, c, qm, em, D, B, R.B0pot, f, H, J);
}

// Bounded waits of the field-tile staging (polls of the mbarrier).
constexpr uint32_t STAGE_WAIT_POLLS = 1u << 22;

// Block prologue of a staged push (every thread of the block calls it).
// The block's alive particles are sorted by cell; the cells their last push
// or sort left in P.cell give the block's range of coefficient cells, and
// if the tile around it (one cell of margin for the RK4 stages' motion, one
// more for the half-node sub-grids) fits STAGE_TI x STAGE_TJ, one thread
// loads the six components' tiles into shared memory with TMA.  P.cell only
// steers the choice of tile: a gather outside the tile reads global memory.
__device__ __forceinline__ StageTile stage_fields(const PushK& k, long long p, bool valid, double* s_coef,
                                                  uint64_t* mbar, int* s_red)
{
    const uint32_t Nth = (uint32_t)k.run.G.Nth;
    int imin = INT_MAX, imax = INT_MIN, jmin = INT_MAX, jmax = INT_MIN;
    if (valid && k.P.alive[p]) {
        const uint32_t cell = k.P.cell[p];
        imin = imax = (int)(cell / Nth);
        jmin = jmax = (int)(cell % Nth);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        imin = min(imin, __shfl_xor_sync(0xffffffffu, imin, o));
        imax = max(imax, __shfl_xor_sync(0xffffffffu, imax, o));
        jmin = min(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
        jmax = max(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_red[4 * warp + 0] = imin;
        s_red[4 * warp + 1] = imax;
        s_red[4 * warp + 2] = jmin;
        s_red[4 * warp + 3] = jmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            imin = min(imin, s_red[4 * w + 0]);
            imax = max(imax, s_red[4 * w + 1]);
            jmin = min(jmin, s_red[4 * w + 2]);
            jmax = max(jmax, s_red[4 * w + 3]);
        }
        const int ok = imax >= imin && imax - imin + 4 <= STAGE_TI && jmax - jmin + 4 <= STAGE_TJ;
        const int i0 = imin - 2, j0 = jmin - 2;
        if (ok) {
            tc::mbar_init(mbar, 1);
            tc::mbar_arrive_expect_tx(mbar, 6u * STAGE_TI * STAGE_TJ * 4u * 8u);
#pragma unroll
            for (int c = 0; c < 6; ++c)
                tc::tma_load_2d(s_coef + c * STAGE_TI * STAGE_TJ * 4, k.stage_maps + 128 * c, 4 * j0, i0, mbar);
        }
        s_red[4 * nw + 0] = ok;
        s_red[4 * nw + 1] = i0;
        s_red[4 * nw + 2] = j0;
        if (ok) atomicAdd((unsigned long long*)&k.cnt[CNT_STAGED], 1ull);
    }
    __syncthreads();
    StageTile T{nullptr, s_red[4 * nw + 1], s_red[4 * nw + 2]};
    if (s_red[4 * nw + 0]) {
        if (tc::mbar_wait(mbar, 0, STAGE_WAIT_POLLS)) {
            T.s = s_coef;
        } else {
            // the copies did not land in time: count it, give them one more
            // bounded wait (the shared memory must not be left to a later
            // block while they are in flight) and read global memory
            atomicAdd((unsigned long long*)&k.cnt[CNT_ERR], 1ull);
            tc::mbar_wait(mbar, 0, STAGE_WAIT_POLLS);
        }
    }
    return T;
}

// Newton form of the implicit-midpoint iteration (Sec. 2.2.2 names a Newton
// scheme): with zp = z^n + h F(y) the fixed-point update at the midpoint y
// of z^n and the current iterate zk, the Newton matrix 1 - (h/2) dF keeps
// the momentum columns of dF,
//   A_il = d(dx^i/dt)/du_l = (alpha / Gamma) (g^il - u^i u^l / Gamma^2),
//   J_il = d(du_i/dt)/du_l = ks ((g^{.l} x B)_i - (u x B)_i u^l / Gamma^2)
// (the magnetic force; ks = qm alpha sqrt(gamma) / Gamma), and the step is
//   (1 - (h/2) J) du = u_k - u_p,  u_new = u_k - du,  x_new = x_p - (h/2) A du.
// The 3 x 3 system is solved by Cramer's rule.  Same fixed point as the
// plain update, fewer iterations where the gyration dominates.
__device__ __forceinline__ void newton_update(const RhsJ& J, double hh, const double zk[6], double zn[6])
{
    const double w = hh * J.ks;
    const double wB0 = w * J.B[0], wB1 = w * J.B[1], wB2 = w * J.B[2];
    const double w2 = w * (J.iG * J.iG);
    const double c0 = w2 * J.cx[0], c1 = w2 * J.cx[1], c2 = w2 * J.cx[2];
    // M = 1 - w X + w2 (u x B) u^T, X's columns g^{.l} x B
    const double m00 = fma(c0, J.U[0], fma(J.gurp, wB1, 1.0));
    const double m01 = fma(c0, J.U[1], -J.gutt * wB2);
    const double m02 = fma(c0, J.U[2], J.gupp * wB1);
    const double m10 = fma(c1, J.U[0], fma(J.gurr, wB2, -J.gurp * wB0));
    const double m11 = fma(c1, J.U[1], 1.0);
    const double m12 = fma(c1, J.U[2], fma(J.gurp, wB2, -J.gupp * wB0));
    const double m20 = fma(c2, J.U[0], -J.gurr * wB1);
    const double m21 = fma(c2, J.U[1], J.gutt * wB0);
    const double m22 = fma(c2, J.U[2], fma(-J.gurp, wB1, 1.0));
    const double b0 = zk[3] - zn[3], b1 = zk[4] - zn[4], b2 = zk[5] - zn[5];
    const double a00 = fma(m11, m22, -m12 * m21), a01 = fma(m02, m21, -m01 * m22), a02 = fma(m01, m12, -m02 * m11);
    const double a10 = fma(m12, m20, -m10 * m22), a11 = fma(m00, m22, -m02 * m20), a12 = fma(m02, m10, -m00 * m12);
    const double a20 = fma(m10, m21, -m11 * m20), a21 = fma(m01, m20, -m00 * m21), a22 = fma(m00, m11, -m01 * m10);
    const double idet = rcp_nr(fma(m00, a00, fma(m01, a10, m02 * a20)));
    const double d0 = idet * fma(a00, b0, fma(a01, b1, a02 * b2));
    const double d1 = idet * fma(a10, b0, fma(a11, b1, a12 * b2));
    const double d2 = idet * fma(a20, b0, fma(a21, b1, a22 * b2));
    zn[3] = zk[3] - d0;
    zn[4] = zk[4] - d1;
    zn[5] = zk[5] - d2;
    // A du = (alpha / Gamma) (g^-1 du - u (u . du) / Gamma^2)
    const double ud = fma(J.U[0], d0, fma(J.U[1], d1, J.U[2] * d2)) * (J.iG * J.iG);
    const double ha = hh * J.aiG;
    zn[0] = fma(-ha, fma(J.gurr, d0, fma(J.gurp, d2, -J.U[0] * ud)), zn[0]);
    zn[1] = fma(-ha, fma(J.gutt, d1, -J.U[1] * ud), zn[1]);
    zn[2] = fma(-ha, fma(J.gurp, d0, fma(J.gupp, d2, -J.U[2] * ud)), zn[2]);
}

// Particle boundaries (Sec. 2.5) and write-back of a finished step.
// Particle boundary in th (Sec. 2.5): half-theta domain, reflection at the
// poles (reading: th -> -th or 2 pi - th, u_th -> -u_th, ph -> ph + pi);
// full-theta domain, periodic (th wrapped into [tn[0], tn[0] + P), nothing
// else changes).
static __device__ __noinline__ double theta_period_wrap(double th, double tlo, double tper)
{
    th = th < tlo ? th + tper : th;
    return th >= tlo + tper ? th - tper : th;
}

__device__ __forceinline__ void theta_boundary(const GridDev& G, double z[6])
{
    if (G.full) {
        z[1] = theta_period_wrap(z[1], G.tlo, G.tper);
    } else if (z[1] < 0.0) {
        z[1] = -z[1];
        z[4] = -z[4];
        z[2] += M_PI;
    } else if (z[1] > M_PI) {
        z[1] = 2.0 * M_PI - z[1];
        z[4] = -z[4];
        z[2] += M_PI;
    }
}

__device__ __forceinline__ bool finish(const RunK& R, const PartDev& P, long long p, double z[6], double H,
                                       int implicit, int iters)
{
    theta_boundary(R.G, z);
    const bool alive = (z[0] >= R.r_h) && (z[0] <= R.r_max);
    store_state(P, p, z);
    P.Hn[p] = H;
    P.scheme[p] = (uint8_t)implicit;
    P.iters[p] = (uint8_t)min(iters, 255);
    P.alive[p] = alive ? 1 : 0;
    if (P.cell) P.cell[p] = R.has_grid ? cell_of(R.G, z[0], z[1]) : 0u;
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

// Rows of the corrector form's slot-indexed scratch stg (6 each): the RK4
// slopes k1, k2, acc = k1 + 2 k2 + 2 k3, k4, the state z^n, the trial
// z_RK4, and the corrected implicit guess.
enum { STG_K1 = 0, STG_K2 = 6, STG_ACC = 12, STG_K4 = 18, STG_Z0 = 24, STG_TRIAL = 30, STG_GUESS = 36,
       STG_ROWS = 42 };

// Corrector form, rejected particle in queue slot idx: its slopes k1, k2
// (kept in shared memory, column threadIdx.x), acc, k4, z^n and the trial go
// to stg at column idx (a warp's rejected lanes hold consecutive slots, so
// the stores coalesce).  Plain copies: the arithmetic on them runs where
// every lane of a warp has a queue entry, and every later read is
// slot-ordered.
__device__ __forceinline__ void trial_store(const PushK& k, unsigned long long idx, const double (*sk)[128],
                                            const double acc[6], const double k4[6], const double z0[6],
                                            const double zt[6])
{
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        k.stg[(size_t)(STG_K1 + i) * k.n + idx] = sk[i][t];
        k.stg[(size_t)(STG_K2 + i) * k.n + idx] = sk[6 + i][t];
        k.stg[(size_t)(STG_ACC + i) * k.n + idx] = acc[i];
        k.stg[(size_t)(STG_K4 + i) * k.n + idx] = k4[i];
        k.stg[(size_t)(STG_Z0 + i) * k.n + idx] = z0[i];
        k.stg[(size_t)(STG_TRIAL + i) * k.n + idx] = zt[i];
    }
}

// MODE 0: RK4 only.  MODE 1: hybrid (RK4 trial + test + enqueue).  MODE 2:
// hybrid that also parks the RK4 slopes of each rejected particle
// (corrector form of the learned guess); k1, k2 wait in shared memory
// (12 KB per block) rather than in registers across the later stages.
template <int MODE, bool BATCHED = false, bool STAGED = false>
__global__ void __launch_bounds__(128) k_explicit(const __grid_constant__ PushK k)
{
    __shared__ double sk[MODE == 2 ? 12 : 1][128];
    __shared__ __align__(128) double s_coef[STAGED ? 6 * STAGE_TI * STAGE_TJ * 4 : 2];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_red[4 * 4 + 4];
    const long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long p = k.p_begin + w;
    StageTile tile{nullptr, 0, 0};
    if (STAGED) tile = stage_fields(k, p, p < (k.p_end ? k.p_end : k.n), s_coef, &s_mbar, s_red);
    if (k.work) {
        if (w >= k.cnt[CNT_WORK]) return;
        p = k.work[w];
    } else if (p >= (k.p_end ? k.p_end : k.n)) {
        return;
    }
    if (k.count_alive) {
        const unsigned act = __activemask();
        const unsigned al = __ballot_sync(act, k.P.alive[p] != 0);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1)
            atomicAdd((unsigned long long*)&k.cnt[CNT_ALIVE], (unsigned long long)__popc(al));
    }
    const uint8_t alive0 = k.P.alive[p];
    if (k.before.r) k.before.alive[p] = alive0;
    if (!alive0) {
        k.P.scheme[p] = 0;
        k.P.iters[p] = 0;
        return;
    }
    const RunK& R = BATCHED ? k.runs[run_of(k.runs, k.nruns, p)] : k.run;
    double z0[6], kk[6], acc[6], y[6];
    load_state(k.P, p, z0);
    if (k.before.r) {
        k.before.r[p] = z0[0];
        k.before.th[p] = z0[1];
        k.before.ur[p] = z0[3];
        k.before.uth[p] = z0[4];
        k.before.uph[p] = z0[5];
    }
    const double qm = k.P.qm[p];
    const bool em = (R.has_fields || R.B0field != 0.0) && qm != 0.0;
    const double dt = k.dt, hdt = 0.5 * k.dt;
    double Hd, s0, c0, sn, cn;
    // k1 = F(z^n): from the slope cache when this particle's state is the
    // one stored there, else evaluated
    const bool reuse = !BATCHED && k.slope && !k.slope_cold && slope_valid(k, p, z0, qm);
    if (!BATCHED && k.slope) {
        const unsigned act = __activemask();
        const unsigned rm = __ballot_sync(act, reuse);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1 && rm)
            atomicAdd((unsigned long long*)&k.cnt[CNT_SLOPE], (unsigned long long)__popc(rm));
    }
    if (reuse) {
#pragma unroll
        for (int i = 0; i < 6; ++i) kk[i] = __ldcs(k.slope + (size_t)(SLOPE_F + i) * k.n + p);
        s0 = __ldcs(k.slope + (size_t)SLOPE_S * k.n + p);
        c0 = __ldcs(k.slope + (size_t)SLOPE_C * k.n + p);
    } else {
        sincos(z0[1], &s0, &c0);
        F_at_sc<false, STAGED>(R, z0, s0, c0, qm, em, kk, Hd, nullptr, &tile);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        acc[i] = kk[i];
        y[i] = fma(hdt, kk[i], z0[i]);
        if (MODE == 2) sk[i][threadIdx.x] = kk[i];
    }
    sincos_near(z0[1], s0, c0, y[1], sn, cn);
    F_at_sc<false, STAGED>(R, y, sn, cn, qm, em, kk, Hd, nullptr, &tile);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        acc[i] = fma(2.0, kk[i], acc[i]);
        y[i] = fma(hdt, kk[i], z0[i]);
        if (MODE == 2) sk[6 + i][threadIdx.x] = kk[i];
    }
    sincos_near(z0[1], s0, c0, y[1], sn, cn);
    F_at_sc<false, STAGED>(R, y, sn, cn, qm, em, kk, Hd, nullptr, &tile);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = fma(2.0, kk[i], acc[i]); y[i] = fma(dt, kk[i], z0[i]); }
    sincos_near(z0[1], s0, c0, y[1], sn, cn);
    F_at_sc<false, STAGED>(R, y, sn, cn, qm, em, kk, Hd, nullptr, &tile);
    const double d6 = k.d6;
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = fma(d6, acc[i] + kk[i], z0[i]);
    sincos_near(z0[1], s0, c0, y[1], sn, cn);
    // H of the trial; with the slope cache the whole right-hand side at the
    // trial point, kept for the next step if the trial is accepted
    double H1, fy[6];
    const bool keep = !BATCHED && k.slope && !k.record;
    if (keep) F_at_sc<false, STAGED>(R, y, sn, cn, qm, em, fy, H1, nullptr, &tile);
    else H1 = eval_H_sc(R.bh, y, sn, cn, qm, R.B0pot);
    bool accept = true;
    double Hn0 = 0.0, D00 = 1.0;     // H^n and D_0, kept for the stash of a rejected particle
    if (MODE >= 1) {
        // Hyb2: Ht^{n+1} = |H1 - H0| / D0 < thr; Hyb1: (Ht^{n+1} - Ht^n) / dt
        // < thr.  With D0, dt > 0 both are taken as products,
        // |H1 - H0| < thr D0 and |H1 - H0| - |H^n - H0| < (thr dt) D0: the
        // same decisions up to the rounding of the quotients, without three
        // FP64 divisions per particle.
        const double H0 = k.P.H0[p], D0 = k.P.D0[p];
        const double e1 = fabs(H1 - H0);
        D00 = D0;
        if (k.scheme == FPIC_HYB2) {
            accept = e1 < k.thr * D0;
            if (!accept && k.z0s) Hn0 = k.P.Hn[p];
        } else {
            Hn0 = k.P.Hn[p];
            accept = e1 - fabs(Hn0 - H0) < k.thr_dt * D0;
        }
    }
    const float label = accept ? 0.f : 1.f;
    if (k.record) {                 // sampling: label, then every particle goes implicit
        if (MODE != 2) k.recS[p] = label;
        accept = false;
    }
    const unsigned act = __activemask();
    const unsigned rej = __ballot_sync(act, !accept);
    if (accept) {
        const double th_trial = y[1];
        const bool alive = finish(R, k.P, p, y, H1, 0, 0);
        if (!alive) atomicAdd((unsigned long long*)&k.cnt[CNT_REMOVED], 1ull);
        if (k.t) k.t[p] += dt;
        if (keep && alive) {
            if (y[1] != th_trial && !R.G.full) {   // reflected at a pole: the slope of the stored state
                sn = -sn;                              // (a full-theta wrap changes neither F nor sin/cos)
                F_at_sc<false, STAGED>(R, y, sn, cn, qm, em, fy, Hd, nullptr, &tile);
            }
            slope_store(k, p, y, qm, fy, sn, cn);
        }
    } else if (keep) {
        slope_drop(k, p);                 // the implicit partner sets its own entry, if any
    }
    if (rej) {
        const int leader = __ffs(act) - 1;
        unsigned long long base = 0;
        if ((int)(threadIdx.x & 31) == leader)
            base = atomicAdd((unsigned long long*)&k.cnt[CNT_QUEUE], (unsigned long long)__popc(rej));
        base = __shfl_sync(act, base, leader);
        if (!accept) {
            const unsigned long long idx = base + __popc(rej & lanemask_lt());
            k.queue[idx] = (uint32_t)p;
            if (k.dt_imp == dt) {
#pragma unroll
                for (int i = 0; i < 6; ++i) k.guess[(size_t)i * k.n + p] = y[i];
            } else {
                // adaptive step: the trial's increment scaled to the implicit step
                // (rounded product, then sum: the same value as the plain C form)
                const double ratio = k.imp_ratio;
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    k.guess[(size_t)i * k.n + p] = __dadd_rn(z0[i], __dmul_rn(__dsub_rn(y[i], z0[i]), ratio));
            }
            k.sc0[p] = s0;
            k.sc0[k.n + p] = c0;
            if (k.z0s) {
#pragma unroll
                for (int i = 0; i < 6; ++i) k.z0s[(size_t)i * k.n + idx] = z0[i];
                k.z0s[(size_t)6 * k.n + idx] = qm;
                k.z0s[(size_t)7 * k.n + idx] = Hn0;
                k.z0s[(size_t)8 * k.n + idx] = D00;
            }
            if (MODE == 2) {
                trial_store(k, idx, sk, acc, kk, z0, y);
                if (k.record) k.recS[idx] = label;
            }
        }
    }
}

__device__ __forceinline__ bool conv6(const double a[6], const double b[6], double tol)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) ok = ok && le_nonneg(fabs(a[i] - b[i]), tol * (fabs(a[i]) + 1.0));
    return ok;
}

// Processing order of the implicit queue: slots of particles within
// AXIS_PRIORITY_TH of the polar axis first.  Near the axis the u_ph^2 /
// sin^3 th terms make the Picard iteration contract slowly or cycle (the
// solves that run to max_iter are found there), so starting them first lets
// their long solves overlap the bulk instead of trailing it.  The order only
// decides which lane takes which particle; every particle's arithmetic, and
// hence its result, is the same.
constexpr double AXIS_PRIORITY_TH = 0.01;
__global__ void k_order(PushK k)
{
    const long long qn = k.cnt[CNT_QUEUE];
    for (long long slot = blockIdx.x * (long long)blockDim.x + threadIdx.x; slot < qn;
         slot += (long long)gridDim.x * blockDim.x) {
        // host-resident particles: from the device stash, not over the link
        const double th = k.z0s ? k.z0s[(size_t)1 * k.n + slot] : k.P.th[k.queue[slot]];
        const bool prio = th < AXIS_PRIORITY_TH || th > M_PI - AXIS_PRIORITY_TH;
        const unsigned act = __activemask();
        const unsigned pm = __ballot_sync(act, prio);
        const int leader = __ffs(act) - 1;
        unsigned long long bp = 0, bn = 0;
        if ((int)(threadIdx.x & 31) == leader) {
            if (pm) bp = atomicAdd((unsigned long long*)&k.cnt[CNT_PRIO], (unsigned long long)__popc(pm));
            const unsigned nn = __popc(act & ~pm);
            if (nn) bn = atomicAdd((unsigned long long*)&k.cnt[CNT_NORM], (unsigned long long)nn);
        }
        bp = __shfl_sync(act, bp, leader);
        bn = __shfl_sync(act, bn, leader);
        const unsigned below = lanemask_lt();
        // priority slots fill the order from the front, the others from the back
        const long long pos = prio ? (long long)(bp + __popc(pm & below))
                                   : qn - 1 - (long long)(bn + __popc(act & ~pm & below));
        k.order[pos] = (uint32_t)slot;
    }
}

// Persistent lane-refilling implicit-midpoint solver (Sec. 2.2.2):
// z^[k] = z^n + dt F((z^n + z^[k-1]) / 2) until two iterates agree to tol.
// NEWTON: the Newton form of the same iteration (newton_update), which also
// stops, from the second iteration on, when each component's a-posteriori
// error bound theta_i / (1 - theta_i) |dz_i| (theta_i the ratio of its last
// two updates) passes the tolerance.
// all_mode: the queue is every particle (pure IMR, guess z^n); otherwise
// entries come from k_explicit with their trial and sin/cos of th^n (sc0).
// Each loop trip is one right-hand side per lane; a lane whose solve ends
// parks the result in the guess slot and takes the next particle at once.
// H at the converged point and the write-back run afterwards in
// k_imr_finish (one thread per particle, no lane waits on them here).
// RESTART 1 (corrector form of the learned guess): the start is the
// corrected guess of the queue slot (stg); with k.restart_after > 0, a solve
// that has not converged after that many iterations from it restarts once,
// with the full max_iter budget, from the trial in stg.
template <int RESTART, bool BATCHED = false, bool NEWTON = false>
__global__ void __launch_bounds__(128, NEWTON ? 3 : 4) k_imr(const __grid_constant__ PushK k, int all_mode)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long qn = all_mode ? k.n : k.cnt[CNT_QUEUE];
    const RunK* R = &k.run;
    long long p = -1, qi = 0;
    bool exhausted = false, again = false;
    double z0[6], zk[6];
    // the smallest update so far and its iteration: a solve that reaches
    // max_iter replays its iterations from the start up to that one (the
    // sequence is deterministic) and returns that iterate
    double best_dz = INFINITY;
    int best_it = 0, replay_to = 0;
    double dprev[6];        // the previous iteration's |update| per component (a-posteriori stop)
    double qm = 0.0, s0 = 0.0, c0 = 1.0;
    bool em = false;
    int it = 0;
    long long n_it = 0, n_nc = 0, n_ev = 0;
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
                    const long long slot = (!all_mode && k.order) ? (long long)k.order[idx] : idx;
                    const long long q = all_mode ? idx : (long long)k.queue[slot];
                    if (all_mode && !k.P.alive[q]) {
                        k.P.scheme[q] = 0;
                        k.P.iters[q] = 0;
                    } else {
                        p = q;
                        qi = slot;
                        if (BATCHED) R = k.runs + run_of(k.runs, k.nruns, p);
                        again = RESTART != 0;
                        if (!all_mode && k.z0s) {
#pragma unroll
                            for (int i = 0; i < 6; ++i) z0[i] = k.z0s[(size_t)i * k.n + slot];
                        } else {
                            load_state(k.P, p, z0);
                        }
                        if (all_mode) {
                            sincos(z0[1], &s0, &c0);
                            k.sc0[p] = s0;
                            k.sc0[k.n + p] = c0;
#pragma unroll
                            for (int i = 0; i < 6; ++i) zk[i] = z0[i];
                        } else {
                            s0 = k.sc0[p];
                            c0 = k.sc0[k.n + p];
#pragma unroll
                            for (int i = 0; i < 6; ++i)
                                zk[i] = RESTART ? k.stg[(size_t)(STG_GUESS + i) * k.n + slot]
                                                : k.guess[(size_t)i * k.n + p];
                        }
                        qm = (!all_mode && k.z0s) ? k.z0s[(size_t)6 * k.n + slot] : k.P.qm[p];
                        em = (R->has_fields || R->B0field != 0.0) && qm != 0.0;
                        it = 0;
                        best_dz = INFINITY;
                        best_it = 0;
                        replay_to = 0;
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
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] = 0.5 * (z0[i] + zk[i]);
            double sy, cy;
            sincos_near(z0[1], s0, c0, y[1], sy, cy);
            RhsJ J;
            F_at_sc<NEWTON>(*R, y, sy, cy, qm, em, f, H, &J);
            ++n_ev;
            double zn[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) zn[i] = fma(k.dt_imp, f[i], z0[i]);
            if (NEWTON) newton_update(J, 0.5 * k.dt_imp, zk, zn);
            bool done = false, conv = false;
            if (replay_to) {
                // replaying an unconverged solve up to its smallest-update iterate
#pragma unroll
                for (int i = 0; i < 6; ++i) zk[i] = zn[i];
                if (++it < replay_to) continue;
                done = true;
            } else {
                double di[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) di[i] = fabs(zn[i] - zk[i]);
                bool ok = true;
#pragma unroll
                for (int i = 0; i < 6; ++i) ok = ok && le_nonneg(di[i], k.tol * (fabs(zn[i]) + 1.0));
                if (NEWTON && !ok && it >= 1) {
                    // a-posteriori stop: theta_i / (1 - theta_i) d_i <= tol (|z_i| + 1),
                    // theta_i = d_i / p_i, written without division
                    ok = true;
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        ok = ok && lt_nonneg(di[i], dprev[i]) &&
                             le_nonneg(di[i] * di[i], k.tol * (fabs(zn[i]) + 1.0) * (dprev[i] - di[i]));
                }
                double dz = 0.0;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    dz = fmax_nonneg(dz, di[i]);
                    dprev[i] = di[i];
                }
                if (lt_nonneg(dz, best_dz)) {
                    best_dz = dz;
                    best_it = it + 1;
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) zk[i] = zn[i];
                ++it;
                if (RESTART && !ok && k.restart_after > 0 && it >= min(k.max_iter, k.restart_after) && again) {
                    // the corrected start did not converge: the plain trial is the fallback
                    again = false;
                    n_it += it;
                    it = 0;
                    best_dz = INFINITY;
                    best_it = 0;
#pragma unroll
                    for (int i = 0; i < 6; ++i) zk[i] = k.stg[(size_t)(STG_TRIAL + i) * k.n + qi];
                } else if (ok) {
                    done = conv = true;
                } else if (it >= k.max_iter) {
                    // not converged (Sec. 2.2.2 gives no policy): the iterate with
                    // the smallest update, the last one or one replayed from the start
                    n_it += it;
                    if (best_it == it) {
                        done = true;
                    } else {
                        replay_to = best_it;
                        it = 0;
#pragma unroll
                        for (int i = 0; i < 6; ++i)
                            zk[i] = all_mode ? z0[i]
                                  : RESTART ? k.stg[(size_t)((again ? STG_GUESS : STG_TRIAL) + i) * k.n + qi]
                                            : k.guess[(size_t)i * k.n + p];
                    }
                }
            }
            if (done) {
                const int its_done = conv ? it : k.max_iter;
                if (conv) n_it += it;
                else ++n_nc;
                if (!conv && k.substeps > 0 && !k.record) k.strag_flag[qi] = 1;
                if (k.record && k.featS) {
                    // corrector form: row = queue slot, (gap to the trial - leading-order gap) / (s_i oscale_i)
                    float* t = k.recT + 16 * qi;
                    const float* sc = k.featS + 16 * qi;
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        const double g = (zk[i] - k.guess[(size_t)i * k.n + p] - (double)sc[8 + i]) /
                                         ((double)sc[i] * (double)k.oscale[i]);
                        t[i] = sc[i] > 0.f ? (float)fmin(4.0, fmax(-4.0, g)) : 0.f;
                    }
                    t[6] = 0.f;
                    t[7] = (float)(its_done - 8) * 0.25f;
                    t[8] = 0.f;
                } else if (k.record) {
                    float* t = k.recT + 16 * p;
#pragma unroll
                    for (int i = 0; i < 6; ++i) t[i] = (float)((zk[i] - z0[i]) / k.inc_scale[i]);
                    t[6] = 0.f;
                    t[7] = (float)(its_done - 8) * 0.25f;
                    t[8] = 0.f;
                } else {
#pragma unroll
                    for (int i = 0; i < 6; ++i) k.guess[(size_t)i * k.n + p] = zk[i];
                    if (k.its && !all_mode) k.its[qi] = (uint8_t)min(its_done, 255);
                    else k.P.iters[p] = (uint8_t)min(its_done, 255);
                }
                p = -1;
            }
        }
    }
    warp_add(&k.cnt[CNT_ITERS], n_it, FULL);
    warp_add(&k.cnt[CNT_NOTCONV], n_nc, FULL);
    warp_add(&k.cnt[CNT_EVALS], n_ev, FULL);
}

// One implicit-midpoint solve of step h from zs (guess zs) by one thread,
// with k_imr's iteration and stop rule; true if it converged within
// max_iter (result in out), iterations added to its.
template <bool NEWTON>
__device__ bool imr_solve_serial(const PushK& k, const RunK& R, const double zs[6], double h, double qm, bool em,
                                 int max_iter, double out[6], long long& its, long long& evals)
{
    double ss, cs, zk[6], dprev[6];
    sincos(zs[1], &ss, &cs);
#pragma unroll
    for (int i = 0; i < 6; ++i) zk[i] = zs[i];
    for (int it = 0; it < max_iter; ++it) {
        double y[6], f[6], H, zn[6], sy, cy;
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] = 0.5 * (zs[i] + zk[i]);
        sincos_near(zs[1], ss, cs, y[1], sy, cy);
        RhsJ J;
        F_at_sc<NEWTON>(R, y, sy, cy, qm, em, f, H, &J);
        ++evals;
#pragma unroll
        for (int i = 0; i < 6; ++i) zn[i] = fma(h, f[i], zs[i]);
        if (NEWTON) newton_update(J, 0.5 * h, zk, zn);
        double di[6];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            di[i] = fabs(zn[i] - zk[i]);
            ok = ok && le_nonneg(di[i], k.tol * (fabs(zn[i]) + 1.0));
        }
        if (NEWTON && !ok && it >= 1) {
            ok = true;
#pragma unroll
            for (int i = 0; i < 6; ++i)
                ok = ok && lt_nonneg(di[i], dprev[i]) &&
                     le_nonneg(di[i] * di[i], k.tol * (fabs(zn[i]) + 1.0) * (dprev[i] - di[i]));
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            dprev[i] = di[i];
            zk[i] = zn[i];
        }
        if (ok) {
            its += it + 1;
#pragma unroll
            for (int i = 0; i < 6; ++i) out[i] = zk[i];
            return true;
        }
    }
    its += max_iter;
    return false;
}

// Launch k_imr in the iteration form the push asked for (k.imr_newton).
template <int RESTART, bool BATCHED = false>
static void launch_imr(unsigned grid, unsigned block, cudaStream_t s, const PushK& k, int all_mode)
{
    if (k.imr_newton) k_imr<RESTART, BATCHED, true><<<grid, block, 0, s>>>(k, all_mode);
    else k_imr<RESTART, BATCHED, false><<<grid, block, 0, s>>>(k, all_mode);
}

// The end of an implicit step of particle p (queue slot idx) at z: the
// particle boundaries and write-back (finish), the particle's time and, with
// the slope cache, F at the stored state.  f, H: the right-hand side (keep)
// and H at z.  Returns whether the particle stays in the domain.
__device__ __forceinline__ bool implicit_end(const PushK& k, const RunK& R, long long p, double z[6], double sn,
                                             double cn, double qm, bool em, double H, double f[6], bool keep, int its)
{
    const double th_new = z[1];
    const bool alive = finish(R, k.P, p, z, H, 1, its);
    if (k.t) k.t[p] += k.dt_imp;
    if (keep && alive) {
        if (z[1] != th_new && !R.G.full) {     // reflected at a pole (a full-theta wrap changes nothing)
            double Hd;
            sn = -sn;
            F_at_sc(R, z, sn, cn, qm, em, f, Hd);
        }
        slope_store(k, p, z, qm, f, sn, cn);
    }
    return alive;
}

// After k_imr: H at each implicit step's end point (sin/cos of th^{n+1} by
// angle addition from th^n) and the write-back with the particle
// boundaries of Sec. 2.5.  With substeps (k.substeps > 0) a step whose solve
// did not converge, or whose |H - H^n| / D_0 exceeds substep_tol, is listed
// for k_imr_substep instead (the top bit of the entry marks the former).
template <bool BATCHED = false>
__global__ void __launch_bounds__(256) k_imr_finish(const __grid_constant__ PushK k, int all_mode)
{
    const long long qn = all_mode ? k.n : k.cnt[CNT_QUEUE];
    long long n_rm = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < qn;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long p = all_mode ? idx : (long long)k.queue[idx];
        if (all_mode && !k.P.alive[p]) continue;
        double z[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) z[i] = k.guess[(size_t)i * k.n + p];
        double sn, cn;
        const bool st = k.z0s && !all_mode;
        const double th0 = st ? k.z0s[(size_t)1 * k.n + idx] : k.P.th[p];
        sincos_near(th0, k.sc0[p], k.sc0[k.n + p], z[1], sn, cn);
        const RunK& R = BATCHED ? k.runs[run_of(k.runs, k.nruns, p)] : k.run;
        const double qm = st ? k.z0s[(size_t)6 * k.n + idx] : k.P.qm[p];
        const bool keep = !BATCHED && k.slope && !all_mode && !k.record;
        double H, f[6];
        const bool em = (R.has_fields || R.B0field != 0.0) && qm != 0.0;
        if (keep) F_at_sc(R, z, sn, cn, qm, em, f, H);
        else H = eval_H_sc(R.bh, z, sn, cn, qm, R.B0pot);
        if (k.substeps > 0 && !k.record) {
            const bool flagged = k.strag_flag[idx] != 0;
            const double Hn_p = st ? k.z0s[(size_t)7 * k.n + idx] : k.P.Hn[p];
            const double D0_p = st ? k.z0s[(size_t)8 * k.n + idx] : k.P.D0[p];
            if (flagged || (k.substep_tol > 0.0 && fabs(H - Hn_p) / D0_p > k.substep_tol)) {
                if (flagged) k.strag_flag[idx] = 0;
                const unsigned long long e = atomicAdd((unsigned long long*)&k.cnt[CNT_STRAG], 1ull);
                k.strag[e] = (uint32_t)idx | (flagged ? 0x80000000u : 0u);
                continue;
            }
        }
        const int its = (k.its && !all_mode) ? k.its[idx] : k.P.iters[p];
        if (!implicit_end(k, R, p, z, sn, cn, qm, em, H, f, keep, its)) ++n_rm;
    }
    warp_add(&k.cnt[CNT_REMOVED], n_rm, 0xffffffffu);
}

// Iteration cap of each substep's solve: a level whose substeps need more
// is too coarse, and the next level is tried.
constexpr int SUBSTEP_MAX_ITER = 16;

// Implicit steps listed by k_imr_finish (a solve that did not converge, or
// an end point off by more than substep_tol in H): the step redone from z^n
// as m = 2, 4, ..., 2^K substeps of dt_imp / m, each a solve (capped at
// SUBSTEP_MAX_ITER iterations) from its own start state with the pole
// reflection after it.  The first level whose
// solves all converge and whose end point has |H - H(z^n)| / D_0 <=
// substep_tol (0: no H condition) is taken, else the finest level whose
// solves all converged, else the full step's own result; then the step
// ends as in k_imr_finish.  One thread per listed step: they are rare.
template <bool BATCHED, bool NEWTON>
__global__ void __launch_bounds__(128) k_imr_substep(const __grid_constant__ PushK k, int all_mode)
{
    const long long ns = k.cnt[CNT_STRAG];
    long long n_it = 0, n_ev = 0, n_fix = 0, n_rm = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ns;
         e += (long long)gridDim.x * blockDim.x) {
        const uint32_t ent = k.strag[e];
        const bool unconv = (ent & 0x80000000u) != 0;
        const long long qi = ent & 0x7fffffffu;
        const long long p = all_mode ? qi : (long long)k.queue[qi];
        const RunK& R = BATCHED ? k.runs[run_of(k.runs, k.nruns, p)] : k.run;
        const bool st = !all_mode && k.z0s;
        double z0[6];
        if (st) {
#pragma unroll
            for (int i = 0; i < 6; ++i) z0[i] = k.z0s[(size_t)i * k.n + qi];
        } else {
            load_state(k.P, p, z0);
        }
        const double qm = st ? k.z0s[(size_t)6 * k.n + qi] : k.P.qm[p];
        const bool em = (R.has_fields || R.B0field != 0.0) && qm != 0.0;
        const double Href = eval_H(R.bh, z0, qm, R.B0pot), D0 = st ? k.z0s[(size_t)8 * k.n + qi] : k.P.D0[p];
        double z[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) z[i] = k.guess[(size_t)i * k.n + p];     // the full step's result
        bool have = false;
        long long its = 0;
        const int sub_iter = min(k.max_iter, SUBSTEP_MAX_ITER);
        for (int lev = 1; lev <= k.substeps; ++lev) {
            const int m = 1 << lev;
            const double h = k.dt_imp / m;
            double zs[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) zs[i] = z0[i];
            bool ok = true;
            for (int sub = 0; sub < m && ok; ++sub) {
                double zn[6];
                ok = imr_solve_serial<NEWTON>(k, R, zs, h, qm, em, sub_iter, zn, its, n_ev);
                theta_boundary(R.G, zn);
#pragma unroll
                for (int i = 0; i < 6; ++i) zs[i] = zn[i];
            }
            if (!ok) continue;
#pragma unroll
            for (int i = 0; i < 6; ++i) z[i] = zs[i];
            have = true;
            if (k.substep_tol <= 0.0 || fabs(eval_H(R.bh, zs, qm, R.B0pot) - Href) / D0 <= k.substep_tol) break;
        }
        n_it += its;
        if (have && unconv) ++n_fix;
        const int its0 = (k.its && !all_mode) ? k.its[qi] : k.P.iters[p];
        const int its_out = (int)min((long long)its0 + its, 255LL);
        double sn, cn, H, f[6];
        sincos(z[1], &sn, &cn);
        const bool keep = !BATCHED && k.slope && !all_mode;
        if (keep) F_at_sc(R, z, sn, cn, qm, em, f, H);
        else H = eval_H_sc(R.bh, z, sn, cn, qm, R.B0pot);
        if (!implicit_end(k, R, p, z, sn, cn, qm, em, H, f, keep, its_out)) ++n_rm;
    }
    warp_add(&k.cnt[CNT_ITERS], n_it, 0xffffffffu);
    warp_add(&k.cnt[CNT_EVALS], n_ev, 0xffffffffu);
    warp_add(&k.cnt[CNT_NOTCONV], -n_fix, 0xffffffffu);
    warp_add(&k.cnt[CNT_REMOVED], n_rm, 0xffffffffu);
}

// k_imr_finish and, with substeps, the substep kernel over what it listed.
template <bool BATCHED = false>
static void finish_implicit(unsigned grid, cudaStream_t s, const PushK& k, int all_mode)
{
    k_imr_finish<BATCHED><<<grid, 256, 0, s>>>(k, all_mode);
    if (k.substeps > 0 && !k.record) {
        if (k.imr_newton) k_imr_substep<BATCHED, true><<<grid, 128, 0, s>>>(k, all_mode);
        else k_imr_substep<BATCHED, false><<<grid, 128, 0, s>>>(k, all_mode);
    }
}

// ---------------------------------------------------------------------------
// Discrete-gradient Hamiltonian scheme for geodesics (Sec. 2.2.3, App. D).
// The symmetrised gradient averages the coordinate-increment gradients of
// the 12 update orders (3! pair orders x {coordinate-first, momentum-first});
// since H does not depend on ph and u_ph never changes, they reduce to four
// distinct orders over (r, u_r, th, u_th), each of weight 1/4, and the
// u_ph component to dH/du_ph averaged over the states where u_ph is visited
// (weights 2,1,1,2 / 6).  Every quotient (H(z') - H(z)) / dz is taken in
// the closed form of App. D: alpha' G' - alpha G = (alpha' + alpha)/2 (G' - G)
// + (G' + G)/2 (alpha' - alpha), G'^2 - G^2 and the metric differences with
// the increment divided out, so no digits are lost to cancellation and no
// switch to the partial derivative is needed.  The metric is needed at the
// four (r, th) combinations of z^n and the iterate.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Geo geo_at(const BH& bh, double r, double s, double c)
{
    Geo g;
    geo_eval(bh, r, s, c, g);
    return g;
}

// Gamma = sqrt(1 + g^ij u_i u_j) at a metric point
__device__ __forceinline__ double dg_gam(const Geo& g, double ur, double ut, double up)
{
    return sqrt(fma(g.gurr * ur, ur, fma(2.0 * g.gurp * ur, up, fma(g.gutt * ut, ut, fma(g.gupp * up, up, 1.0)))));
}

// Metric differences per unit increment of a position move b -> a.
struct PD {
    double dgrr, dgrp, dgtt, dgpp, dal, dbe, asum;
};

__device__ __forceinline__ PD pd_common(const BH& bh, const Geo& b, const Geo& a, double d_rho2, double d_f,
                                        double d_s2)
{
    PD d;
    const double irr = b.irho2 * a.irho2;            // 1 / (rho^2 rho'^2)
    const double d_irho2 = -d_rho2 * irr;
    const double ixx = b.ixi * a.ixi;                // 1 / (xi xi')
    const double sb = b.xi * b.alpha, sa = a.xi * a.alpha;   // sqrt(xi), sqrt(xi')
    d.dbe = d_f * ixx;
    d.dal = -d_f * (b.alpha * a.alpha) / (sb + sa);
    const double d_s2irho2 = fma(d_s2, b.rho2, -b.s2 * d_rho2) * irr;
    d.dgrr = fma(bh.a2, d_s2irho2, -d.dbe);          // d(1/xi) = -d(beta)
    d.dgrp = bh.a * d_irho2;
    d.dgtt = d_irho2;
    d.dgpp = -fma(d_rho2, a.s2, b.rho2 * d_s2) * (b.t * a.t);
    d.asum = b.alpha + a.alpha;
    return d;
}

// r move (th fixed): d(rho^2) = r + r', d(2 M r / rho^2) = 2 M (a^2 c^2 - r r') / (rho^2 rho'^2)
__device__ __forceinline__ PD pd_r(const BH& bh, const Geo& b, const Geo& a, double r0, double r1)
{
    const double d_f = bh.twoM * fma(bh.a2, b.c * b.c, -r0 * r1) * (b.irho2 * a.irho2);
    return pd_common(bh, b, a, r0 + r1, d_f, 0.0);
}

// th move (r fixed) with d(cos th) per unit increment dc: d(c^2) = (c + c') dc,
// d(rho^2) = a^2 d(c^2), d(2 M r / rho^2) = -2 M r d(rho^2) / (rho^2 rho'^2), d(s^2) = -d(c^2)
__device__ __forceinline__ PD pd_th(const BH& bh, const Geo& b, const Geo& a, double r, double dc)
{
    const double d_c2 = (b.c + a.c) * dc;
    const double d_rho2 = bh.a2 * d_c2;
    const double d_f = -bh.twoM * r * d_rho2 * (b.irho2 * a.irho2);
    return pd_common(bh, b, a, d_rho2, d_f, -d_c2);
}

// Quotient of a position move at momenta (ur, ut, up), Gamma at both ends given.
__device__ __forceinline__ double dq_pos(const PD& d, double gb, double ga, double ur, double ut, double up)
{
    const double dG2 = fma(d.dgrr * ur, ur, fma(2.0 * d.dgrp * ur, up, fma(d.dgtt * ut, ut, d.dgpp * up * up)));
    const double gs = ga + gb;
    return fma(0.5 * d.asum, dG2 / gs, fma(0.5 * gs, d.dal, -d.dbe * ur));
}

// Quotients of the momentum moves at a metric point (u_r: u0 -> u1 at u_th = ut; u_th: v0 -> v1 at u_r = ur).
__device__ __forceinline__ double dq_ur(const Geo& g, double gb, double ga, double u0, double u1, double up)
{
    return g.alpha * fma(g.gurr, u0 + u1, 2.0 * g.gurp * up) / (ga + gb) - g.beta;
}

__device__ __forceinline__ double dq_ut(const Geo& g, double gb, double ga, double v0, double v1)
{
    return g.alpha * g.gutt * (v0 + v1) / (ga + gb);
}

// sin(h) / h, by its series below |h| = 1e-3
__device__ __forceinline__ double sinc_dev(double h)
{
    if (fabs(h) < 1e-3) {
        const double h2 = h * h;
        return fma(h2, fma(h2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    }
    return sin(h) / h;
}

__global__ void __launch_bounds__(128) k_dg(PushK k, int all_mode)
{
    const long long qn = all_mode ? k.n : k.cnt[CNT_QUEUE];
    long long n_it = 0, n_nc = 0, n_rm = 0;
    const BH& bh = k.run.bh;
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
        double s0, c0;
        sincos(T0, &s0, &c0);
        const Geo m00 = geo_at(bh, R0, s0, c0);
        const double g00 = dg_gam(m00, U0, V0, P);
        const double f00 = m00.alpha * fma(m00.gurp, U0, m00.gupp * P) / g00;
        int it = 0;
        bool ok = false;
        while (it < k.max_iter) {
            const double R1 = zk[0], T1 = zk[1], U1 = zk[3], V1 = zk[4];
            double s1, c1;
            sincos(T1, &s1, &c1);
            const Geo m10 = geo_at(bh, R1, s0, c0), m01 = geo_at(bh, R0, s1, c1), m11 = geo_at(bh, R1, s1, c1);
            const double dT = T1 - T0;
            // d(cos th) / d th across the th move, without cancellation
            const double dc = -sin(0.5 * (T0 + T1)) * sinc_dev(0.5 * dT);
            const PD r_T0 = pd_r(bh, m00, m10, R0, R1), r_T1 = pd_r(bh, m01, m11, R0, R1);
            const PD t_R0 = pd_th(bh, m00, m01, R0, dc), t_R1 = pd_th(bh, m10, m11, R1, dc);
            // Gamma at the visited states
            const double g00_u1 = dg_gam(m00, U1, V0, P), g00_v1 = dg_gam(m00, U0, V1, P);
            const double g10 = dg_gam(m10, U0, V0, P), g10_u1 = dg_gam(m10, U1, V0, P), g10_uv = dg_gam(m10, U1, V1, P);
            const double g01 = dg_gam(m01, U0, V0, P), g01_v1 = dg_gam(m01, U0, V1, P), g01_uv = dg_gam(m01, U1, V1, P);
            const double g11_u1 = dg_gam(m11, U1, V0, P), g11_uv = dg_gam(m11, U1, V1, P), g11_v1 = dg_gam(m11, U0, V1, P);
            // order A: r, u_r, th, u_th
            const double rA = dq_pos(r_T0, g00, g10, U0, V0, P);
            const double uA = dq_ur(m10, g10, g10_u1, U0, U1, P);
            const double tA = dq_pos(t_R1, g10_u1, g11_u1, U1, V0, P);
            const double vA = dq_ut(m11, g11_u1, g11_uv, V0, V1);
            // order B: u_r, r, u_th, th
            const double uB = dq_ur(m00, g00, g00_u1, U0, U1, P);
            const double rB = dq_pos(r_T0, g00_u1, g10_u1, U1, V0, P);
            const double vB = dq_ut(m10, g10_u1, g10_uv, V0, V1);
            const double tB = dq_pos(t_R1, g10_uv, g11_uv, U1, V1, P);
            // order C: th, u_th, r, u_r
            const double tC = dq_pos(t_R0, g00, g01, U0, V0, P);
            const double vC = dq_ut(m01, g01, g01_v1, V0, V1);
            const double rC = dq_pos(r_T1, g01_v1, g11_v1, U0, V1, P);
            const double uC = dq_ur(m11, g11_v1, g11_uv, U0, U1, P);
            // order D: u_th, th, u_r, r
            const double vD = dq_ut(m00, g00, g00_v1, V0, V1);
            const double tD = dq_pos(t_R0, g00_v1, g01_v1, U0, V1, P);
            const double uD = dq_ur(m01, g01_v1, g01_uv, U0, U1, P);
            const double rD = dq_pos(r_T1, g01_uv, g11_uv, U1, V1, P);
            const double Gr = 0.25 * (rA + rB + rC + rD);
            const double Gt = 0.25 * (tA + tB + tC + tD);
            const double Gu = 0.25 * (uA + uB + uC + uD);
            const double Gv = 0.25 * (vA + vB + vC + vD);
            const double Gp = (2.0 * f00 + m10.alpha * fma(m10.gurp, U1, m10.gupp * P) / g10_u1 +
                               m01.alpha * fma(m01.gurp, U0, m01.gupp * P) / g01_v1 +
                               2.0 * m11.alpha * fma(m11.gurp, U1, m11.gupp * P) / g11_uv) / 6.0;
            double zn[6];
            zn[0] = fma(k.dt_imp, Gu, z0[0]);
            zn[1] = fma(k.dt_imp, Gv, z0[1]);
            zn[2] = fma(k.dt_imp, Gp, z0[2]);
            zn[3] = fma(-k.dt_imp, Gr, z0[3]);
            zn[4] = fma(-k.dt_imp, Gt, z0[4]);
            zn[5] = z0[5];
            ok = conv6(zn, zk, k.tol);
            for (int i = 0; i < 6; ++i) zk[i] = zn[i];
            ++it;
            if (ok) break;
        }
        if (!ok) ++n_nc;
        n_it += it;
        const double H1 = eval_H(bh, zk, 0.0, 0.0);
        if (!finish(k.run, k.P, p, zk, H1, 1, it)) ++n_rm;
        if (k.t) k.t[p] += k.dt_imp;
    }
    const unsigned m = __activemask();
    warp_add(&k.cnt[CNT_ITERS], n_it, m);
    warp_add(&k.cnt[CNT_NOTCONV], n_nc, m);
    warp_add(&k.cnt[CNT_EVALS], n_it, m);
    warp_add(&k.cnt[CNT_REMOVED], n_rm, m);
}

// ---------------------------------------------------------------------------
// Discrete-gradient scheme for charged particles in the analytic Wald field
// (an extension, not in the paper): the same scheme on
//   H_c(x, pi) = alpha Gamma(u) - beta^r u_r - (q/m) A_0,  u = pi - (q/m) A(x),
// in canonical momenta pi_i = u_i + (q/m) A_i with the potentials of Eq. (Amu)
// (A_th = 0); pi_ph is conserved.  Quotients in closed form as above, the
// position moves also carrying the potential differences (P = r / rho^2,
// K = 1 + c^2: A_0 = a B0 M K P, A_r = (B0/2)(2 a M K P - a s^2),
// A_ph = (B0/2) s^2 (r^2 + a^2 - 2 M a^2 K P)).  Neutral particles take the
// same path with q = 0.
// ---------------------------------------------------------------------------
struct PotP {
    double Ar, Aph, K, P;      // potentials and K, P at a metric point
};

__device__ __forceinline__ PotP pot_at(const BH& bh, double B0, double r, const Geo& g)
{
    PotP o;
    o.K = fma(g.c, g.c, 1.0);
    o.P = r * g.irho2;
    const double KP = o.K * o.P;
    o.Ar = 0.5 * B0 * bh.a * fma(2.0 * bh.M, KP, -g.s2);
    o.Aph = 0.5 * B0 * g.s2 * fma(-2.0 * bh.M * bh.a2, KP, fma(r, r, bh.a2));
    return o;
}

struct PDem {
    PD m;                      // metric differences per unit increment
    double dAr, dAph, dA0;     // potential differences per unit increment
};

__device__ __forceinline__ PDem pdem_r(const BH& bh, double B0, const Geo& b, const Geo& a, const PotP& pb,
                                       double r0, double r1)
{
    PDem d;
    d.m = pd_r(bh, b, a, r0, r1);
    const double dP = fma(bh.a2, b.c * b.c, -r0 * r1) * (b.irho2 * a.irho2);
    const double dKP = pb.K * dP;
    d.dA0 = bh.a * B0 * bh.M * dKP;
    d.dAr = d.dA0;
    d.dAph = 0.5 * B0 * b.s2 * fma(-2.0 * bh.M * bh.a2, dKP, r0 + r1);
    return d;
}

__device__ __forceinline__ PDem pdem_th(const BH& bh, double B0, const Geo& b, const Geo& a, const PotP& pb,
                                        const PotP& pa, double r, double dc)
{
    PDem d;
    d.m = pd_th(bh, b, a, r, dc);
    const double dc2 = (b.c + a.c) * dc;
    const double dP = -r * bh.a2 * dc2 * (b.irho2 * a.irho2);
    const double dKP = fma(dc2, pa.P, pb.K * dP);
    d.dA0 = bh.a * B0 * bh.M * dKP;
    d.dAr = 0.5 * B0 * bh.a * fma(2.0 * bh.M, dKP, dc2);
    const double Ya = fma(-2.0 * bh.M * bh.a2, pa.K * pa.P, fma(r, r, bh.a2));
    d.dAph = 0.5 * B0 * fma(-dc2, Ya, -2.0 * bh.M * bh.a2 * b.s2 * dKP);
    return d;
}

// Quotient of a position move; (ub_r, ub_p) and (ua_r, ua_p) the kinetic
// momenta at the two ends (same pi), ut the th momentum.
__device__ __forceinline__ double dq_pos_em(const PDem& d, const Geo& b, double qm, double gb, double ga,
                                            double ub_r, double ub_p, double ua_r, double ua_p, double ut)
{
    const double dur = -qm * d.dAr, dup = -qm * d.dAph;
    double dG2 = fma(d.m.dgrr * ua_r, ua_r, fma(2.0 * d.m.dgrp * ua_r, ua_p, fma(d.m.dgtt * ut, ut, d.m.dgpp * ua_p * ua_p)));
    dG2 = fma(b.gurr * dur, ua_r + ub_r, dG2);
    dG2 = fma(2.0 * b.gurp, fma(dur, ua_p, ub_r * dup), dG2);
    dG2 = fma(b.gupp * dup, ua_p + ub_p, dG2);
    const double gs = ga + gb;
    return fma(0.5 * d.m.asum, dG2 / gs, fma(0.5 * gs, d.m.dal, -fma(d.m.dbe, ua_r, fma(b.beta, dur, qm * d.dA0))));
}

__global__ void __launch_bounds__(128) k_dg_em(PushK k, int all_mode)
{
    const long long qn = all_mode ? k.n : k.cnt[CNT_QUEUE];
    long long n_it = 0, n_nc = 0, n_rm = 0;
    const BH& bh = k.run.bh;
    const double B0 = k.run.B0field;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < qn;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long p = all_mode ? idx : (long long)k.queue[idx];
        if (all_mode && !k.P.alive[p]) {
            k.P.scheme[p] = 0;
            k.P.iters[p] = 0;
            continue;
        }
        const double qm = k.P.qm[p];
        double z0[6], zk[6];
        load_state(k.P, p, z0);
        if (all_mode) {
            for (int i = 0; i < 6; ++i) zk[i] = z0[i];
        } else {
            for (int i = 0; i < 6; ++i) zk[i] = k.guess[(size_t)i * k.n + p];
        }
        const double R0 = z0[0], T0 = z0[1];
        double s0, c0;
        sincos(T0, &s0, &c0);
        const Geo m00 = geo_at(bh, R0, s0, c0);
        const PotP p00 = pot_at(bh, B0, R0, m00);
        // canonical momenta of z^n and of the start
        const double U0 = fma(qm, p00.Ar, z0[3]), V0 = z0[4], P = fma(qm, p00.Aph, z0[5]);
        {
            double sk, ck;
            sincos(zk[1], &sk, &ck);
            const Geo gk = geo_at(bh, zk[0], sk, ck);
            const PotP pk = pot_at(bh, B0, zk[0], gk);
            zk[3] = fma(qm, pk.Ar, zk[3]);
            zk[5] = fma(qm, pk.Aph, zk[5]);
        }
        zk[5] = P;
        // kinetic momenta at m00
        const double u00r = fma(-qm, p00.Ar, U0), u00p = fma(-qm, p00.Aph, P);
        const double g00 = dg_gam(m00, u00r, V0, u00p);
        const double f00 = m00.alpha * fma(m00.gurp, u00r, m00.gupp * u00p) / g00;
        int it = 0;
        bool ok = false;
        double wn[6];
        while (it < k.max_iter) {
            const double R1 = zk[0], T1 = zk[1], U1 = zk[3], V1 = zk[4];
            double s1, c1;
            sincos(T1, &s1, &c1);
            const Geo m10 = geo_at(bh, R1, s0, c0), m01 = geo_at(bh, R0, s1, c1), m11 = geo_at(bh, R1, s1, c1);
            const PotP p10 = pot_at(bh, B0, R1, m10), p01 = pot_at(bh, B0, R0, m01), p11 = pot_at(bh, B0, R1, m11);
            const double dT = T1 - T0;
            const double dc = -sin(0.5 * (T0 + T1)) * sinc_dev(0.5 * dT);
            const PDem r_T0 = pdem_r(bh, B0, m00, m10, p00, R0, R1), r_T1 = pdem_r(bh, B0, m01, m11, p01, R0, R1);
            const PDem t_R0 = pdem_th(bh, B0, m00, m01, p00, p01, R0, dc);
            const PDem t_R1 = pdem_th(bh, B0, m10, m11, p10, p11, R1, dc);
            // kinetic u_r, u_ph at each metric point for pi_r = U0 / U1 (pi_ph = P)
            const double a00 = qm * p00.Ar, a10 = qm * p10.Ar, a01 = qm * p01.Ar, a11 = qm * p11.Ar;
            const double up00 = u00p, up10 = fma(-qm, p10.Aph, P), up01 = fma(-qm, p01.Aph, P),
                         up11 = fma(-qm, p11.Aph, P);
            const double r00_0 = U0 - a00, r00_1 = U1 - a00, r10_0 = U0 - a10, r10_1 = U1 - a10;
            const double r01_0 = U0 - a01, r01_1 = U1 - a01, r11_0 = U0 - a11, r11_1 = U1 - a11;
            // Gamma at the visited states
            const double g00_u1 = dg_gam(m00, r00_1, V0, up00), g00_v1 = dg_gam(m00, r00_0, V1, up00);
            const double g10 = dg_gam(m10, r10_0, V0, up10), g10_u1 = dg_gam(m10, r10_1, V0, up10),
                         g10_uv = dg_gam(m10, r10_1, V1, up10);
            const double g01 = dg_gam(m01, r01_0, V0, up01), g01_v1 = dg_gam(m01, r01_0, V1, up01),
                         g01_uv = dg_gam(m01, r01_1, V1, up01);
            const double g11_u1 = dg_gam(m11, r11_1, V0, up11), g11_uv = dg_gam(m11, r11_1, V1, up11),
                         g11_v1 = dg_gam(m11, r11_0, V1, up11);
            // order A: r, u_r, th, u_th
            const double rA = dq_pos_em(r_T0, m00, qm, g00, g10, r00_0, up00, r10_0, up10, V0);
            const double uA = dq_ur(m10, g10, g10_u1, r10_0, r10_1, up10);
            const double tA = dq_pos_em(t_R1, m10, qm, g10_u1, g11_u1, r10_1, up10, r11_1, up11, V0);
            const double vA = dq_ut(m11, g11_u1, g11_uv, V0, V1);
            // order B: u_r, r, u_th, th
            const double uB = dq_ur(m00, g00, g00_u1, r00_0, r00_1, up00);
            const double rB = dq_pos_em(r_T0, m00, qm, g00_u1, g10_u1, r00_1, up00, r10_1, up10, V0);
            const double vB = dq_ut(m10, g10_u1, g10_uv, V0, V1);
            const double tB = dq_pos_em(t_R1, m10, qm, g10_uv, g11_uv, r10_1, up10, r11_1, up11, V1);
            // order C: th, u_th, r, u_r
            const double tC = dq_pos_em(t_R0, m00, qm, g00, g01, r00_0, up00, r01_0, up01, V0);
            const double vC = dq_ut(m01, g01, g01_v1, V0, V1);
            const double rC = dq_pos_em(r_T1, m01, qm, g01_v1, g11_v1, r01_0, up01, r11_0, up11, V1);
            const double uC = dq_ur(m11, g11_v1, g11_uv, r11_0, r11_1, up11);
            // order D: u_th, th, u_r, r
            const double vD = dq_ut(m00, g00, g00_v1, V0, V1);
            const double tD = dq_pos_em(t_R0, m00, qm, g00_v1, g01_v1, r00_0, up00, r01_0, up01, V1);
            const double uD = dq_ur(m01, g01_v1, g01_uv, r01_0, r01_1, up01);
            const double rD = dq_pos_em(r_T1, m01, qm, g01_uv, g11_uv, r01_1, up01, r11_1, up11, V1);
            const double Gr = 0.25 * (rA + rB + rC + rD);
            const double Gt = 0.25 * (tA + tB + tC + tD);
            const double Gu = 0.25 * (uA + uB + uC + uD);
            const double Gv = 0.25 * (vA + vB + vC + vD);
            const double Gp = (2.0 * f00 + m10.alpha * fma(m10.gurp, r10_1, m10.gupp * up10) / g10_u1 +
                               m01.alpha * fma(m01.gurp, r01_0, m01.gupp * up01) / g01_v1 +
                               2.0 * m11.alpha * fma(m11.gurp, r11_1, m11.gupp * up11) / g11_uv) / 6.0;
            wn[0] = fma(k.dt_imp, Gu, z0[0]);
            wn[1] = fma(k.dt_imp, Gv, z0[1]);
            wn[2] = fma(k.dt_imp, Gp, z0[2]);
            wn[3] = fma(-k.dt_imp, Gr, U0);
            wn[4] = fma(-k.dt_imp, Gt, V0);
            wn[5] = P;
            ok = conv6(wn, zk, k.tol);
            for (int i = 0; i < 6; ++i) zk[i] = wn[i];
            ++it;
            if (ok) break;
        }
        if (!ok) ++n_nc;
        n_it += it;
        // back to kinetic momenta at x^{n+1}
        {
            double sk, ck;
            sincos(zk[1], &sk, &ck);
            const Geo gk = geo_at(bh, zk[0], sk, ck);
            const PotP pk = pot_at(bh, B0, zk[0], gk);
            zk[3] = fma(-qm, pk.Ar, zk[3]);
            zk[5] = fma(-qm, pk.Aph, zk[5]);
        }
        const double H1 = eval_H(bh, zk, qm, k.run.B0pot);
        if (!finish(k.run, k.P, p, zk, H1, 1, it)) ++n_rm;
        if (k.t) k.t[p] += k.dt_imp;
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

namespace fpic {
// Explicit pass split into chunks whose launches wait for per-chunk events
// (set by the caller after each chunk's host-to-device copies).
struct PushChunks {
    int k;
    const long long* bounds;    // k + 1 particle offsets
    const cudaEvent_t* ready;   // k events
};
}  // namespace fpic

namespace fpic {
// Per-cell bilinear coefficients of the six field components (see gather_c),
// one thread per (node row, column); cells past a sub-grid's last node pair
// are never read (the cell search clamps to the last cell).
__global__ void k_field_coef(GridDev G, Fields F, double* out, size_t sz)
{
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= G.Nth; j += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const bool ro = (k == 0 || k == 4 || k == 5);
            const bool to = (k == 1 || k == 3 || k == 5);
            // full-theta domain: the half-node wrap cell (Nth - 1) also has
            // coefficients (its upper column Nth is the image of column 0)
            const int NRk = ro ? G.Nr : G.Nr + 1, NTk = to ? G.Nth + G.full : G.Nth + 1;
            if (i >= NRk - 1 || j >= NTk - 1) continue;
            const size_t o = (size_t)i * G.ld + j;
            const double* f = F.f[k];
            const double f00 = f[o], f01 = f[o + 1], f10 = f[o + G.ld], f11 = f[o + G.ld + 1];
            const double b = f10 - f00, c = f01 - f00;
            double2* q = reinterpret_cast<double2*>(out + (size_t)k * 4 * sz + 4 * o);
            q[0] = make_double2(f00, b);
            q[1] = make_double2(c, (f11 - f10) - c);
        }
    }
}
}  // namespace fpic

// Builds the context's coefficient copy of the fields on stream s and points
// R at it.
static int field_coefs(fpic_ctx* c, const double* const fields[6], RunK& R, cudaStream_t s)
{
    const size_t sz = (size_t)(c->Nr + 1) * c->ld;
    const size_t bytes = 6 * 4 * sz * sizeof(double);
    if (c->fcoef_bytes < bytes) {
        retire(c, &c->d_fcoef);
        c->fcoef_bytes = 0;
        for (int i = 0; i < 6; ++i) c->fcoef_src[i] = nullptr;
        FPIC_CUDA(cudaMalloc(&c->d_fcoef, bytes));
        c->fcoef_bytes = bytes;
    }
    Fields F;
    for (int i = 0; i < 6; ++i) F.f[i] = fields[i];
    double* out = (double*)c->d_fcoef;
    bool same = c->static_fields != 0;
    for (int i = 0; i < 6; ++i) same = same && c->fcoef_src[i] == fields[i];
    if (!same) {
        k_field_coef<<<dim3((unsigned)((c->Nth + 1 + 127) / 128), c->Nr + 1), 128, 0, s>>>(c->G, F, out, sz);
        FPIC_CUDA(cudaGetLastError());
        for (int i = 0; i < 6; ++i) c->fcoef_src[i] = fields[i];
    }
    for (int i = 0; i < 6; ++i) R.FC.c[i] = out + (size_t)i * 4 * sz;
    R.has_coef = 1;
    return 0;
}

// Tensor maps of the six coefficient arrays for the field-tile staging
// (FPIC_TUNE_STAGE_FIELDS): each component is a 2-D FP64 tensor of Nr + 1
// rows of 4 ld values (a cell's four coefficients side by side), read in
// boxes of STAGE_TI rows x 4 STAGE_TJ values.  Encoded on the host through
// the driver's cuTensorMapEncodeTiled and copied to a library-owned device
// buffer (a fresh one per coefficient buffer; the old one is retired).
typedef CUresult (*PfnEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int stage_maps(fpic_ctx* c, PushK& k)
{
    if (!(c->d_stage_maps && c->stage_key == c->d_fcoef && c->stage_key_Nr == c->Nr && c->stage_key_ld == c->ld)) {
        static PfnEncodeTiled enc = nullptr;
        if (!enc) {
            void* f = nullptr;
            cudaDriverEntryPointQueryResult q;
            FPIC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
            if (q != cudaDriverEntryPointSuccess || !f)
                return set_error(FPIC_ECUDA, "field staging: cuTensorMapEncodeTiled not found");
            enc = (PfnEncodeTiled)f;
        }
        alignas(64) CUtensorMap maps[6];
        const size_t sz = (size_t)(c->Nr + 1) * c->ld;
        const cuuint64_t dims[2] = {(cuuint64_t)4 * c->ld, (cuuint64_t)c->Nr + 1};
        const cuuint64_t strides[1] = {(cuuint64_t)4 * c->ld * sizeof(double)};
        const cuuint32_t box[2] = {4u * STAGE_TJ, (cuuint32_t)STAGE_TI};
        const cuuint32_t es[2] = {1u, 1u};
        for (int i = 0; i < 6; ++i) {
            CUresult r = enc(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (double*)c->d_fcoef + (size_t)i * 4 * sz, dims,
                             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return set_error(FPIC_ECUDA, "field staging: cuTensorMapEncodeTiled failed (%d)", (int)r);
        }
        retire(c, &c->d_stage_maps);
        FPIC_CUDA(cudaMalloc(&c->d_stage_maps, sizeof maps));
        FPIC_CUDA(cudaMemcpy(c->d_stage_maps, maps, sizeof maps, cudaMemcpyHostToDevice));
        c->stage_key = c->d_fcoef;
        c->stage_key_Nr = c->Nr;
        c->stage_key_ld = c->ld;
    }
    k.stage_maps = (const uint8_t*)c->d_stage_maps;
    return 0;
}

// Slope cache of a push (FPIC_TUNE_REUSE_SLOPE): points k at the context's
// cache and marks it cold when the push's key differs from the previous
// one's (another particle set or size, other fields, another grid) or the
// cache was just (re)allocated.  Off when grid fields may change between
// pushes (FPIC_TUNE_STATIC_FIELDS = 0).
static int slope_setup(fpic_ctx* c, const fpic_particles* p, const double* const fields[6], double B0field, PushK& k)
{
    k.slope = nullptr;
    k.slope_cold = 1;
    if (!c->reuse_slope || (fields && !c->static_fields) || p->n <= 0) return 0;
    const size_t need = (size_t)SLOPE_ROWS * (size_t)p->n * sizeof(double);
    bool cold = false;
    if (c->slope_bytes < need) {
        retire(c, &c->d_slope);
        c->slope_bytes = 0;
        FPIC_CUDA(cudaMalloc(&c->d_slope, need));
        c->slope_bytes = need;
        cold = true;
    }
    cold = cold || c->slope_key_r != (const void*)p->r || c->slope_key_n != p->n ||
           c->slope_key_B0field != B0field || c->slope_key_grid != c->grid_gen;
    for (int i = 0; i < 6; ++i) {
        const double* f = fields ? fields[i] : nullptr;
        cold = cold || c->slope_key_f[i] != f;
        c->slope_key_f[i] = f;
    }
    c->slope_key_r = p->r;
    c->slope_key_n = p->n;
    c->slope_key_B0field = B0field;
    c->slope_key_grid = c->grid_gen;
    k.slope = (double*)c->d_slope;
    k.slope_cold = cold ? 1 : 0;
    return 0;
}

// Step of the implicit solves: the hybrid's partner takes dt_implicit when
// set (adaptive steps, Sec. 3.1.2); pure schemes take dt.
static double implicit_step(const fpic_push_params* prm)
{
    const bool hyb = prm->scheme == FPIC_HYB1 || prm->scheme == FPIC_HYB2;
    return (hyb && prm->dt_implicit != 0.0) ? prm->dt_implicit : prm->dt;
}

static bool dt_implicit_ok(const fpic_push_params* prm)
{
    return prm->dt_implicit == 0.0 || (std::isfinite(prm->dt_implicit) && (prm->dt_implicit > 0.0) == (prm->dt > 0.0));
}

// fpic_push_stats from the push's counters (host after a synchronising
// read, or on the device for FPIC_TUNE_ASYNC).  Slope reuse: k1 only where
// not reused, the full right-hand side at every trial's end point and at
// every converged IMR solve.
__host__ __device__ inline void stats_from_counters(const long long* h, int scheme, int implicit, bool explicit_pass,
                                                    bool slope, fpic_push_stats* st)
{
    st->n_alive_before = h[CNT_ALIVE];
    st->n_implicit = scheme == FPIC_RK4 ? 0 : (scheme >= FPIC_HYB1 ? h[CNT_QUEUE] : h[CNT_ALIVE]);
    st->n_iter_total = h[CNT_ITERS];
    st->n_notconv = h[CNT_NOTCONV];
    st->n_removed = h[CNT_REMOVED];
    st->n_rhs_evals = h[CNT_EVALS] + (explicit_pass ? 4 * h[CNT_ALIVE] : 0);
    st->n_slope_reused = h[CNT_SLOPE];
    st->n_tiles_staged = h[CNT_STAGED];
    if (slope) {
        st->n_rhs_evals += h[CNT_ALIVE] - h[CNT_SLOPE];
        if (scheme >= FPIC_HYB1 && implicit == FPIC_IMR) st->n_rhs_evals += h[CNT_QUEUE];
    }
}

__global__ void k_stats_final(const long long* cnt, fpic_push_stats* out, int scheme, int implicit, int explicit_pass,
                              int slope)
{
    stats_from_counters(cnt, scheme, implicit, explicit_pass != 0, slope != 0, out);
}

static int push_core(fpic_ctx* c, fpic_particles* p, const double* const fields[6], const fpic_push_params* prm,
                     fpic_push_stats* stats, cudaStream_t s, const PushChunks* ch, bool host_state = false);

// Argument checks shared by fpic_push and fpic_push_host (who: the caller's
// name in the message).
static int check_push_args(const fpic_ctx* c, const fpic_particles* p, const double* const fields[6],
                           const fpic_push_params* prm, const char* who)
{
    if (!c || !p || !prm) return set_error(FPIC_EINVAL, "%s: NULL ctx/particles/params", who);
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "%s: n out of range [0, 2^31)", who);
    if (!particles_ok(p, true)) return set_error(FPIC_EINVAL, "%s: a particle array is NULL", who);
    if (!(std::isfinite(prm->dt)) || prm->dt == 0.0) return set_error(FPIC_EINVAL, "%s: dt must be finite and nonzero", who);
    if (!dt_implicit_ok(prm)) return set_error(FPIC_EINVAL, "%s: dt_implicit must be 0 or finite with the sign of dt", who);
    if (prm->B0field != 0.0 && (fields || !std::isfinite(prm->B0field) || c->M != 1.0))
        return set_error(FPIC_EINVAL, "%s: B0field needs fields == NULL, a finite value and M = 1", who);
    if (prm->scheme < FPIC_RK4 || prm->scheme > FPIC_HYB2) return set_error(FPIC_EINVAL, "%s: unknown scheme %d", who, prm->scheme);
    if (prm->scheme >= FPIC_HYB1 && prm->implicit != FPIC_IMR && prm->implicit != FPIC_HAM)
        return set_error(FPIC_EINVAL, "%s: implicit partner must be FPIC_IMR or FPIC_HAM", who);
    if (prm->max_iter < 1 || prm->max_iter > 255) return set_error(FPIC_EINVAL, "%s: max_iter must be in [1, 255]", who);
    if (!(prm->tol >= 0.0)) return set_error(FPIC_EINVAL, "%s: tol must be >= 0", who);
    if (prm->imr_substeps < 0 || prm->imr_substeps > 12 || !(prm->substep_tol >= 0.0) || !std::isfinite(prm->substep_tol))
        return set_error(FPIC_EINVAL, "%s: imr_substeps must be in [0, 12] and substep_tol finite and >= 0", who);
    if (fields) {
        for (int i = 0; i < 6; ++i)
            if (!fields[i]) return set_error(FPIC_EINVAL, "%s: fields[%d] is NULL", who, i);
        if (!c->has_grid) return set_error(FPIC_EINVAL, "%s: fields given but no grid set", who);
    }
    if (prm->guess) return set_error(FPIC_EINVAL, "%s: learned guesses need fpic_push_learned", who);
    if (prm->before) {
        const fpic_particles* b = prm->before;
        if (prm->scheme != FPIC_RK4 && prm->scheme < FPIC_HYB1)
            return set_error(FPIC_EINVAL, "%s: before needs RK4 or a hybrid scheme (the explicit pass writes it)", who);
        if (!b->r || !b->th || !b->ur || !b->uth || !b->uph || !b->alive)
            return set_error(FPIC_EINVAL, "%s: before has a NULL r, th, ur, uth, uph or alive array", who);
        if (b->n < p->n) return set_error(FPIC_EINVAL, "%s: before holds fewer than n particles", who);
    }
    return 0;
}

extern "C" int fpic_push(fpic_ctx* c, fpic_particles* p, const double* const fields[6],
                         const fpic_push_params* prm, fpic_push_stats* stats, void* stream)
{
    const int rc = check_push_args(c, p, fields, prm, "fpic_push");
    if (rc) return rc;
    return push_core(c, p, fields, prm, stats, (cudaStream_t)stream, nullptr);
}

static int push_core(fpic_ctx* c, fpic_particles* p, const double* const fields[6], const fpic_push_params* prm,
                     fpic_push_stats* stats, cudaStream_t s, const PushChunks* ch, bool host_state)
{
    const bool has_fields = fields != nullptr;
    const long long n = p->n;
    FPIC_CUDA(cudaSetDevice(c->device));
    // guess 6n, sin/cos 2n (doubles) | queue, order, straggler list (u32) |
    // host state: z^n, q/m, H^n and D_0 by slot 9n (doubles, 16-byte aligned),
    // iteration counts n (bytes) | straggler flags n (bytes, 16-byte aligned)
    const size_t base_need = ((size_t)n * (8 * sizeof(double) + 3 * sizeof(uint32_t)) + 15) & ~(size_t)15;
    const size_t flag_off = (base_need + (host_state ? (size_t)n * (9 * sizeof(double) + 1) : 0) + 15) & ~(size_t)15;
    const size_t need = flag_off + (size_t)n + 256;
    int rc = ensure_scratch(c, need);
    if (rc) return rc;
    PushK k{};
    k.run.bh = c->bh;
    k.run.G = c->G;
    k.run.has_grid = c->has_grid;
    k.run.has_fields = has_fields;
    for (int i = 0; i < 6; ++i) k.run.F.f[i] = has_fields ? fields[i] : nullptr;
    k.dt = prm->dt;
    k.dt_imp = implicit_step(prm);
    k.imr_newton = prm->imr_newton ? 1 : 0;
    k.t = prm->t;
    k.thr = prm->thr;
    push_constants(k);
    k.tol = prm->tol;
    k.dg_eps = prm->dg_eps;
    k.run.B0pot = prm->B0pot;
    k.run.B0field = has_fields ? 0.0 : prm->B0field;
    k.run.r_h = c->r_h;
    k.run.r_max = prm->r_max;
    k.scheme = prm->scheme;
    k.max_iter = prm->max_iter;
    k.n = n;
    k.P = PartDev{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                  p->alive, p->scheme, p->iters, p->cell};
    if (prm->before) {
        const fpic_particles* b = prm->before;
        k.before = PartDev{b->r, b->th, nullptr, b->ur, b->uth, b->uph, nullptr, nullptr, nullptr, nullptr,
                           b->alive, nullptr, nullptr, nullptr};
    }
    if (has_fields && n > 0) {
        rc = field_coefs(c, fields, k.run, s);
        if (rc) return rc;
        if (c->stage_fields && !ch && !host_state && p->cell) {
            rc = stage_maps(c, k);
            if (rc) return rc;
        }
    }
    if (prm->scheme == FPIC_RK4 || prm->scheme >= FPIC_HYB1) {
        rc = slope_setup(c, p, fields, k.run.B0field, k);
        if (rc) return rc;
    }
    k.guess = (double*)c->d_scratch;
    k.sc0 = k.guess + (size_t)n * 6;
    k.queue = (uint32_t*)((char*)c->d_scratch + (size_t)n * 8 * sizeof(double));
    k.order = k.queue + n;
    k.strag = k.order + n;
    k.strag_flag = (uint8_t*)c->d_scratch + flag_off;
    k.substeps = prm->imr_substeps;
    k.substep_tol = prm->substep_tol;
    if (host_state) {
        k.z0s = (double*)((char*)c->d_scratch + base_need);
        k.its = (uint8_t*)(k.z0s + (size_t)n * 9);
    }
    k.cnt = c->d_cnt;
    k.learned = nullptr;
    FPIC_CUDA(cudaMemsetAsync(c->d_cnt, 0, CNT_N * sizeof(long long), s));
    if (n == 0) {
        if (stats) *stats = fpic_push_stats{};
        return FPIC_OK;
    }
    if (k.substeps > 0) FPIC_CUDA(cudaMemsetAsync(k.strag_flag, 0, (size_t)n, s));
    const int TB = 128;
    const unsigned persist = (unsigned)c->sm_count * 8u;
    const unsigned imr_grid = (unsigned)c->sm_count * (unsigned)c->imr_blocks_per_sm;
    cudaEvent_t* ev = prm->events ? (cudaEvent_t*)prm->events : nullptr;
    const bool explicit_pass = prm->scheme == FPIC_RK4 || prm->scheme >= FPIC_HYB1;
    // few particles (under 4 blocks of 128 per SM): one-warp blocks, so the
    // latency-bound steps spread over every SM instead of a few
    const int TBx = n <= (long long)c->sm_count * 4 * 128 ? 32 : TB;
    const unsigned nbx = (unsigned)((n + TBx - 1) / TBx);
    // with an explicit pass the alive count rides along in it (after each
    // chunk's copies have landed); otherwise a separate pass counts
    if (stats && !explicit_pass) {
        if (ch)
            for (int j = 0; j < ch->k; ++j) FPIC_CUDA(cudaStreamWaitEvent(s, ch->ready[j], 0));
        k_count_alive<<<persist, 256, 0, s>>>(k.P, n, c->d_cnt);
    }
    k.count_alive = stats && explicit_pass ? 1 : 0;
    if (ev) FPIC_CUDA(cudaEventRecord(ev[0], s));
    if (ch && !explicit_pass)
        for (int j = 0; j < ch->k; ++j) FPIC_CUDA(cudaStreamWaitEvent(s, ch->ready[j], 0));
    if (explicit_pass) {
        const int nck = ch ? ch->k : 1;
        for (int j = 0; j < nck; ++j) {
            k.p_begin = ch ? ch->bounds[j] : 0;
            k.p_end = ch ? ch->bounds[j + 1] : n;
            const long long len = k.p_end - k.p_begin;
            if (ch) FPIC_CUDA(cudaStreamWaitEvent(s, ch->ready[j], 0));
            if (len <= 0) continue;
            const unsigned nbj = (unsigned)((len + TBx - 1) / TBx);
            if (k.stage_maps) {
                if (prm->scheme == FPIC_RK4) k_explicit<0, false, true><<<nbj, TBx, 0, s>>>(k);
                else k_explicit<1, false, true><<<nbj, TBx, 0, s>>>(k);
            } else if (prm->scheme == FPIC_RK4) {
                k_explicit<0><<<nbj, TBx, 0, s>>>(k);
            } else {
                k_explicit<1><<<nbj, TBx, 0, s>>>(k);
            }
        }
        k.p_begin = 0;
        k.p_end = 0;
    }
    if (ev) {
        FPIC_CUDA(cudaEventRecord(ev[1], s));
        FPIC_CUDA(cudaEventRecord(ev[2], s));
    }
    if (prm->scheme == FPIC_IMR) {
        launch_imr<0>(imr_grid, TB, s, k, 1);
        finish_implicit<>(persist, s, k, 1);
    } else if (prm->scheme == FPIC_HAM) {
        if (k.run.B0field != 0.0) k_dg_em<<<nbx, TBx, 0, s>>>(k, 1);
        else k_dg<<<nbx, TBx, 0, s>>>(k, 1);
    } else if (prm->scheme >= FPIC_HYB1 && prm->implicit == FPIC_IMR) {
        k_order<<<persist, 256, 0, s>>>(k);
        launch_imr<0>(imr_grid, TB, s, k, 0);
        finish_implicit<>(persist, s, k, 0);
    } else if (prm->scheme >= FPIC_HYB1) {
        if (k.run.B0field != 0.0) k_dg_em<<<nbx, TBx, 0, s>>>(k, 0);
        else k_dg<<<nbx, TBx, 0, s>>>(k, 0);
    }
    if (ev) FPIC_CUDA(cudaEventRecord(ev[3], s));
    FPIC_CUDA(cudaGetLastError());
    if (stats && c->async) {
        // assembled on the device, copied without waiting (FPIC_TUNE_ASYNC)
        fpic_push_stats* d_st = (fpic_push_stats*)(c->d_cnt + CNT_N);
        k_stats_final<<<1, 1, 0, s>>>(c->d_cnt, d_st, prm->scheme, prm->implicit, explicit_pass ? 1 : 0,
                                      k.slope ? 1 : 0);
        FPIC_CUDA(cudaMemcpyAsync(stats, d_st, sizeof(fpic_push_stats), cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaGetLastError());
        return FPIC_OK;
    }
    if (stats) {
        FPIC_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, CNT_N * sizeof(long long), cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        stats_from_counters(c->h_cnt, prm->scheme, prm->implicit, explicit_pass, k.slope != nullptr, stats);
        const long long* h = c->h_cnt;
        if (h[CNT_ERR] > 0) return set_error(FPIC_ETIMEOUT, "fpic_push: %lld field-tile loads timed out", h[CNT_ERR]);
        if (h[CNT_NOTCONV] > 0) return FPIC_ENOTCONVERGED;
    }
    return FPIC_OK;
}

extern "C" int fpic_push_host(fpic_ctx* c, fpic_particles* hp, const double* const fields[6],
                              const fpic_push_params* prm, fpic_push_stats* stats, void* stream)
{
    const int rc_args = check_push_args(c, hp, fields, prm, "fpic_push_host");
    if (rc_args) return rc_args;
    if (prm->before) return set_error(FPIC_EINVAL, "fpic_push_host: before is not supported with host particles");
    const long long n = hp->n;
    cudaStream_t s = (cudaStream_t)stream;
    FPIC_CUDA(cudaSetDevice(c->device));
    // Pinned (page-locked, mapped) host arrays are reachable from the GPU over
    // NVLink-C2C: the push then reads and writes them in place, with no
    // staging copies (each byte still crosses the link once per direction).
    if (n > 0 && !c->host_staging) {
        fpic_particles z = *hp;
        bool mapped = true;
        void** fields_h[] = {(void**)&z.r, (void**)&z.th, (void**)&z.ph, (void**)&z.ur, (void**)&z.uth,
                             (void**)&z.uph, (void**)&z.qm, (void**)&z.w, (void**)&z.H0, (void**)&z.D0,
                             (void**)&z.Hn, (void**)&z.alive, (void**)&z.scheme, (void**)&z.iters,
                             (void**)&z.cell};
        for (void** f : fields_h) {
            if (!*f) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, *f) != cudaSuccess || at.type != cudaMemoryTypeHost ||
                !at.devicePointer) {
                cudaGetLastError();
                mapped = false;
                break;
            }
            *f = at.devicePointer;
        }
        if (mapped) {
            int rc0 = push_core(c, &z, fields, prm, stats, s, nullptr, true);
            if (rc0 < 0) return rc0;
            if (!c->async) FPIC_CUDA(cudaStreamSynchronize(s));
            return rc0;
        }
    }
    // device mirror: 11 double arrays, 3 byte arrays, 1 u32 array
    const size_t nd = (size_t)n * sizeof(double), nb = (size_t)n, n4 = (size_t)n * 4;
    int rc = ensure_scratch2(c, 11 * nd + 3 * nb + n4 + 64);
    if (rc) return rc;
    rc = ensure_copy_stream(c);
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
    // Host-to-device copies in FPIC_HOST_CHUNKS particle chunks on the
    // context's copy stream; the explicit pass of chunk j starts as soon as
    // its inputs have landed, overlapping the copies of the later chunks.
    // w is not read by the push and is not copied.
    long long bounds[FPIC_HOST_CHUNKS + 1];
    for (int j = 0; j <= FPIC_HOST_CHUNKS; ++j) bounds[j] = n * j / FPIC_HOST_CHUNKS;
    FPIC_CUDA(cudaEventRecord(c->copy_ev[FPIC_HOST_CHUNKS], s));
    FPIC_CUDA(cudaStreamWaitEvent(c->copy_stream, c->copy_ev[FPIC_HOST_CHUNKS], 0));
    for (int j = 0; j < FPIC_HOST_CHUNKS; ++j) {
        const size_t o = (size_t)bounds[j], len = (size_t)(bounds[j + 1] - bounds[j]);
        if (len) {
            for (int i = 0; i < 11; ++i)
                if (i != 7 && hd[i])
                    FPIC_CUDA(cudaMemcpyAsync(*dd[i] + o, hd[i] + o, len * sizeof(double), cudaMemcpyHostToDevice,
                                              c->copy_stream));
            FPIC_CUDA(cudaMemcpyAsync(d.alive + o, hp->alive + o, len, cudaMemcpyHostToDevice, c->copy_stream));
        }
        FPIC_CUDA(cudaEventRecord(c->copy_ev[j], c->copy_stream));
    }
    const PushChunks ch{FPIC_HOST_CHUNKS, bounds, c->copy_ev};
    rc = push_core(c, &d, fields, prm, stats, s, &ch);
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
    if (!c->async) FPIC_CUDA(cudaStreamSynchronize(s));
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
constexpr size_t kNoAllocBytes = kNoAllocCountersBytes + (size_t)kNoAllocMax * (8 * sizeof(double) + 2 * sizeof(uint32_t));

// Shared by every call on a device and held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Per-device set-up cache: the device address of g_noalloc_scratch (the host
// symbol is only a stand-in and must never be passed to a kernel) and the
// SM count, filled by the first call on each device and tagged with the ID of
// the CUDA context it was looked up in.  A later call under another context
// (after cudaDeviceReset, or from a driver-API context of its own) repeats
// the look-up, since the module and its array may then sit at another
// address.  One mutex guards the cache: host threads making their first calls
// at the same time see either no entry or a complete one.
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocSlot {
    unsigned long long ctx_id;
    void* ptr;
    int sms;
};
static NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the
// library does not link the driver library directly).
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

static int current_ctx_id(int dev, unsigned long long* id)
{
    static PfnCtxGetCurrent get_cur = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_cur || !get_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        FPIC_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0));
        FPIC_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1));
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return set_error(FPIC_ECUDA, "fpic_push_noalloc: driver entry points cuCtxGetCurrent/cuCtxGetId not found");
        get_cur = (PfnCtxGetCurrent)f0;
        get_id = (PfnCtxGetId)f1;
    }
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) {
        // no context bound to this thread yet: bind the device's primary one
        FPIC_CUDA(cudaSetDevice(dev));
        if (get_cur(&ctx) != CUDA_SUCCESS || !ctx)
            return set_error(FPIC_ECUDA, "fpic_push_noalloc: no current CUDA context on device %d", dev);
    }
    if (get_id(ctx, id) != CUDA_SUCCESS) return set_error(FPIC_ECUDA, "fpic_push_noalloc: cuCtxGetId failed");
    return 0;
}

static int noalloc_setup(int dev, void** ptr_out, int* sms_out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(FPIC_EINVAL, "fpic_push_noalloc: device id %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    int rc = current_ctx_id(dev, &id);
    if (rc) return rc;
    NoAllocSlot& sl = g_noalloc_slot[dev];
    if (!sl.ptr || sl.ctx_id != id) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return set_error(FPIC_ECUDA, "fpic_push_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        int sms = 0;
        FPIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (sms < 1) return set_error(FPIC_ECUDA, "fpic_push_noalloc: device %d reports %d SMs", dev, sms);
        sl = NoAllocSlot{id, ptr, sms};
    }
    *ptr_out = sl.ptr;
    *sms_out = sl.sms;
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
    if (!dt_implicit_ok(prm)) return set_error(FPIC_EINVAL, "fpic_push_noalloc: bad dt_implicit");
    if (prm->B0field != 0.0 && (!std::isfinite(prm->B0field) || M != 1.0))
        return set_error(FPIC_EINVAL, "fpic_push_noalloc: B0field needs a finite value and M = 1");
    if (prm->scheme < FPIC_RK4 || prm->scheme > FPIC_HYB2) return set_error(FPIC_EINVAL, "fpic_push_noalloc: unknown scheme %d", prm->scheme);
    if (prm->scheme >= FPIC_HYB1 && prm->implicit != FPIC_IMR && prm->implicit != FPIC_HAM)
        return set_error(FPIC_EINVAL, "fpic_push_noalloc: implicit partner must be FPIC_IMR or FPIC_HAM");
    if (prm->max_iter < 1 || prm->max_iter > 255) return set_error(FPIC_EINVAL, "fpic_push_noalloc: max_iter must be in [1, 255]");
    if (!(prm->tol >= 0.0)) return set_error(FPIC_EINVAL, "fpic_push_noalloc: tol must be >= 0");
    if (prm->guess) return set_error(FPIC_EINVAL, "fpic_push_noalloc: learned guesses are not supported here");
    if (prm->imr_substeps != 0) return set_error(FPIC_EINVAL, "fpic_push_noalloc: imr_substeps is not supported here");
    if (prm->before) return set_error(FPIC_EINVAL, "fpic_push_noalloc: before is not supported here");
    int dev = 0, sms = 0;
    void* scratch = nullptr;
    FPIC_CUDA(cudaGetDevice(&dev));
    int rc = noalloc_setup(dev, &scratch, &sms);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    unsigned char* base = (unsigned char*)scratch;
    PushK k{};
    k.run.bh = BH{M, a, a * a, 2.0 * M};
    k.run.has_grid = 0;
    k.run.has_fields = 0;
    k.dt = prm->dt;
    k.dt_imp = implicit_step(prm);
    k.imr_newton = prm->imr_newton ? 1 : 0;
    k.t = prm->t;
    k.thr = prm->thr;
    push_constants(k);
    k.tol = prm->tol;
    k.dg_eps = prm->dg_eps;
    k.run.B0pot = prm->B0pot;
    k.run.B0field = prm->B0field;
    k.run.r_h = M + sqrt(M * M - a * a);
    k.run.r_max = prm->r_max;
    k.scheme = prm->scheme;
    k.max_iter = prm->max_iter;
    k.n = n;
    k.P = PartDev{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                  p->alive, p->scheme, p->iters, p->cell};
    k.cnt = (long long*)base;
    k.guess = (double*)(base + kNoAllocCountersBytes);
    k.sc0 = k.guess + (size_t)n * 6;
    k.queue = (uint32_t*)(base + kNoAllocCountersBytes + (size_t)n * 8 * sizeof(double));
    k.order = k.queue + n;
    k.learned = nullptr;
    // the counters (queue length and head among them) must start at zero
    FPIC_CUDA(cudaMemsetAsync(k.cnt, 0, CNT_N * sizeof(long long), s));
    if (n == 0) {
        if (stats) *stats = fpic_push_stats{};
        return FPIC_OK;
    }
    const int TB = 128;
    const unsigned nb = (unsigned)((n + TB - 1) / TB);
    const unsigned persist = (unsigned)sms * 8u;
    cudaEvent_t* ev = prm->events ? (cudaEvent_t*)prm->events : nullptr;
    if (stats) k_count_alive<<<persist, 256, 0, s>>>(k.P, n, k.cnt);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[0], s));
    if (prm->scheme == FPIC_RK4) k_explicit<0><<<nb, TB, 0, s>>>(k);
    else if (prm->scheme >= FPIC_HYB1) k_explicit<1><<<nb, TB, 0, s>>>(k);
    if (ev) {
        FPIC_CUDA(cudaEventRecord(ev[1], s));
        FPIC_CUDA(cudaEventRecord(ev[2], s));
    }
    if (prm->scheme == FPIC_IMR) {
        launch_imr<0>(persist / 2, TB, s, k, 1);
        finish_implicit<>(persist, s, k, 1);
    } else if (prm->scheme == FPIC_HAM) {
        if (k.run.B0field != 0.0) k_dg_em<<<nb, TB, 0, s>>>(k, 1);
        else k_dg<<<nb, TB, 0, s>>>(k, 1);
    } else if (prm->scheme >= FPIC_HYB1 && prm->implicit == FPIC_IMR) {
        k_order<<<persist, 256, 0, s>>>(k);
        launch_imr<0>(persist / 2, TB, s, k, 0);
        finish_implicit<>(persist, s, k, 0);
    } else if (prm->scheme >= FPIC_HYB1) {
        if (k.run.B0field != 0.0) k_dg_em<<<nb, TB, 0, s>>>(k, 0);
        else k_dg<<<nb, TB, 0, s>>>(k, 0);
    }
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
        stats->n_slope_reused = 0;
        stats->n_tiles_staged = 0;
        if (h[CNT_NOTCONV] > 0) return FPIC_ENOTCONVERGED;
    }
    return FPIC_OK;
}


// ---------------------------------------------------------------------------
// Learned guess: features, sampling from the plain method, learned push.
// ---------------------------------------------------------------------------
namespace fpic {

struct FeatK {
    BH bh;
    GridDev G;
    const float* f32[6];    // FP32 copies of the six field arrays (inputs only)
    int has_fields;
    const double *r, *th, *ur, *uth, *uph, *qm, *H0, *D0, *Hn;
    const uint8_t* alive;
    long long n;
    float dt;
    float mean[16], istd[16];
    float* X;
    float* T;   // nullable: zero rows of removed particles
    float* S;
};

__device__ __forceinline__ float lerp_f(const float* f, int ld, int i, int j, float wr, float wt)
{
    const float* q = f + (size_t)i * ld + j;
    const float f00 = __ldg(q), f01 = __ldg(q + 1), f10 = __ldg(q + ld), f11 = __ldg(q + ld + 1);
    const float lo = fmaf(wt, f01 - f00, f00), hi = fmaf(wt, f11 - f10, f10);
    return fmaf(wr, hi - lo, lo);
}

__global__ void k_features(FeatK k)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= k.n) return;
    float f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = 0.f;
    if (!k.alive[p]) {
        for (int i = 0; i < 16; ++i) k.X[p * 16 + i] = 0.f;
        if (k.T) for (int i = 0; i < 16; ++i) k.T[p * 16 + i] = 0.f;
        if (k.S) k.S[p] = 0.f;
        return;
    }
    const double r = k.r[p], th = k.th[p];
    const float rf = (float)r, tf = (float)th;
    f[0] = __logf(rf);
    f[1] = tf;
    f[2] = (float)k.ur[p];
    f[3] = (float)k.uth[p];
    f[4] = (float)k.uph[p];
    float wr_cell = 0.f;
    if (k.has_fields) {
        const GridDev& G = k.G;
        int i0, i1, j0, j1;
        double w0, w1, v0, v1;
        const float lr = f[0];
        locate(G.rn, G.irn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i0, w0);
        locate(G.rh, G.irh, G.Nr, r, (lr - G.lrh0) * G.ilr, i1, w1);
        locate(G.tn, G.itn, G.Nth + 1, th, (tf - G.t0) * G.it, j0, v0);
        locate(G.th, G.ith, G.Nth, th, (tf - G.th0) * G.it, j1, v1);
        const float a0 = (float)w0, a1 = (float)w1, b0 = (float)v0, b1 = (float)v1;
        wr_cell = a0;
        f[5] = lerp_f(k.f32[0], G.ld, i1, j0, a1, b0);    // D^r  (i+1/2, j)
        f[6] = lerp_f(k.f32[1], G.ld, i0, j1, a0, b1);    // D^th (i, j+1/2)
        f[7] = lerp_f(k.f32[2], G.ld, i0, j0, a0, b0);    // D^ph (i, j)
        f[8] = lerp_f(k.f32[3], G.ld, i0, j1, a0, b1);    // B^r  (i, j+1/2)
        f[9] = lerp_f(k.f32[4], G.ld, i1, j0, a1, b0);    // B^th (i+1/2, j)
        f[10] = lerp_f(k.f32[5], G.ld, i1, j1, a1, b1);   // B^ph (i+1/2, j+1/2)
    }
    // the hybrid test depends on the current energy error and on where the
    // particle sits in its cell (the interpolation error pattern)
    f[11] = (float)((k.Hn[p] - k.H0[p]) / k.D0[p]);
    f[12] = wr_cell;
    f[13] = (float)k.qm[p] * k.dt;
#pragma unroll
    for (int i = 0; i < 14; ++i) k.X[p * 16 + i] = (f[i] - k.mean[i]) * k.istd[i];
    k.X[p * 16 + 14] = 0.f;
    k.X[p * 16 + 15] = 0.f;
}

// Route each alive particle: predicted rejected -> implicit queue (guess
// z^n + scale * y), else -> explicit work list.
__global__ void k_split(PushK k, float skip_logit)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= k.n) return;
    if (!k.P.alive[p]) {
        k.P.scheme[p] = 0;
        k.P.iters[p] = 0;
        return;
    }
    const float* y = k.learned + 16 * p;
    const bool skip = y[6] > skip_logit;
    const unsigned act = __activemask();
    const unsigned sk = __ballot_sync(act, skip);
    const int leader = __ffs(act) - 1;
    const int lane = threadIdx.x & 31;
    unsigned long long bq = 0, bw = 0;
    if (lane == leader) {
        if (sk) bq = atomicAdd((unsigned long long*)&k.cnt[CNT_QUEUE], (unsigned long long)__popc(sk));
        const unsigned nw = __popc(act & ~sk);
        if (nw) bw = atomicAdd((unsigned long long*)&k.cnt[CNT_WORK], (unsigned long long)nw);
    }
    bq = __shfl_sync(act, bq, leader);
    bw = __shfl_sync(act, bw, leader);
    if (skip) {
        k.queue[bq + __popc(sk & lanemask_lt())] = (uint32_t)p;
        const double z0[6] = {k.P.r[p], k.P.th[p], k.P.ph[p], k.P.ur[p], k.P.uth[p], k.P.uph[p]};
#pragma unroll
        for (int i = 0; i < 6; ++i) k.guess[(size_t)i * k.n + p] = fma(k.inc_scale[i], (double)y[i], z0[i]);
        double s0, c0;
        sincos(z0[1], &s0, &c0);
        k.sc0[p] = s0;
        k.sc0[k.n + p] = c0;
    } else {
        k.work[bw + __popc(act & ~sk & lanemask_lt())] = (uint32_t)p;
    }
}

static bool push_prm_ok(const fpic_push_params* prm)
{
    return std::isfinite(prm->dt) && prm->dt != 0.0 && prm->scheme >= FPIC_HYB1 && prm->scheme <= FPIC_HYB2 &&
           prm->implicit == FPIC_IMR && prm->max_iter >= 1 && prm->max_iter <= 255 && prm->tol >= 0.0 &&
           prm->imr_substeps >= 0 && prm->imr_substeps <= 12 && prm->substep_tol >= 0.0 &&
           std::isfinite(prm->substep_tol);
}

static void fill_pushk(PushK& k, fpic_ctx* c, fpic_particles* p, const double* const fields[6],
                       const fpic_push_params* prm)
{
    k.run.bh = c->bh;
    k.run.G = c->G;
    k.run.has_grid = c->has_grid;
    k.run.has_fields = fields != nullptr;
    for (int i = 0; i < 6; ++i) k.run.F.f[i] = fields ? fields[i] : nullptr;
    k.dt = prm->dt;
    k.dt_imp = prm->dt;
    k.imr_newton = prm->imr_newton ? 1 : 0;
    k.t = nullptr;
    k.thr = prm->thr;
    push_constants(k);
    k.tol = prm->tol;
    k.dg_eps = prm->dg_eps;
    k.run.B0pot = prm->B0pot;
    k.run.B0field = 0.0;
    k.run.r_h = c->r_h;
    k.run.r_max = prm->r_max;
    k.scheme = prm->scheme;
    k.max_iter = prm->max_iter;
    k.substeps = prm->imr_substeps;
    k.substep_tol = prm->substep_tol;
    k.n = p->n;
    k.P = PartDev{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                  p->alive, p->scheme, p->iters, p->cell};
    k.cnt = c->d_cnt;
}

// scratch: guess 6n doubles | sc0 2n doubles | stg STG_ROWS n doubles | queue n | work n | order n | strag n | X 16n floats |
// Y 16n floats | featS 16n floats | 6 FP32 field copies
static int learned_scratch(fpic_ctx* c, long long n, PushK& k, float** X, float** Y, float** f32)
{
    const size_t fsz = c->has_grid ? 6 * (size_t)(c->Nr + 1) * c->ld : 0;
    const size_t need = (size_t)n * ((8 + STG_ROWS) * sizeof(double) + 4 * sizeof(uint32_t) + 48 * sizeof(float) + 1) +
                        fsz * sizeof(float) + 2048;
    int rc = ensure_scratch(c, need);
    if (rc) return rc;
    char* b = (char*)c->d_scratch;
    k.guess = (double*)b;
    b += (size_t)n * 6 * sizeof(double);
    k.sc0 = (double*)b;
    b += (size_t)n * 2 * sizeof(double);
    k.stg = (double*)b;
    b += (size_t)n * STG_ROWS * sizeof(double);
    k.queue = (uint32_t*)b;
    b += (size_t)n * sizeof(uint32_t);
    k.work = (uint32_t*)b;
    b += (size_t)n * sizeof(uint32_t);
    k.order = (uint32_t*)b;
    b += (size_t)n * sizeof(uint32_t);
    k.strag = (uint32_t*)b;
    b += (size_t)n * sizeof(uint32_t);
    b = (char*)(((uintptr_t)b + 255) & ~(uintptr_t)255);
    *X = (float*)b;
    b += (size_t)n * 16 * sizeof(float);
    *Y = (float*)b;
    b += (size_t)n * 16 * sizeof(float);
    k.featS = (float*)b;
    b += (size_t)n * 16 * sizeof(float);
    *f32 = (float*)b;
    b += fsz * sizeof(float);
    k.strag_flag = (uint8_t*)b;
    return 0;
}

static void set_corrector(PushK& k, const fpic_learned_cfg* cfg, float* X)
{
    k.featX = X;
    k.restart_after = cfg->restart_after;
    for (int i = 0; i < 6; ++i) k.oscale[i] = cfg->inc_scale[i] > 0.0 ? (float)cfg->inc_scale[i] : 1.f;
    for (int i = 0; i < 14; ++i) {
        k.fmean[i] = cfg->feat_mean[i];
        k.fistd[i] = cfg->feat_std[i] > 0.f ? 1.f / cfg->feat_std[i] : 1.f;
    }
}

// Corrector form, implicit-queue slot idx (particle p = queue[idx]): the 14
// trial features f and, per component, the scale s_i and the leading-order
// gap g_i between the implicit midpoint step and the RK4 trial.  From the
// slopes parked in stg: A = dt (k3 - k2), B = dt (k4 - 2 k2 + k1) with
// k3 = (acc - k1) / 2 - k2; features A_i / s_i, B_i / s_i (s_i = |A_i| +
// |B_i|, zero when both vanish), ln r and ln(|A| / |z_RK4 - z^n|) over u_r,
// u_th (a measure of the step's expansion parameter (omega dt)^2), then
// standardised.  g = (2/3) A - (1/6) B: expanding both steps in dt,
// IMR - RK4 = dt^3 (f'f'f / 12 - f''(f,f) / 24) + O(dt^4), while k3 - k2 =
// dt^2 f'f'f / 4 + O(dt^3) and k4 - 2 k2 + k1 = dt^2 (f'f'f / 2 +
// f''(f,f) / 4) + O(dt^3).  FP32 after the differences: the features feed
// a bf16 network and the gap only has to be a good start for the solve.
__device__ __forceinline__ void trial_row(const PushK& k, long long idx, float f[16], float sc[6], float gl[6],
                                          float dz[6])
{
    const float dt = (float)k.dt;
    float num = 0.f, den = 0.f;
    double r0 = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double k1 = k.stg[(size_t)(STG_K1 + i) * k.n + idx], k2 = k.stg[(size_t)(STG_K2 + i) * k.n + idx];
        const double acc = k.stg[(size_t)(STG_ACC + i) * k.n + idx], k4 = k.stg[(size_t)(STG_K4 + i) * k.n + idx];
        const double z0 = k.stg[(size_t)(STG_Z0 + i) * k.n + idx];
        if (i == 0) r0 = z0;
        // the differences in FP64 (they cancel), the rest in FP32
        const float a = dt * (float)fma(0.5, acc - k1, -2.0 * k2);
        const float b = dt * (float)((k4 - k2) - (k2 - k1));
        dz[i] = fabsf((float)(k.stg[(size_t)(STG_TRIAL + i) * k.n + idx] - z0));
        const float sm = fabsf(a) + fabsf(b);
        gl[i] = fmaf(2.f / 3.f, a, -b * (1.f / 6.f));
        const float is = sm > 0.f ? 1.f / sm : 0.f;
        f[i] = a * is;
        f[6 + i] = b * is;
        sc[i] = sm;
        if (i == 3 || i == 4) {
            num += fabsf(a);
            den += dz[i];
        }
    }
    f[12] = __logf((float)r0);
    f[13] = (num > 0.f && den > 0.f) ? __logf(num / den) : 0.f;
#pragma unroll
    for (int i = 0; i < 14; ++i) f[i] = (f[i] - k.fmean[i]) * k.fistd[i];
    f[14] = f[15] = 0.f;
}

// Sampling (corrector form): features of every queue slot to featX, the
// scales s_i and gaps g_i to featS (0-5, 8-13).
__global__ void k_trial_feat(PushK k)
{
    const long long qn = k.cnt[CNT_QUEUE];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < qn;
         idx += (long long)gridDim.x * blockDim.x) {
        float f[16], sc[6], gl[6], dz[6];
        trial_row(k, idx, f, sc, gl, dz);
        float4* x = (float4*)(k.featX + 16 * idx);
        float4* o = (float4*)(k.featS + 16 * idx);
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        o[0] = make_float4(sc[0], sc[1], sc[2], sc[3]);
        o[1] = make_float4(sc[4], sc[5], 0.f, 0.f);
        o[2] = make_float4(gl[0], gl[1], gl[2], gl[3]);
        o[3] = make_float4(gl[4], gl[5], 0.f, 0.f);
    }
}

// Guard of the corrector: the IMR - RK4 gap is O(dt^3) against the O(dt)
// step, so a component whose correction exceeds CORR_MAX times the trial's
// own increment (or whose output is outside [-16, 16] or not finite) keeps
// the trial value.
constexpr float CORR_MAX = 0.05f;

// Corrector form in the push, one fused persistent kernel per step
// (mlp_dev.cuh): one CTA of 512 threads per SM runs four independent
// 128-slot tile pipelines of the implicit queue (its length read on the
// device) over the shared resident weights.  Thread t % 128 of group t / 128
// builds its slot's features straight into the group's bf16 input tile,
// the four layers run on the tensor cores, and the same thread applies its
// row's output: the slot's implicit guess (stg, read by k_imr<1>) becomes
// z_RK4 + g_i + s_i oscale_i y_i.
__global__ void __launch_bounds__(G4_THREADS, 1) k_mlp_correct4(PushK k, MlpDev w, int* err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const long long qn = k.cnt[CNT_QUEUE];
    const long long ntiles = (qn + 127) / 128;
    if ((long long)blockIdx.x * G4_GROUPS >= ntiles) return;     // whole block, before any allocation
    const float* sb = (const float*)(smem + G4_B);
    const int g = threadIdx.x >> 7, r = threadIdx.x & 127, wq = (threadIdx.x >> 5) & 3;
    const uint32_t tbase0 = mlp_cta_setup4(w, smem);
    const uint32_t tbase = tbase0 + (uint32_t)(128 * g);
    uint64_t* mbar = (uint64_t*)(smem + G4_BAR) + g;
    uint8_t* sX = smem + G4_TILE0 + g * G4_TILE_BYTES;
    uint32_t phase = 0;
    int ok = 1;
    for (long long tile = (long long)blockIdx.x * G4_GROUPS + g; tile < ntiles && ok;
         tile += (long long)gridDim.x * G4_GROUPS) {
        const long long idx = tile * 128 + r;
        const bool valid = idx < qn;
        float f[16], sc[6], gl[6], dz[6];
        if (valid) {
            trial_row(k, idx, f, sc, gl, dz);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) f[i] = 0.f;
        }
        *(uint4*)(sX + tc::kmajor_off(r, 0, 128)) =
            make_uint4(tc::pack_bf2(f[0], f[1]), tc::pack_bf2(f[2], f[3]), tc::pack_bf2(f[4], f[5]),
                       tc::pack_bf2(f[6], f[7]));
        *(uint4*)(sX + tc::kmajor_off(r, 8, 128)) =
            make_uint4(tc::pack_bf2(f[8], f[9]), tc::pack_bf2(f[10], f[11]), tc::pack_bf2(f[12], f[13]),
                       tc::pack_bf2(f[14], f[15]));
        ok = mlp_tile_layers_g(g, tbase, smem, mbar, phase);
        if (!ok) break;
        float v[16];
        tc::tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16), v);
        if (valid) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const float y = v[i] + sb[384 + i];
                const double zt = k.stg[(size_t)(STG_TRIAL + i) * k.n + idx];
                const double z0 = k.stg[(size_t)(STG_Z0 + i) * k.n + idx];
                const float d = fmaf(sc[i] * k.oscale[i], y, gl[i]);
                const bool use = fabsf(y) <= 16.f && fabsf(d) <= CORR_MAX * (float)fabs(zt - z0);
                k.stg[(size_t)(STG_GUESS + i) * k.n + idx] = use ? zt + (double)d : zt;
            }
        }
    }
    mlp_cta_teardown4(tbase0, ok, err);
}


// FP32 copies of the field arrays (network inputs are rounded to bf16 anyway;
// converting the grid once is cheaper than converting 24 gathered values per
// particle on the FP64 pipe).
__global__ void k_fields_f32(Fields F, float* out, size_t sz)
{
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < sz; o += (size_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 6; ++k) out[k * sz + o] = (float)F.f[k][o];
}

static FeatK make_featk(fpic_ctx* c, const fpic_particles* p, const double* const fields[6], double dt,
                        const fpic_learned_cfg* cfg, float* X, float* f32, cudaStream_t s)
{
    FeatK f{};
    f.bh = c->bh;
    f.G = c->G;
    f.has_fields = fields != nullptr;
    if (fields) {
        const size_t sz = (size_t)(c->Nr + 1) * c->ld;
        Fields F;
        for (int i = 0; i < 6; ++i) F.f[i] = fields[i];
        k_fields_f32<<<256, 256, 0, s>>>(F, f32, sz);
        for (int i = 0; i < 6; ++i) f.f32[i] = f32 + i * sz;
    }
    f.r = p->r; f.th = p->th; f.ur = p->ur; f.uth = p->uth; f.uph = p->uph; f.qm = p->qm;
    f.H0 = p->H0; f.D0 = p->D0; f.Hn = p->Hn;
    f.alive = p->alive;
    f.n = p->n;
    f.dt = (float)dt;
    for (int i = 0; i < 16; ++i) {
        f.mean[i] = cfg ? cfg->feat_mean[i] : 0.f;
        const float sd = cfg ? cfg->feat_std[i] : 1.f;
        f.istd[i] = sd > 0.f ? 1.f / sd : 1.f;
    }
    f.X = X;
    return f;
}

}  // namespace fpic

extern "C" int fpic_features(fpic_ctx* c, const fpic_particles* p, const double* const fields[6], double dt,
                             const fpic_learned_cfg* cfg, float* X, void* stream)
{
    if (c && c->G.full) return set_error(FPIC_EINVAL, "fpic_features: not built for the full-theta domain");
    if (!c || !p || !X) return set_error(FPIC_EINVAL, "fpic_features: NULL argument");
    if (p->n < 0) return set_error(FPIC_EINVAL, "fpic_features: n < 0");
    if (fields && !c->has_grid) return set_error(FPIC_EINVAL, "fpic_features: fields given but no grid set");
    if (p->n == 0) return FPIC_OK;
    FPIC_CUDA(cudaSetDevice(c->device));
    PushK k{};
    float *Xs, *Ys, *f32;
    int rc = learned_scratch(c, p->n, k, &Xs, &Ys, &f32);
    if (rc) return rc;
    FeatK f = make_featk(c, p, fields, dt, cfg, X, f32, (cudaStream_t)stream);
    k_features<<<(unsigned)((p->n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(f);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_learn_sample(fpic_ctx* c, fpic_particles* p, const double* const fields[6],
                                 const fpic_push_params* prm, const fpic_learned_cfg* cfg, float* X, float* T,
                                 float* S, void* stream)
{
    if (!c || !p || !prm || !X || !T || !S) return set_error(FPIC_EINVAL, "fpic_learn_sample: NULL argument");
    if ((!cfg || cfg->mode == FPIC_LEARN_SKIP) && c->G.full)
        return set_error(FPIC_EINVAL, "fpic_learn_sample: the skip form is not built for the full-theta domain");
    if (!push_prm_ok(prm)) return set_error(FPIC_EINVAL, "fpic_learn_sample: need a Hyb1/Hyb2 scheme with the IMR partner");
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_learn_sample: n out of range");
    if (!particles_ok(p, true)) return set_error(FPIC_EINVAL, "fpic_learn_sample: NULL particle array");
    if (fields && !c->has_grid) return set_error(FPIC_EINVAL, "fpic_learn_sample: fields given but no grid set");
    if (p->n == 0) return FPIC_OK;
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    PushK k{};
    fill_pushk(k, c, p, fields, prm);
    float *Xs, *Ys, *f32;
    int rc = learned_scratch(c, n, k, &Xs, &Ys, &f32);
    if (rc) return rc;
    if (fields) {
        rc = field_coefs(c, fields, k.run, s);
        if (rc) return rc;
    }
    k.work = nullptr;
    k.record = 1;
    k.recT = T;
    k.recS = S;
    for (int i = 0; i < 6; ++i) k.inc_scale[i] = cfg ? cfg->inc_scale[i] : 1.0;
    FPIC_CUDA(cudaMemsetAsync(c->d_cnt, 0, CNT_N * sizeof(long long), s));
    const unsigned nb = (unsigned)((n + 127) / 128);
    if (cfg && cfg->mode == FPIC_LEARN_CORRECT) {
        // rows = implicit-queue slots (every alive particle is queued)
        FPIC_CUDA(cudaMemsetAsync(X, 0, (size_t)n * 16 * sizeof(float), s));
        FPIC_CUDA(cudaMemsetAsync(T, 0, (size_t)n * 16 * sizeof(float), s));
        FPIC_CUDA(cudaMemsetAsync(S, 0, (size_t)n * sizeof(float), s));
        set_corrector(k, cfg, X);
        k.order = nullptr;
        k_explicit<2><<<nb, 128, 0, s>>>(k);
        k_trial_feat<<<(unsigned)c->sm_count * 8u, 256, 0, s>>>(k);
        launch_imr<0>((unsigned)c->sm_count * (unsigned)c->imr_blocks_per_sm, 128, s, k, 0);
        FPIC_CUDA(cudaGetLastError());
        return FPIC_OK;
    }
    k.featS = nullptr;
    k.order = nullptr;
    FeatK f = make_featk(c, p, fields, prm->dt, cfg, X, f32, s);
    f.T = T;
    f.S = S;
    k_features<<<nb, 128, 0, s>>>(f);
    k_explicit<1><<<nb, 128, 0, s>>>(k);
    launch_imr<0>((unsigned)c->sm_count * (unsigned)c->imr_blocks_per_sm, 128, s, k, 0);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_push_learned(fpic_ctx* c, fpic_mlp* m, fpic_particles* p, const double* const fields[6],
                                 const fpic_push_params* prm, const fpic_learned_cfg* cfg, fpic_push_stats* stats,
                                 void* stream)
{
    if (!c || !m || !p || !prm || !cfg) return set_error(FPIC_EINVAL, "fpic_push_learned: NULL argument");
    if (!push_prm_ok(prm)) return set_error(FPIC_EINVAL, "fpic_push_learned: need a Hyb1/Hyb2 scheme with the IMR partner");
    if (prm->dt_implicit != 0.0 && prm->dt_implicit != prm->dt)
        return set_error(FPIC_EINVAL, "fpic_push_learned: the learned guess is trained for dt_implicit = dt");
    if (prm->B0field != 0.0) return set_error(FPIC_EINVAL, "fpic_push_learned: B0field is not supported");
    if (prm->before) return set_error(FPIC_EINVAL, "fpic_push_learned: before is not supported");
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_push_learned: n out of range");
    if (!particles_ok(p, true)) return set_error(FPIC_EINVAL, "fpic_push_learned: NULL particle array");
    if (fields && !c->has_grid) return set_error(FPIC_EINVAL, "fpic_push_learned: fields given but no grid set");
    if (cfg->mode != FPIC_LEARN_SKIP && cfg->mode != FPIC_LEARN_CORRECT)
        return set_error(FPIC_EINVAL, "fpic_push_learned: unknown cfg->mode");
    if (cfg->mode == FPIC_LEARN_SKIP && !(cfg->p_skip > 0.f && cfg->p_skip < 1.f))
        return set_error(FPIC_EINVAL, "fpic_push_learned: p_skip must be in (0, 1)");
    if (cfg->mode == FPIC_LEARN_SKIP && c->G.full)
        return set_error(FPIC_EINVAL, "fpic_push_learned: the skip form is not built for the full-theta domain");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    PushK k{};
    fill_pushk(k, c, p, fields, prm);
    float *X, *Y, *f32;
    int rc = learned_scratch(c, n > 0 ? n : 1, k, &X, &Y, &f32);
    if (rc) return rc;
    if (fields && n > 0) {
        rc = field_coefs(c, fields, k.run, s);
        if (rc) return rc;
    }
    for (int i = 0; i < 6; ++i) k.inc_scale[i] = cfg->inc_scale[i];
    k.learned = Y;
    rc = slope_setup(c, p, fields, 0.0, k);
    if (rc) return rc;
    FPIC_CUDA(cudaMemsetAsync(c->d_cnt, 0, CNT_N * sizeof(long long), s));
    if (n == 0) {
        if (stats) *stats = fpic_push_stats{};
        return FPIC_OK;
    }
    if (k.substeps > 0) FPIC_CUDA(cudaMemsetAsync(k.strag_flag, 0, (size_t)n, s));
    const unsigned nb = (unsigned)((n + 127) / 128);
    const unsigned persist = (unsigned)c->sm_count * 8u;
    cudaEvent_t* ev = prm->events ? (cudaEvent_t*)prm->events : nullptr;
    if (stats) k_count_alive<<<persist, 256, 0, s>>>(k.P, n, c->d_cnt);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[0], s));
    const bool correct = cfg->mode == FPIC_LEARN_CORRECT;
    if (correct) {
        // RK4 trial + plain test for all; network on the rejected ones only
        k.work = nullptr;
        set_corrector(k, cfg, X);
        k_explicit<2><<<nb, 128, 0, s>>>(k);
        if (ev) FPIC_CUDA(cudaEventRecord(ev[1], s));
        static bool attr_set = false;
        if (!attr_set) {
            FPIC_CUDA(cudaFuncSetAttribute(k_mlp_correct4, cudaFuncAttributeMaxDynamicSharedMemorySize, G4_SMEM));
            attr_set = true;
        }
        // one CTA of four tile pipelines per SM; the kernel reads the queue
        // length itself and idle CTAs leave at once
        const long long nct = (n + 127) / 128 / G4_GROUPS + 1, cap = mlp_sm_count(m);
        k_mlp_correct4<<<(unsigned)(nct < cap ? nct : cap), G4_THREADS, G4_SMEM, s>>>(k, mlp_weights(m),
                                                                                      mlp_err(m));
        if (ev) FPIC_CUDA(cudaEventRecord(ev[2], s));
    } else {
        // network on every particle first; predicted rejections skip the trial
        k.featS = nullptr;
        FeatK f = make_featk(c, p, fields, prm->dt, cfg, X, f32, s);
        k_features<<<nb, 128, 0, s>>>(f);
        rc = mlp_forward_dev(m, X, Y, n, s);
        if (rc) return rc;
        const float skip_logit = logf(cfg->p_skip / (1.f - cfg->p_skip));
        k_split<<<nb, 128, 0, s>>>(k, skip_logit);
        k_explicit<1><<<nb, 128, 0, s>>>(k);
        if (ev) {
            FPIC_CUDA(cudaEventRecord(ev[1], s));
            FPIC_CUDA(cudaEventRecord(ev[2], s));
        }
        k.work = nullptr;
    }
    const unsigned imr_grid = (unsigned)c->sm_count * (unsigned)c->imr_blocks_per_sm;
    k_order<<<persist, 256, 0, s>>>(k);
    if (correct) launch_imr<1>(imr_grid, 128, s, k, 0);
    else launch_imr<0>(imr_grid, 128, s, k, 0);
    finish_implicit<>(persist, s, k, 0);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[3], s));
    FPIC_CUDA(cudaGetLastError());
    if (stats) {
        FPIC_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, CNT_N * sizeof(long long), cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        const long long* h = c->h_cnt;
        stats->n_alive_before = h[CNT_ALIVE];
        stats->n_implicit = h[CNT_QUEUE];
        stats->n_iter_total = h[CNT_ITERS];
        stats->n_notconv = h[CNT_NOTCONV];
        stats->n_removed = h[CNT_REMOVED];
        stats->n_rhs_evals = h[CNT_EVALS] + 4 * (correct ? h[CNT_ALIVE] : h[CNT_WORK]);
        stats->n_slope_reused = h[CNT_SLOPE];
        stats->n_tiles_staged = 0;
        if (k.slope) stats->n_rhs_evals += (correct ? h[CNT_ALIVE] : h[CNT_WORK]) - h[CNT_SLOPE] + h[CNT_QUEUE];
        if (h[CNT_NOTCONV] > 0) return FPIC_ENOTCONVERGED;
    }
    return FPIC_OK;
}


// ---------------------------------------------------------------------------
// Batched push: many independent runs (spacetime, grid, fields, particle
// range) in one explicit launch and one persistent implicit launch.
// ---------------------------------------------------------------------------
// The batched push, plain (m == nullptr) or with the learned corrector (m,
// cfg: the corrector form of fpic_push_learned on the batched kernels).
static int push_batched(const fpic_run* runs, int nruns, fpic_mlp* m, fpic_particles* p, const fpic_push_params* prm,
                        const fpic_learned_cfg* cfg, fpic_push_stats* stats, void* stream)
{
    if (!runs || nruns < 1 || !p || !prm) return set_error(FPIC_EINVAL, "fpic_push_batched: NULL argument or nruns < 1");
    if (m) {
        if (!cfg || cfg->mode != FPIC_LEARN_CORRECT)
            return set_error(FPIC_EINVAL, "fpic_push_batched_learned: need a corrector-form cfg (FPIC_LEARN_CORRECT)");
        if (prm->scheme != FPIC_HYB1 && prm->scheme != FPIC_HYB2)
            return set_error(FPIC_EINVAL, "fpic_push_batched_learned: need a Hyb1/Hyb2 scheme with the IMR partner");
        if (prm->dt_implicit != 0.0 && prm->dt_implicit != prm->dt)
            return set_error(FPIC_EINVAL, "fpic_push_batched_learned: the learned guess is trained for dt_implicit = dt");
    }
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_push_batched: n out of range");
    if (!particles_ok(p, true)) return set_error(FPIC_EINVAL, "fpic_push_batched: NULL particle array");
    if (!(std::isfinite(prm->dt)) || prm->dt == 0.0) return set_error(FPIC_EINVAL, "fpic_push_batched: bad dt");
    if (!dt_implicit_ok(prm)) return set_error(FPIC_EINVAL, "fpic_push_batched: bad dt_implicit");
    if (prm->B0field != 0.0) return set_error(FPIC_EINVAL, "fpic_push_batched: B0field is not supported");
    if (prm->before) return set_error(FPIC_EINVAL, "fpic_push_batched: before is not supported");
    if (prm->scheme != FPIC_RK4 && prm->scheme != FPIC_IMR && prm->scheme != FPIC_HYB1 && prm->scheme != FPIC_HYB2)
        return set_error(FPIC_EINVAL, "fpic_push_batched: scheme must be RK4, IMR, Hyb1 or Hyb2");
    if (prm->scheme >= FPIC_HYB1 && prm->implicit != FPIC_IMR)
        return set_error(FPIC_EINVAL, "fpic_push_batched: the implicit partner must be FPIC_IMR");
    if (prm->max_iter < 1 || prm->max_iter > 255 || !(prm->tol >= 0.0))
        return set_error(FPIC_EINVAL, "fpic_push_batched: bad max_iter or tol");
    if (prm->imr_substeps < 0 || prm->imr_substeps > 12 || !(prm->substep_tol >= 0.0) || !std::isfinite(prm->substep_tol))
        return set_error(FPIC_EINVAL, "fpic_push_batched: imr_substeps must be in [0, 12] and substep_tol finite and >= 0");
    fpic_ctx* c = runs[0].ctx;
    if (!c) return set_error(FPIC_EINVAL, "fpic_push_batched: runs[0].ctx is NULL");
    for (int i = 0; i < nruns; ++i) {
        const fpic_run& r = runs[i];
        if (!r.ctx || r.ctx->device != c->device) return set_error(FPIC_EINVAL, "fpic_push_batched: run %d: bad ctx", i);
        if (r.begin != (i == 0 ? 0 : runs[i - 1].end) || r.end < r.begin)
            return set_error(FPIC_EINVAL, "fpic_push_batched: runs must tile [0, n) in order (run %d)", i);
        const int nf = (r.fields[0] != nullptr) + (r.fields[1] != nullptr) + (r.fields[2] != nullptr) +
                       (r.fields[3] != nullptr) + (r.fields[4] != nullptr) + (r.fields[5] != nullptr);
        if (nf != 0 && nf != 6) return set_error(FPIC_EINVAL, "fpic_push_batched: run %d: give all six fields or none", i);
        if (nf == 6 && !r.ctx->has_grid) return set_error(FPIC_EINVAL, "fpic_push_batched: run %d: fields but no grid", i);
    }
    if (runs[nruns - 1].end != p->n) return set_error(FPIC_EINVAL, "fpic_push_batched: the runs must end at n");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    if (c->runs_cap < nruns) {
        retire(c, &c->d_runs);
        retire(c, &c->h_runs, true);
        c->runs_cap = 0;
        FPIC_CUDA(cudaMalloc(&c->d_runs, sizeof(RunK) * nruns));
        FPIC_CUDA(cudaMallocHost(&c->h_runs, sizeof(RunK) * nruns));
        c->runs_cap = nruns;
    }
    const long long nn = n > 0 ? n : 1;
    PushK k{};
    float *X = nullptr, *Y = nullptr, *f32 = nullptr;
    int rc = m ? learned_scratch(c, nn, k, &X, &Y, &f32)
               : ensure_scratch(c, (size_t)nn * (8 * sizeof(double) + 3 * sizeof(uint32_t) + 1) + 256);
    if (rc) return rc;
    std::vector<RunK> tab(nruns);
    for (int i = 0; i < nruns; ++i) {
        const fpic_run& r = runs[i];
        RunK R{};
        R.bh = r.ctx->bh;
        R.G = r.ctx->G;
        R.has_grid = r.ctx->has_grid;
        R.has_fields = r.fields[0] != nullptr;
        for (int q = 0; q < 6; ++q) R.F.f[q] = r.fields[q];
        R.B0pot = r.B0pot;
        R.r_h = r.ctx->r_h;
        R.r_max = r.r_max;
        R.begin = r.begin;
        R.end = r.end;
        // interpolation coefficients in the run's context (when no other run shares it)
        int uses = 0;
        for (int j = 0; j < nruns; ++j) uses += runs[j].ctx == r.ctx ? 1 : 0;
        if (R.has_fields && uses == 1 && r.end > r.begin) {
            int rc0 = field_coefs(r.ctx, r.fields, R, s);
            if (rc0) return rc0;
        }
        tab[i] = R;
    }
    // The pinned staging table is rewritten only when it changes; outside a
    // stream capture the previous asynchronous copy out of it is waited for
    // first.  (A captured graph reads the table at replay time.)
    if (memcmp(c->h_runs, tab.data(), sizeof(RunK) * nruns) != 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        FPIC_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) FPIC_CUDA(cudaStreamSynchronize(s));
        memcpy(c->h_runs, tab.data(), sizeof(RunK) * nruns);
    }
    FPIC_CUDA(cudaMemcpyAsync(c->d_runs, c->h_runs, sizeof(RunK) * nruns, cudaMemcpyHostToDevice, s));
    // the single-run kernels with a per-particle run lookup (BATCHED)
    k.runs = (const RunK*)c->d_runs;
    k.nruns = nruns;
    k.dt = prm->dt;
    k.dt_imp = implicit_step(prm);
    k.imr_newton = prm->imr_newton ? 1 : 0;
    k.t = prm->t;
    k.thr = prm->thr;
    push_constants(k);
    k.tol = prm->tol;
    k.dg_eps = prm->dg_eps;
    k.scheme = prm->scheme;
    k.max_iter = prm->max_iter;
    k.n = n;
    k.P = PartDev{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                  p->alive, p->scheme, p->iters, p->cell};
    if (m) {
        // buffers laid out by learned_scratch; the corrector's parameters
        set_corrector(k, cfg, X);
        for (int i = 0; i < 6; ++i) k.inc_scale[i] = cfg->inc_scale[i];
        k.learned = Y;
        k.work = nullptr;
    } else {
        k.guess = (double*)c->d_scratch;
        k.sc0 = k.guess + (size_t)nn * 6;
        k.queue = (uint32_t*)((char*)c->d_scratch + (size_t)nn * 8 * sizeof(double));
        k.order = k.queue + nn;
        k.strag = k.order + nn;
        k.strag_flag = (uint8_t*)(k.strag + nn);
    }
    k.substeps = prm->imr_substeps;
    k.substep_tol = prm->substep_tol;
    k.cnt = c->d_cnt;
    FPIC_CUDA(cudaMemsetAsync(c->d_cnt, 0, CNT_N * sizeof(long long), s));
    if (n == 0) {
        if (stats) *stats = fpic_push_stats{};
        return FPIC_OK;
    }
    if (k.substeps > 0) FPIC_CUDA(cudaMemsetAsync(k.strag_flag, 0, (size_t)n, s));
    const unsigned nb = (unsigned)((n + 127) / 128);
    const unsigned persist = (unsigned)c->sm_count * 8u;
    const unsigned imr_grid = (unsigned)c->sm_count * (unsigned)c->imr_blocks_per_sm;
    cudaEvent_t* ev = prm->events ? (cudaEvent_t*)prm->events : nullptr;
    if (stats) k_count_alive<<<persist, 256, 0, s>>>(k.P, n, c->d_cnt);
    if (ev) FPIC_CUDA(cudaEventRecord(ev[0], s));
    if (m) {
        // RK4 trial + plain test for all; the network on the rejected ones
        k_explicit<2, true><<<nb, 128, 0, s>>>(k);
        if (ev) FPIC_CUDA(cudaEventRecord(ev[1], s));
        FPIC_CUDA(cudaFuncSetAttribute(k_mlp_correct4, cudaFuncAttributeMaxDynamicSharedMemorySize, G4_SMEM));
        const long long nct = (n + 127) / 128 / G4_GROUPS + 1, cap = mlp_sm_count(m);
        k_mlp_correct4<<<(unsigned)(nct < cap ? nct : cap), G4_THREADS, G4_SMEM, s>>>(k, mlp_weights(m), mlp_err(m));
        if (ev) FPIC_CUDA(cudaEventRecord(ev[2], s));
        k_order<<<persist, 256, 0, s>>>(k);
        launch_imr<1, true>(imr_grid, 128, s, k, 0);
        finish_implicit<true>(persist, s, k, 0);
    } else {
        if (prm->scheme == FPIC_RK4) k_explicit<0, true><<<nb, 128, 0, s>>>(k);
        else if (prm->scheme >= FPIC_HYB1) k_explicit<1, true><<<nb, 128, 0, s>>>(k);
        if (ev) {
            FPIC_CUDA(cudaEventRecord(ev[1], s));
            FPIC_CUDA(cudaEventRecord(ev[2], s));
        }
        if (prm->scheme == FPIC_IMR) {
            launch_imr<0, true>(imr_grid, 128, s, k, 1);
            finish_implicit<true>(persist, s, k, 1);
        } else if (prm->scheme >= FPIC_HYB1) {
            k_order<<<persist, 256, 0, s>>>(k);
            launch_imr<0, true>(imr_grid, 128, s, k, 0);
            finish_implicit<true>(persist, s, k, 0);
        }
    }
    if (ev) FPIC_CUDA(cudaEventRecord(ev[3], s));
    FPIC_CUDA(cudaGetLastError());
    if (stats) {
        FPIC_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, CNT_N * sizeof(long long), cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        const long long* h = c->h_cnt;
        stats->n_alive_before = h[CNT_ALIVE];
        stats->n_implicit = prm->scheme == FPIC_RK4 ? 0 : (prm->scheme >= FPIC_HYB1 ? h[CNT_QUEUE] : h[CNT_ALIVE]);
        stats->n_iter_total = h[CNT_ITERS];
        stats->n_notconv = h[CNT_NOTCONV];
        stats->n_removed = h[CNT_REMOVED];
        stats->n_rhs_evals = h[CNT_EVALS] + (prm->scheme != FPIC_IMR ? 4 * h[CNT_ALIVE] : 0);
        stats->n_slope_reused = 0;
        stats->n_tiles_staged = 0;
        if (h[CNT_NOTCONV] > 0) return FPIC_ENOTCONVERGED;
    }
    return FPIC_OK;
}

extern "C" int fpic_push_batched(const fpic_run* runs, int nruns, fpic_particles* p, const fpic_push_params* prm,
                                 fpic_push_stats* stats, void* stream)
{
    return push_batched(runs, nruns, nullptr, p, prm, nullptr, stats, stream);
}

extern "C" int fpic_push_batched_learned(const fpic_run* runs, int nruns, fpic_mlp* m, fpic_particles* p,
                                         const fpic_push_params* prm, const fpic_learned_cfg* cfg,
                                         fpic_push_stats* stats, void* stream)
{
    if (!m) return set_error(FPIC_EINVAL, "fpic_push_batched_learned: NULL network");
    return push_batched(runs, nruns, m, p, prm, cfg, stats, stream);
}

extern "C" int fpic_set_tuning(fpic_ctx* c, int key, int value)
{
    if (!c) return set_error(FPIC_EINVAL, "fpic_set_tuning: NULL ctx");
    switch (key) {
    case FPIC_TUNE_IMR_BLOCKS_PER_SM:
        if (value < 1 || value > 4)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: IMR blocks per SM must be in [1, 4], got %d", value);
        c->imr_blocks_per_sm = value;
        return FPIC_OK;
    case FPIC_TUNE_DEP_THREADS:
        if (value != 64 && value != 128 && value != 256)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: deposit threads must be 64, 128 or 256, got %d", value);
        c->dep_threads = value;
        return FPIC_OK;
    case FPIC_TUNE_STATIC_FIELDS:
        if (value != 0 && value != 1)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: static fields must be 0 or 1, got %d", value);
        c->static_fields = value;
        for (int i = 0; i < 6; ++i) c->fcoef_src[i] = nullptr;   // rebuilt at the next push
        c->slope_key_n = -1;                                      // cached slopes dropped
        return FPIC_OK;
    case FPIC_TUNE_REUSE_SLOPE:
        if (value != 0 && value != 1)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: slope reuse must be 0 or 1, got %d", value);
        c->reuse_slope = value;
        c->slope_key_n = -1;
        return FPIC_OK;
    case FPIC_TUNE_STAGE_FIELDS:
        if (value != 0 && value != 1)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: field staging must be 0 or 1, got %d", value);
        c->stage_fields = value;
        return FPIC_OK;
    case FPIC_TUNE_DEP_LATTICE:
        if (value != 0 && value != 1)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: deposit lattice must be 0 or 1, got %d", value);
        c->dep_lattice = value;
        return FPIC_OK;
    case FPIC_TUNE_ASYNC:
        if (value != 0 && value != 1)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: async must be 0 or 1, got %d", value);
        c->async = value;
        return FPIC_OK;
    case FPIC_TUNE_HOST_STAGING:
        if (value != 0 && value != 1)
            return set_error(FPIC_EINVAL, "fpic_set_tuning: host staging must be 0 or 1, got %d", value);
        c->host_staging = value;
        return FPIC_OK;
    default:
        return set_error(FPIC_EINVAL, "fpic_set_tuning: unknown key %d", key);
    }
}

extern "C" int fpic_get_tuning(const fpic_ctx* c, int key, int* value)
{
    if (!c || !value) return set_error(FPIC_EINVAL, "fpic_get_tuning: NULL argument");
    switch (key) {
    case FPIC_TUNE_IMR_BLOCKS_PER_SM:
        *value = c->imr_blocks_per_sm;
        return FPIC_OK;
    case FPIC_TUNE_DEP_THREADS:
        *value = c->dep_threads;
        return FPIC_OK;
    case FPIC_TUNE_STATIC_FIELDS:
        *value = c->static_fields;
        return FPIC_OK;
    case FPIC_TUNE_REUSE_SLOPE:
        *value = c->reuse_slope;
        return FPIC_OK;
    case FPIC_TUNE_STAGE_FIELDS:
        *value = c->stage_fields;
        return FPIC_OK;
    case FPIC_TUNE_DEP_LATTICE:
        *value = c->dep_lattice;
        return FPIC_OK;
    case FPIC_TUNE_ASYNC:
        *value = c->async;
        return FPIC_OK;
    case FPIC_TUNE_HOST_STAGING:
        *value = c->host_staging;
        return FPIC_OK;
    default:
        return set_error(FPIC_EINVAL, "fpic_get_tuning: unknown key %d", key);
    }
}
