/*
 * fpic.h -- C ABI of the GB300 (sm_103a) GRPIC hot path.
 *
 * Method: "FPIC: a new Particle-In-Cell code for stationary and axisymmetric
 * black-hole spacetimes" (Meringolo & Rezzolla, arXiv 2602.07452).
 *
 * Conventions shared by every entry point
 *   - Geometrised units G = c = 1; black-hole mass M, spin a (a length).
 *   - Particle state (Sec. 2.2): contravariant position (r, th, ph) and
 *     covariant momentum per unit mass (u_r, u_th, u_ph), FP64, SoA.
 *   - Axisymmetric (r, th) Yee grid (Sec. 2.1, Fig. 1): Nr x Nth cells, node
 *     tables r_i (Nr+1), r_{i+1/2} (Nr), th_j (Nth+1), th_{j+1/2} (Nth).
 *     Component placement:
 *        D^r, J^r (i+1/2, j)   D^th, J^th (i, j+1/2)   D^ph, J^ph, rho (i, j)
 *        B^r      (i, j+1/2)   B^th       (i+1/2, j)   B^ph (i+1/2, j+1/2)
 *     Every grid array is FP64, row-major [i * ld + j] with ld = Nth + 1 and
 *     (Nr + 1) * ld elements (rows/columns a staggered component does not
 *     use are padding, left untouched).
 *   - Device pointers are owned by the caller (e.g. torch tensors); the
 *     library never frees them.  The library owns the context, its node
 *     tables, metric tables and scratch buffers.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) unless its comment says it synchronises.
 *   - Return value: FPIC_OK (0), or a negative error code; the message of the
 *     last error on the calling thread is returned by fpic_last_error().
 *     Arguments are validated on the host before anything is launched; the
 *     kernels never trap.
 */
#ifndef FPIC_H
#define FPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPIC_OK 0
#define FPIC_EINVAL (-1)        /* bad argument (message says which) */
#define FPIC_ECUDA (-2)         /* a CUDA call failed */
#define FPIC_ENOMEM (-3)        /* device allocation of library scratch failed */
#define FPIC_ETIMEOUT (-4)      /* a bounded device wait ran out */
#define FPIC_ENOTCONVERGED 1    /* non-fatal: some implicit solves hit max_iter */

/* Pushers: Sec. 2.2.1 (RK4), Sec. 2.2.2 (IMR), Sec. 2.2.3 (Hamiltonian,
 * geodesics only) and the hybrid of Sec. 3.1.2 (Hyb1 / Hyb2). */
enum { FPIC_RK4 = 0, FPIC_IMR = 1, FPIC_HAM = 2, FPIC_HYB1 = 3, FPIC_HYB2 = 4 };

/* Particle initialisation kinds for fpic_init_particles. */
enum { FPIC_SEED_ORBIT = 0, FPIC_SEED_FIDO = 1 };

typedef struct fpic_ctx fpic_ctx;

/* Particle set, SoA, all device pointers of length n (caller-owned).
 *   r, th, ph, ur, uth, uph : state, updated in place by fpic_push
 *   qm     : charge-to-mass ratio q/m (0 = neutral)
 *   w      : macro-particle weight (Sec. 2.3)
 *   H0, D0 : initial energy H(x0,u0) and its error normaliser
 *            D0 = |alpha Gamma - beta u_r|_0 + |(q/m) A_0|_0
 *   Hn     : H after the last step (read by Hyb1, written by every push)
 *   alive  : 1 = in the domain, 0 = removed (Sec. 2.5)
 *   scheme : written by fpic_push: 0 = explicit step kept, 1 = implicit
 *   iters  : written by fpic_push: implicit iteration count (saturates at 255)
 *   cell   : written by fpic_cell_index / fpic_push: ir * Nth + ith           */
typedef struct {
    int64_t n;
    double *r, *th, *ph, *ur, *uth, *uph;
    double *qm, *w;
    double *H0, *D0, *Hn;
    uint8_t *alive, *scheme, *iters;
    uint32_t *cell;
} fpic_particles;

/* Parameters of one push.
 *   dt        : time step (finite, nonzero)
 *   scheme    : FPIC_RK4 .. FPIC_HYB2
 *   implicit  : FPIC_IMR or FPIC_HAM, the implicit partner of the hybrid
 *   thr       : Hyb2: Htilde_max; Hyb1: (d Htilde / dt)_max   (Sec. 3.1.2)
 *   tol       : implicit stop: max_i |dz_i| / (|z_i| + 1) <= tol
 *   max_iter  : implicit iteration cap (1..255); an IMR solve that reaches
 *               it returns the iterate whose update max_i |dz_i| was the
 *               smallest (the earliest on ties) and counts in n_notconv
 *   r_max     : outer removal radius; the inner one is the horizon r_+
 *   dg_eps    : increment below which the discrete gradient takes the
 *               analytic partial (App. D uses 1e-10)
 *   B0pot     : B0 of the Wald potential A_0 entering H (0 = none)
 *   guess     : nullable device array (n x 8, FP32) of learned implicit
 *               guesses and scheme logits (see fpic_mlp_infer); NULL = plain
 *   events    : nullable array of 4 cudaEvent_t recorded on the stream
 *               around the explicit kernel ([0], [1]) and the implicit
 *               kernel ([2], [3]) for per-kernel timing; NULL = none
 *   dt_implicit: step of the hybrid's implicit partner (adaptive steps,
 *               Sec. 3.1.2 and Tab. C.2: Delta t_Ham != Delta t_RK4); a
 *               rejected particle is advanced from z^n by dt_implicit, its
 *               solve starting from z^n + (z_RK4 - z^n) dt_implicit / dt.
 *               0 = dt.  Same sign as dt.  Pure schemes ignore it; the
 *               learned guess needs 0 or dt.
 *   t         : nullable device array (n doubles): each alive particle's
 *               time, advanced by the step it took (dt or dt_implicit)
 *   B0field   : with fields == NULL, the analytic Wald field of this B0
 *               (App. B.1, M = 1) supplies the Lorentz force instead of a
 *               grid, and the discrete-gradient scheme (FPIC_HAM, alone or as
 *               the hybrid's partner) also takes charged particles: it runs
 *               in canonical momenta pi_i = u_i + (q/m) A_i with the
 *               potentials of Eq. (Amu) and conserves H (with B0pot =
 *               B0field) and L exactly (an extension, not in the paper).
 *               0 = none.  Not with fields, the batched or the learned push.
 *   imr_newton: iteration of the IMR solve (Sec. 2.2.2).  0: the fixed-point
 *               update of Eq. (imr2), z^[k] = z^n + dt F((z^n + z^[k-1])/2).
 *               1: the Newton iteration the section names, with the Newton
 *               matrix 1 - (dt/2) dF reduced to the momentum columns of dF
 *               (d(dx/dt)/du and the magnetic force's d(du/dt)/du, both in
 *               closed form); same fixed point.  It also stops, from its
 *               second iteration on, when every component's a-posteriori
 *               error bound theta_i / (1 - theta_i) |dz_i| (theta_i the
 *               ratio of its last two updates) is within tol (|z_i| + 1):
 *               about a third of the iterations of the fixed-point update
 *               for charged particles.  Any nonzero = 1.
 *   imr_substeps: K > 0: an IMR solve that reaches max_iter without
 *               converging (found within a few 1e-4 rad of the polar axis,
 *               where the step under-resolves the turn) is redone from z^n
 *               as m = 2, 4, ..., 2^K substeps of the implicit step / m,
 *               each an IMR solve of the same form from its own start
 *               state, the pole reflection applied after each; the first
 *               level whose solves all converge and whose end point has
 *               |H - H(z^n)| / D_0 <= substep_tol (0: no H condition) is
 *               kept, else the finest level whose solves all converged,
 *               else the smallest-update iterate of the full step (counted
 *               in n_notconv).  Iterations of every attempt count in
 *               n_iter_total.  0 = off (0..12).
 *   substep_tol: see imr_substeps.
 *   before    : nullable; the state of every particle at the start of the
 *               step -- r, th, ur, uth, uph and alive (n entries) -- is
 *               written into these arrays of *before (device, before->n >=
 *               n; its other arrays are not touched) by the explicit pass as
 *               it reads the state: what fpic_deposit_conserving needs as
 *               its `before`, without a separate copy.  fpic_push with RK4 or
 *               a hybrid scheme only (FPIC_EINVAL elsewhere). */
typedef struct {
    double dt;
    int scheme;
    int implicit;
    double thr;
    double tol;
    int max_iter;
    double r_max;
    double dg_eps;
    double B0pot;
    const float *guess;
    void *const *events;
    double dt_implicit;
    double *t;
    double B0field;
    int imr_newton;
    int imr_substeps;
    double substep_tol;
    fpic_particles *before;
} fpic_push_params;

/* Host-side counters of one push (filled only when a pointer is passed;
 * that makes fpic_push synchronise the stream). */
typedef struct {
    int64_t n_alive_before;
    int64_t n_implicit;       /* particles that took the implicit scheme */
    int64_t n_iter_total;     /* sum of implicit iterations */
    int64_t n_notconv;        /* implicit solves stopped by max_iter */
    int64_t n_removed;        /* particles removed by the boundaries */
    int64_t n_rhs_evals;      /* right-hand-side evaluations performed */
    int64_t n_slope_reused;   /* particles whose first RK4 stage came from the
                                 slope cache (FPIC_TUNE_REUSE_SLOPE) */
    int64_t n_tiles_staged;   /* blocks of the explicit pass that staged their
                                 field tile (FPIC_TUNE_STAGE_FIELDS) */
} fpic_push_stats;

/* Create a context for the Kerr spacetime of mass M > 0 and spin |a| <= M
 * (Appendix A).  *ctx receives a library-owned handle; release it with
 * fpic_destroy.  Binds to the current CUDA device.
 * Errors: FPIC_EINVAL (M <= 0, |a| > M, ctx NULL), FPIC_ENOMEM. */
int fpic_init_metric(fpic_ctx **ctx, double M, double a);

/* Release the context and every buffer the library allocated for it. */
void fpic_destroy(fpic_ctx *ctx);

/* Message of the last error on the calling thread ("" if none). */
const char *fpic_last_error(void);

/* Set the (r, th) grid (Sec. 2.1; half-th domain, Sec. 2.5).  rn (Nr+1),
 * rh (Nr), tn (Nth+1), th (Nth) are HOST arrays of strictly increasing node
 * coordinates with rn[0] > 0, copied into the context; cell location against
 * them is exact (FP64 comparisons only).  Also builds the metric tables at
 * every Yee point (Sec. 2.1: "computed only initially and stored").
 * Synchronises the device.  Errors: FPIC_EINVAL (sizes < 2, non-monotone or
 * non-positive nodes), FPIC_ENOMEM, FPIC_ECUDA. */
int fpic_set_grid(fpic_ctx *ctx, int Nr, int Nth, const double *rn, const double *rh,
                  const double *tn, const double *th);

/* Geometry of the th direction (Sec. 2.5).  FPIC_THETA_HALF (the default
 * after fpic_set_grid): th between the poles, particles reflected at them.
 * FPIC_THETA_FULL: th covers one period, tn[Nth] - tn[0] = 2 pi (e.g.
 * tn[j] = eps + j dth, dth = 2 pi / Nth, eps = pi / (2 Nth), so both poles
 * lie midway between a node and a half node); th in (pi, 2 pi) is the other
 * half of the meridional plane, described by the same closed forms with
 * sin th < 0.  Particles cross the poles and wrap around periodically (no
 * reflection); gathers wrap too: column Nth of every field array must hold
 * the image of column 0 (fpic_init_wald writes it), and the half-node
 * sub-grid's wrap cell runs from th[Nth-1] to th[0] + 2 pi.  Supported in
 * the full-theta domain: the pushes (fpic_push, fpic_push_host,
 * fpic_push_batched, the corrector form of the learned push),
 * fpic_cell_index, fpic_sort, fpic_init_wald, fpic_hamiltonian,
 * fpic_init_particles, and fpic_fdtd_step with periodic field boundaries
 * (the th differences at the seam wrap around, no axis rows; it keeps
 * column Nth of what it writes equal to column 0, as the paper's vacuum
 * Wald run in the full domain needs); the other grid-side solvers
 * (deposits, cleaning, injection, BZ power, split-monopole initial field)
 * and the skip form's features return FPIC_EINVAL.  Setting the mode drops cached slopes and
 * coefficients.  Errors: FPIC_EINVAL (no grid, unknown mode, a full-theta
 * grid whose period is not 2 pi to 1e-12). */
enum { FPIC_THETA_HALF = 0, FPIC_THETA_FULL = 1 };
int fpic_set_theta_mode(fpic_ctx *ctx, int mode);

/* Sample the Wald electro-vacuum field of strength B0 (Appendix B.1) at
 * every Yee point: fields[0..5] = D^r, D^th, D^ph, B^r, B^th, B^ph, device
 * arrays in the grid layout.  Requires fpic_set_grid and M = 1 (the
 * appendix's units).  Errors: FPIC_EINVAL. */
int fpic_init_wald(fpic_ctx *ctx, double *const fields[6], double B0, void *stream);

/* Sample the vacuum split-monopole field (Sec. 3.4, App. B.2): B^r =
 * d_th Psi / sqrt(gamma) at the B^r Yee points with the flux function
 * Psi = 4 M^2 B0 zeta(th) (1 - cos th) and the smoothed equatorial current
 * sheet zeta = (2/pi) arctan[zeta0 (th - pi/2)]; fields[0..5] = D^r, D^th,
 * D^ph, B^r, B^th, B^ph as for fpic_init_wald, every component but B^r set
 * to zero.  Requires fpic_set_grid.  Errors: FPIC_EINVAL (NULL, no grid,
 * B0 not finite, zeta0 <= 0). */
int fpic_init_split_monopole(fpic_ctx *ctx, double *const fields[6], double B0, double zeta0, void *stream);

/* Initialise particles from caller-supplied random draws (device arrays):
 *   FPIC_SEED_ORBIT: draws is n x K x 5 (r, th, E, L, root sign); the first
 *     candidate for which H(r, th, u_r, 0, L) = E has a root with
 *     E + beta u_r > 0 is used; u_th = 0, u_ph = L, ph = 0.
 *   FPIC_SEED_FIDO : draws is n x 6 (r, th, ph, uhat): FIDO-frame momentum
 *     mapped to u_i = L_ia uhat_a with gamma_ij = L L^T (Cholesky).
 * Then sets H0 = Hn = H and D0 (B0pot as in fpic_push_params), alive = 1.
 * qm and w must already be filled by the caller.  Particles without a valid
 * orbit candidate get alive = 0.  Errors: FPIC_EINVAL. */
int fpic_init_particles(fpic_ctx *ctx, fpic_particles *p, int kind, const double *draws,
                        int K, double B0pot, void *stream);

/* One step of every alive particle (Sec. 2.2 and Sec. 3.1.2): the fields
 * D^i, B^i (fields[0..5], Yee layout, NULL = no field) are gathered at the
 * particle by bilinear interpolation in (r, th) on each component's own
 * sub-grid and held fixed over the step.  Hybrid schemes take an RK4 trial
 * and redo rejected particles with the implicit scheme from z^n, starting
 * from the trial (or from the learned guess when prm->guess is set).
 * After the step: particle boundaries (Sec. 2.5), Hn, scheme, iters, cell.
 * FPIC_HAM (and a hybrid with implicit = FPIC_HAM) pushes geodesics: q/m and
 * fields are ignored by its implicit part.  Uses library scratch (grown on
 * demand).  Returns FPIC_ENOTCONVERGED (> 0) if stats was given and some
 * implicit solve hit max_iter.  Errors: FPIC_EINVAL, FPIC_ENOMEM, FPIC_ECUDA. */
int fpic_push(fpic_ctx *ctx, fpic_particles *p, const double *const fields[6],
              const fpic_push_params *prm, fpic_push_stats *stats, void *stream);

/* One run of a batched push: an independent spacetime (ctx: M, a and grid),
 * its fields (device, or all NULL), its particle range [begin, end) in the
 * batch's particle arrays, its outer removal radius and Wald potential B0. */
typedef struct {
    fpic_ctx *ctx;
    const double *fields[6];
    int64_t begin, end;
    double r_max, B0pot;
} fpic_run;

/* Batched hybrid push (no counterpart in the paper): one explicit launch and
 * one persistent implicit launch advance every run of the batch -- different
 * spins, grids, fields and particle counts -- by one step, each particle
 * with its own run's spacetime and fields, exactly as fpic_push would.
 * runs[0..nruns) must tile [0, p->n) in order (runs[0].begin = 0,
 * runs[i].begin = runs[i-1].end, runs[nruns-1].end = p->n); all contexts on
 * the current device; prm is shared (its r_max and B0pot are ignored in
 * favour of each run's).  The run table is staged through pinned memory
 * owned by runs[0].ctx, so after one call outside capture the call can be
 * captured in a CUDA graph and replayed.  A captured graph holds the
 * addresses of the context's scratch; a later call that needs more scratch
 * (more particles, or the learned push) allocates a larger buffer and keeps
 * the superseded one until fpic_destroy, so graphs captured earlier stay
 * valid for the context's lifetime (the same holds for every library-owned
 * buffer that grows: coefficients, run table, node and metric tables).
 * Errors: FPIC_EINVAL,
 * FPIC_ENOMEM, FPIC_ECUDA; FPIC_ENOTCONVERGED as fpic_push. */
int fpic_push_batched(const fpic_run *runs, int nruns, fpic_particles *p, const fpic_push_params *prm,
                      fpic_push_stats *stats, void *stream);

/* fpic_push on a particle set held in HOST memory.  When every array of
 * *host_p is page-locked, mapped host memory (cudaHostAlloc, cudaHostRegister,
 * torch pin_memory), the kernels read and write it in place over the
 * CPU-GPU link (NVLink-C2C on Grace): no staging copies, each byte crosses
 * once per direction.  Otherwise the input arrays (state, q/m, H_0, D_0,
 * H^n, alive; w is not read by the push and not copied) go to library-owned
 * device buffers in four particle chunks on a library-owned copy stream, the
 * explicit pass of each chunk starting as soon as its copies land (the
 * implicit pass then runs over all queued particles), and the state, Hn,
 * alive, scheme, iters and cell arrays are copied back on `stream`.  Either
 * way the push is exactly fpic_push's and `stream` is synchronised before
 * returning -- except on mapped arrays with FPIC_TUNE_ASYNC = 1, where the
 * call only enqueues the push and the host arrays hold its results once
 * `stream` has been synchronised.  fields stay device arrays.  Errors: as
 * fpic_push. */
int fpic_push_host(fpic_ctx *ctx, fpic_particles *host_p, const double *const fields[6],
                   const fpic_push_params *prm, fpic_push_stats *stats, void *stream);

/* Fixed capacity of fpic_push_noalloc's scratch, in particles. */
#define FPIC_NOALLOC_MAX_PARTICLES 65536

/* Allocation-free variant of fpic_push for pushes without grid fields.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code whose device memory belongs to a
 * host framework or custom allocator that forbids direct cudaMalloc,
 * real-time loops where an allocation (or the synchronisation of a
 * cudaFree) is not allowed, plugin builds without an allocator.  It needs
 * no context (M, a given directly), calls no cudaMalloc, cudaFree or other
 * allocating routine, and keeps its scratch (implicit guesses, queue of
 * rejected particles, counters) in one file-scope device array of fixed
 * size, FPIC_NOALLOC_MAX_PARTICLES * 72 + 256 = 4718848 bytes, that every
 * device which loads the library holds until the process exits.
 *   p, prm, stats, stream : as fpic_push without fields (prm->guess must be
 *     NULL).  Neutral particles move on geodesics of the Kerr metric
 *     (M, a); with prm->B0field != 0 (M = 1) charged particles feel the
 *     analytic Wald field as in fpic_push (the discrete-gradient partner
 *     then works in canonical momenta).
 *   Errors: FPIC_EINVAL if p->n > FPIC_NOALLOC_MAX_PARTICLES (nothing is
 *     launched) or for the argument errors of fpic_push; FPIC_ECUDA.
 * The first call on each device (and the first under a new CUDA context,
 * e.g. after cudaDeviceReset) looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The look-up is guarded by a mutex, so
 * host threads may make their first calls concurrently.  Every call on a
 * device shares the one array and the counters are cleared at the start of
 * each call, so calls whose work overlaps on the GPU (other streams, other
 * threads) race: serialise them on one stream.  Results equal fpic_push's. */
int fpic_push_noalloc(double M, double a, fpic_particles *p, const fpic_push_params *prm,
                      fpic_push_stats *stats, void *stream);

/* Measurement helper (not part of the method): sustained FP64 fused
 * multiply-add rate of the current device, in GFLOP/s (2 flops per FMA),
 * from a kernel of independent FMA chains on every SM, timed with CUDA
 * events.  Synchronises the device.  Errors: FPIC_EINVAL (out NULL),
 * FPIC_ECUDA. */
int fpic_probe_fp64(double *gflops_out, int reps);

/* Launch-shape tuning of a context (read by every later push on it).
 *   FPIC_TUNE_IMR_BLOCKS_PER_SM: resident blocks of 128 threads per SM of
 *     the persistent implicit solver, 1..4 (default 4, the register-limited
 *     maximum).  Fewer lanes process more queued particles each, which
 *     evens out the uneven iteration counts at the end of the queue; more
 *     lanes hide more memory latency.  The autotuner in the Python package
 *     (autotune.py) times the candidates on the caller's own particles.
 *   FPIC_TUNE_DEP_THREADS: threads per block of the deposit's per-particle
 *     kernel (the trapezoid lattices), 64, 128 or 256 (default 128); the
 *     deposit's result does not depend on it.
 *   FPIC_TUNE_STATIC_FIELDS: 1 = the caller does not change the contents of
 *     the field arrays it passes (test particles in a fixed field), so the
 *     per-cell interpolation coefficients each push builds are reused while
 *     the six field pointers stay the same; 0 (default) = rebuilt every push.
 *     Setting it discards the current coefficients.
 *   FPIC_TUNE_REUSE_SLOPE: 1 = fpic_push, fpic_push_host and the corrector
 *     form of fpic_push_learned keep, per particle, the right-hand side
 *     F(z^{n+1}) and sin/cos th^{n+1} at the end of its step (the RK4 trial
 *     evaluates the full right-hand side at its end point instead of H
 *     alone; the IMR solves at their converged point) in a library-owned
 *     array of 15 doubles per particle, and the next push takes its first
 *     RK4 stage k1 = F(z^n) from there for every particle whose state and
 *     q/m are bitwise those the library stored.  The cache applies only
 *     while the right-hand side cannot have changed: no grid fields, or
 *     FPIC_TUNE_STATIC_FIELDS = 1; it is dropped when the particle arrays,
 *     n, the six field pointers, B0field or the grid change.  Results equal
 *     those without it up to rounding (sin/cos of th^{n+1} by angle
 *     addition instead of libm, H of the trial through 1/sqrt instead of
 *     sqrt).  0 (default) = every push evaluates k1.
 *   FPIC_TUNE_STAGE_FIELDS: 1 = the explicit pass of fpic_push with grid
 *     fields stages, per block of 128 particles, the interpolation
 *     coefficients of the cells the block's particles occupy (from p->cell,
 *     as the last push or fpic_sort left it; the block's cells plus two
 *     cells of margin, up to 5 x 16 coefficient cells per component) in
 *     shared memory with TMA tensor loads; gathers outside the tile read
 *     global memory, so results are bitwise those without staging.  Pays
 *     only for particles sorted by cell (the PIC step sorts them in its
 *     deposit).  A tile load whose bounded wait runs out is counted and
 *     reported as FPIC_ETIMEOUT when stats are requested.  0 (default) =
 *     no staging.
 *   FPIC_TUNE_DEP_LATTICE: arithmetic of fpic_deposit's trapezoid lattices
 *     of sqrt(gamma) (Sec. 2.3).  1 (default) = paired FP32 (each value the
 *     sum of two floats, about 48 bits; the square root to about 2^-44
 *     relative), run on the FP32 pipe; 0 = FP64 with the square root from
 *     the hardware estimate and one Goldschmidt step (2^-39.6 measured).
 *     Lattice points, weights and node shares are the same; results differ
 *     by rounding only (1e-13 relative and below on the deposited sources).
 *   FPIC_TUNE_ASYNC: 1 = fpic_push and fpic_push_host never synchronise the
 *     stream: requested stats are assembled on the device and copied into
 *     *stats asynchronously (valid once `stream` has been synchronised; pass
 *     page-locked host memory, else the copy itself blocks; FPIC_ETIMEOUT
 *     and FPIC_ENOTCONVERGED are then not returned, read n_notconv), and
 *     fpic_push_host on mapped host arrays returns before its results are
 *     written (see there).  0 (default) = stats are read, and the host push
 *     completed, before the call returns.
 *   FPIC_TUNE_HOST_STAGING: 1 = fpic_push_host moves even mapped (pinned)
 *     arrays through library-owned device buffers -- DMA copies in four
 *     chunks overlapping the explicit pass, the push on the device, DMA
 *     copies back -- instead of reading and writing them in place over the
 *     link; the results are the same.  In place, the implicit pass's
 *     write-back goes to scattered host addresses, one link transaction per
 *     value; staged, every transfer is a sequential DMA.  0 (default) = in
 *     place for mapped arrays.
 * Errors: FPIC_EINVAL (NULL, unknown key, value out of range). */
enum { FPIC_TUNE_IMR_BLOCKS_PER_SM = 0, FPIC_TUNE_DEP_THREADS = 1, FPIC_TUNE_STATIC_FIELDS = 2,
       FPIC_TUNE_REUSE_SLOPE = 3, FPIC_TUNE_STAGE_FIELDS = 4, FPIC_TUNE_DEP_LATTICE = 5, FPIC_TUNE_ASYNC = 6,
       FPIC_TUNE_HOST_STAGING = 7 };
int fpic_set_tuning(fpic_ctx *ctx, int key, int value);
int fpic_get_tuning(const fpic_ctx *ctx, int key, int *value);

/* Test helper for the library's own FP64 elementary routines, one thread
 * per element of x (device, n values) into y (device):
 *   fn 0: 1/x by the hardware estimate and one third-order refinement
 *         (push metric);
 *   fn 1: sqrt(x) by the hardware reciprocal-square-root estimate and one
 *         Goldschmidt step (deposit trapezoid sums), x > 0 normal;
 *   fn 2: y[2i] = sin x, y[2i+1] = cos x - 1 for a small step x (series
 *         below 2^-7, libm above), as used by the angle-addition updates;
 *   fn 3: y = sqrt(x) in the deposit's paired-FP32 form (x split into two
 *         floats, the result's two floats summed in FP64);
 *   fn 4: as fn 2, in the deposit's paired-FP32 form;
 *   fn 5: 1/sqrt(x) by the hardware estimate and the second-order binomial
 *         correction (push metric lapse and 1/Gamma), x > 0 normal;
 *   fn 6: 1/x in the deposit's paired-FP32 form, x > 0 in the normal float
 *         range;
 *   fn 7: pairs (a, b) = (x[2i], x[2i+1]), i < n/2, of non-negative
 *         doubles or NaNs: y[6i..6i+5] = the integer-compare forms of
 *         a <= b, then the FP64 a <= b, of a < b, then FP64 a < b (1 or 0),
 *         of fmax(a, b) with a running maximum a, then FP64 fmax (the push's
 *         IMR stopping tests); n even.
 * Errors: FPIC_EINVAL (fn out of range, n < 0, NULL with n > 0). */
int fpic_probe_math(int fn, const double *x, double *y, long long n, void *stream);

/* H (Eq. Ham with the Wald A_0 of Sec. 3.1.3 when B0pot != 0) and
 * L = u_ph + (q/m) A_ph for every particle.  H_out, L_out: device arrays of
 * length n, either may be NULL.  Errors: FPIC_EINVAL. */
int fpic_hamiltonian(fpic_ctx *ctx, const fpic_particles *p, double B0pot, double *H_out,
                     double *L_out, void *stream);

/* Cell index ir * Nth + ith of every particle (r_i <= r < r_{i+1}, clamped to
 * the grid), written to p->cell.  Exact: FP64 comparisons against the node
 * tables.  Errors: FPIC_EINVAL. */
int fpic_cell_index(fpic_ctx *ctx, fpic_particles *p, void *stream);

/* Field storage of the FDTD leapfrog (Sec. 2.1), all device arrays in the
 * grid layout, caller-owned:
 *   B0, B1 : B^n and B^{n+1} (3 components each: r, th, ph)
 *   D0, D1 : D^{n+1/2} and D^{n+3/2}
 *   j0, rho0 / j1, rho1 : FIDO current j^i and charge density at n+1 / n+2
 *                          (the deposit of the previous / current step)
 *   E, H, Bh, Dw : work arrays; after stage 1 Bh holds B^{n+3/2} (the field
 *                  the push uses with D1), after stage 2 Dw holds D^{n+2}. */
typedef struct {
    double *B0[3], *B1[3], *D0[3], *D1[3];
    double *j0[3], *rho0, *j1[3], *rho1;
    double *E[3], *H[3], *Bh[3], *Dw[3];
} fpic_fields;

/* FDTD parameters: time step dt and the absorbing layer of Eqs. (abs0)-(abs2):
 * chi(r) = chi0 ((r - r_abs)/(r_max - r_abs))^lambda for r > r_abs (chi0 = 0
 * switches it off); the damping is applied as a factor exp(-chi dt).
 * conserving = 1: the j arrays hold coordinate currents J = alpha j - rho beta
 * (fpic_deposit_conserving), used as they are in sub-steps 8 and 10;
 * 0: FIDO currents j, turned into J with rho (Sec. 2.1). */
typedef struct {
    double dt, chi0, lambda, r_abs, r_max;
    int conserving;
} fpic_fdtd_params;

/* Stable sort of the particles by cell index ir * Nth + ith (removed
 * particles last), permuting every array of *p in place (Sec. 2.3 needs the
 * particles of a cell together; the order inside a cell is the previous
 * order).  Also writes p->cell.  Uses library scratch.
 * Errors: FPIC_EINVAL (no grid, NULL arrays), FPIC_ENOMEM, FPIC_ECUDA. */
int fpic_sort(fpic_ctx *ctx, fpic_particles *p, void *stream);

/* Charge and current deposition (Sec. 2.3): each alive particle of charge
 * Q = w (q/m) and FIDO velocity v^i = gamma^ij u_j / Gamma is shared between
 * the four nodes of its cell on each Yee sub-grid in proportion to the
 * opposite subvolume (4 x 4-point trapezoid of sqrt(gamma) on each
 * sub-rectangle), summed per node in a fixed order (deterministic, no
 * floating-point atomics) and divided by 2 pi times the node's dual-cell
 * volume.  Outputs (device, grid layout, overwritten): rho and j^ph at
 * (i, j), j^r at (i+1/2, j), j^th at (i, j+1/2).  Sorts the particles first
 * (fpic_sort).  Errors: FPIC_EINVAL, FPIC_ENOMEM, FPIC_ECUDA. */
int fpic_deposit(fpic_ctx *ctx, fpic_particles *p, double *rho, double *jr, double *jth, double *jph,
                 void *stream);

/* One half of the FDTD leapfrog step of Sec. 2.1 (Eqs. m3, m4, Ei, and the
 * absorbing layer and boundaries of Sec. 2.5):
 *   stage 1 (sub-steps 1-4): E^{n+1} -> B^{n+3/2} (into Bh) -> E^{n+3/2} ->
 *            B^{n+2} (into B0);
 *   stage 2 (sub-steps 7-10, after the push and the deposit of j1, rho1):
 *            H^{n+3/2} -> D^{n+2} (into Dw, with <J>^{n+3/2}) -> H^{n+2} ->
 *            D^{n+5/2} (into D0, with J^{n+2}),
 * with J = alpha j - rho beta.  After stage 2 the caller swaps B0/B1, D0/D1
 * and (j0, rho0)/(j1, rho1).  Boundaries: in the half-theta domain zero
 * gradient where a stencil is one-sided and D^ph = 0 on the axis rows; in
 * the full-theta domain (fpic_set_theta_mode) periodic in th, with column Nth
 * of every array it writes set to column 0 (the caller's input arrays must
 * hold that image too).  Errors: FPIC_EINVAL (no grid, stage not 1 or 2,
 * NULL array, dt not finite). */
int fpic_fdtd_step(fpic_ctx *ctx, fpic_fields *f, const fpic_fdtd_params *prm, int stage, void *stream);

/* Charge-conserving deposit of one step's moves (an extension: the paper's
 * deposit is not charge-conserving and relies on the cleaning of Sec. 2.4).
 * Each particle alive in *before moves from its state in *before to its
 * state in *after (same n, same order; only r, th, u and alive of *before are
 * read, r, th, u, qm, w of *after).  Node weights are linear (area) weights
 * in r and th; the move is split Esirkepov's way, W_r = dS_r <S_th>,
 * W_th = <S_r> dS_th, over the 3 x 3 nodes of both stencils, and the charge
 * crossing each dual face gives the coordinate currents.  Outputs (device,
 * grid layout):
 *   rho (i, j)      = Q S(x^{n+1}) / (2 pi sqrtg dr_dual dth_dual)
 *   jr  (i+1/2, j)  = J^r,  jth (i, j+1/2) = J^th: charge crossing per unit time
 *                     / (2 pi sqrtg x the dual face's width)
 *   jph (i, j)      = Q <S> (dph/dt) / (2 pi sqrtg dr_dual dth_dual)
 * so that sqrtg (rho^{n+1} - rho^n) + dt Yee-div(sqrtg J) = 0 at every node;
 * with fpic_fdtd_params.conserving = 1 the field update then keeps
 * Yee-div(sqrtg D) - 4 pi sqrtg rho constant.  Moves longer than one cell
 * are skipped and counted in *n_skipped (nullable; reading it synchronises
 * the stream).  Deterministic (per-cell warp sums in particle-index order).
 * Errors: FPIC_EINVAL, FPIC_ENOMEM, FPIC_ECUDA. */
int fpic_deposit_conserving(fpic_ctx *ctx, const fpic_particles *before, const fpic_particles *after, double dt,
                            double *rho, double *jr, double *jth, double *jph, long long *n_skipped,
                            void *stream);

/* Pair injection parameters (Sec. 3.3, 3.4). */
typedef struct {
    double r_lo, r_hi;     /* cells whose centre radius rh[i] lies in [r_lo, r_hi] */
    double multiplicity;   /* inject where n < multiplicity x n_GJ (the paper: 3, 10) */
    double n0;             /* density of one injected pair in units of n_GJ (the paper: 5) */
    double qm_e;           /* |q/m| of the pair particles (> 0): e- gets -qm_e, e+ +qm_e */
    double B0pot;          /* Wald potential strength for H0 / D0 of the new particles
                              (as in fpic_push_params; 0 on a PIC grid) */
} fpic_inject_params;

/* Pair injection (Sec. 3.3, 3.4): every cell whose centre radius lies in
 * [r_lo, r_hi] receives one e-/e+ pair when its plasma density is below
 * multiplicity x n_GJ, with e n = sum of w |q/m| over the cell's alive
 * particles / the cell's proper volume V (2 pi x the 4 x 4 trapezoid of
 * sqrt(gamma), Sec. 2.3) and e n_GJ = |Omega_h B^z| / 4 pi, Omega_h =
 * a / (2 M r_h), B^z = B^r cos th - r sin th B^th at the cell centre (B^r
 * averaged over the cell's r faces, B^th over its th faces).  The pair is
 * placed at one point (r, th) = cell corner + (u_r, u_th) x cell size,
 * ph = 2 pi u_ph, each particle with weight n0 (e n_GJ) V / (2 qm_e) and its
 * FIDO-frame momentum mapped to u_i as in FPIC_SEED_FIDO; H0 = Hn, D0 set,
 * alive = 1, cell written when p->cell is set.  Pairs are appended at
 * p->n, p->n + 1, ... in cell order (c = i Nth + j), e- first, while they
 * fit in capacity (the arrays of p must hold capacity entries).
 *   Br, Bth : B^r, B^th (device, Yee layout) — the magnetic field of the step
 *   draws   : device, 9 per cell c (u_r, u_th, u_ph in [0,1), e- FIDO
 *             momentum, e+ FIDO momentum): the caller's random numbers
 *   flags   : nullable device array of Nr Nth bytes, receives the decisions
 *   wanted  : nullable host out, pairs wanted (including those that did not fit)
 *   n_new   : host out, the new particle count (p->n itself is not changed)
 * The injection is called every Delta t_inj by the caller (the paper:
 * 0.01 M).  Synchronises the stream (the count is returned on the host).
 * Errors: FPIC_EINVAL (NULL, no grid, capacity < n, bad parameters, more
 * than 2^32 particles), FPIC_ECUDA. */
int fpic_inject_pairs(fpic_ctx *ctx, fpic_particles *p, long long capacity, const double *Br, const double *Bth,
                      const fpic_inject_params *prm, const double *draws, unsigned char *flags,
                      long long *wanted, long long *n_new, void *stream);

/* Divergence cleaning (Sec. 2.4, Eq. phi): solve
 *   (1/sqrtg) d_k (sqrtg gamma^kl d_l phi) = (1/sqrtg) d_j (sqrtg D^j) - 4 pi rho
 * at the integer nodes (i = 1 .. Nr-1, all j) by n_iter Jacobi sweeps from
 * phi = 0, then D^i -= gamma^ij d_j phi in place.  D[0..2] = D^r, D^th,
 * D^ph (device, grid layout), rho at the nodes.  The discrete operator uses
 * the Yee divergence's own sqrtg-weighted fluxes, so a converged solve
 * leaves the discrete Gauss law satisfied to rounding at every interior
 * node; phi = 0 on the radial end rows, no flux through the poles.  phi:
 * nullable device array (grid layout) receiving the potential.  Uses the
 * context's second scratch (7 grid arrays).  The paper cleans every 25 steps
 * with 500 sweeps.  Errors: FPIC_EINVAL, FPIC_ENOMEM. */
int fpic_div_clean(fpic_ctx *ctx, double *const D[3], const double *rho, int n_iter, double *phi, void *stream);

/* Blandford-Znajek power through the sphere r = rh[i] (half-r index i in
 * [0, Nr)), Eq. (Pbz): P = 2 pi int S^r sqrt(gamma) dth with S^r = (E_th H_ph
 * - E_ph H_th) / (4 pi sqrt(gamma)), i.e. (1/2) int (E_th H_ph - E_ph H_th)
 * dth, from the auxiliary fields f->E, f->H of the last fpic_fdtd_step
 * (sub-step 9 leaves H^{n+2}; sub-step 3 leaves E^{n+3/2}).  Each product is
 * formed at the cell centres (rh[i], th_{j+1/2}) from its staggered
 * neighbours averaged; midpoint rule over the th cells; fixed-order
 * reduction.  out: one device double.  Errors: FPIC_EINVAL. */
int fpic_bz_power(fpic_ctx *ctx, const fpic_fields *f, int i, double *out, void *stream);

/* ---- Learned implicit guess: MLP 14 -> 128 -> 128 -> 128 -> 9 --------------
 * No counterpart in the paper (its method has no learned component): a
 * network trained on the plain pusher's own steps predicts, per particle,
 * the implicit step and whether the hybrid test would reject the RK4 trial;
 * the push still accepts a step only by its own convergence and H tests.
 * BF16 operands, FP32 accumulation in tensor memory (tcgen05).
 * Parameter vector (FP32, device, fpic_mlp_nparams() entries):
 *   W1 [128][14] b1 [128] W2 [128][128] b2 [128] W3 [128][128] b3 [128]
 *   W4 [9][128] b4 [9]   (row-major [out][in], ReLU after layers 1-3). */
typedef struct fpic_mlp fpic_mlp;

/* Generic tensor-core GEMM C (+)= A B^T: A [M][lda] and B [N][ldb] bf16
 * row-major (K contiguous, 16-byte aligned), C [M][ldc] FP32; N a multiple
 * of 16 in [16, 256], K a multiple of 16.  accumulate != 0 adds into C.
 * *err (device int) is set to 1 if a bounded tensor-core wait ran out.
 * Errors: FPIC_EINVAL. */
int fpic_mma_bf16(const uint16_t *A, int lda, const uint16_t *B, int ldb, float *C, int ldc, int M, int N, int K,
                  int accumulate, int *err, void *stream);

/* Create / destroy a network handle (library-owned bf16 weight buffers). */
int fpic_mlp_create(fpic_mlp **m);
void fpic_mlp_destroy(fpic_mlp *m);
long long fpic_mlp_nparams(void);

/* Load FP32 parameters P (device) into the handle's bf16 tensor-core layouts. */
int fpic_mlp_set_params(fpic_mlp *m, const float *P, void *stream);

/* Forward pass of B samples: X (device, B x 16 FP32: 14 standardised
 * features then two zeros) -> Y (device, B x 16 FP32: 9 outputs then
 * padding).  Errors: FPIC_EINVAL. */
int fpic_mlp_forward(fpic_mlp *m, const float *X, float *Y, long long B, void *stream);

/* Gradient of the training loss over a batch of B samples (B a power of two
 * in [256, 2^24]): X (B x 16 features), T (B x 16 targets: outputs 0-5, 7,
 * 8 regressed, 6 unused), S (B labels in {0, 1} for the scheme logit,
 * output 6), lossw (9 host floats: weight of each regression output).
 * Loss per sample = sum_k lossw_k (y_k - T_k)^2 + log(1 + e^{y_6}) - S y_6,
 * averaged over the batch.  grad (device, fpic_mlp_nparams() FP32, the
 * parameter layout); loss (host, nullable; synchronises when given).
 * All GEMMs (forward and backward) run on the tensor cores.
 * Errors: FPIC_EINVAL, FPIC_ENOMEM. */
int fpic_mlp_grad(fpic_mlp *m, const float *X, const float *T, const float *S, const float *lossw, long long B,
                  float *grad, float *loss, void *stream);

/* One training step: gradient as fpic_mlp_grad, then Adam (Kingma & Ba)
 * on the FP32 master parameters P with moments mom, vel (device, updated in
 * place; step = 1, 2, ... is the Adam time step), then the handle's bf16
 * weights are refreshed from P.  Errors: as fpic_mlp_grad. */
int fpic_mlp_train_step(fpic_mlp *m, float *P, float *mom, float *vel, const float *X, const float *T,
                        const float *S, const float *lossw, long long B, int step, float lr, float beta1,
                        float beta2, float eps, float *loss, void *stream);

/* Configuration of the learned guess in the push.  Two forms:
 *
 * FPIC_LEARN_SKIP (0), decided before the step: the 14 features are
 *     (ln r, th, u_r, u_th, u_ph, D^r, D^th, D^ph, B^r, B^th, B^ph gathered
 *     at the particle, the current energy error (H^n - H_0)/D_0, the
 *     fractional position of r in its cell, (q/m) dt), computed in FP32;
 *     outputs 0-5 are (z^{n+1} - z^n) / inc_scale; a particle whose
 *     predicted rejection probability sigmoid(y_6) exceeds p_skip skips the
 *     RK4 trial and starts the implicit solve from z^n + inc_scale y[0..5].
 *
 * FPIC_LEARN_CORRECT (1), decided after the trial: for each particle whose
 *     RK4 trial the plain test rejects, the features are the RK4 stage
 *     differences A = dt (k3 - k2) and B = dt (k4 - 2 k2 + k1) (k1..k4 the
 *     stage slopes of Sec. 2.2.1), each component i divided by its own scale
 *     s_i = |A_i| + |B_i| (features 0-5: A_i / s_i, 6-11: B_i / s_i), then
 *     ln r (12) and ln(sum |A_i| / sum |(z_RK4 - z^n)_i|) over the momenta
 *     u_r, u_th (13, a measure of the step's expansion parameter
 *     (omega dt)^2).  The
 *     gap between the converged implicit step and
 *     the trial is, to leading order in dt, dt^3 (f'f'f / 12 - f''(f,f) / 24)
 *     = g + O(dt^4) with g = (2/3) A - (1/6) B; outputs 0-5 are the rest of
 *     the gap, (z_IMR - z_RK4 - g)_i / (s_i inc_scale_i), and the implicit
 *     solve starts from z_RK4 + g + s inc_scale y[0..5] instead of z_RK4
 *     (a network with zero output gives the leading-order guess alone).
 *     The plain guess is the fallback: a component whose correction
 *     exceeds 5 % of the trial's own increment, or whose output is not
 *     finite, keeps the trial value; with restart_after > 0 a solve not
 *     converged after that many iterations from the corrected start
 *     restarts from the trial with the full max_iter budget (0: the solve
 *     runs to convergence or max_iter like the plain one).  p_skip is
 *     unused.
 *
 *   feat_mean, feat_std : standardisation (x - mean)/std of the 14 features;
 *   mode : FPIC_LEARN_SKIP or FPIC_LEARN_CORRECT;
 *   restart_after : see FPIC_LEARN_CORRECT (ignored by FPIC_LEARN_SKIP). */
enum { FPIC_LEARN_SKIP = 0, FPIC_LEARN_CORRECT = 1 };
typedef struct {
    float feat_mean[16], feat_std[16];
    double inc_scale[6];
    float p_skip;
    int mode;
    int restart_after;
} fpic_learned_cfg;

/* Network inputs of every particle: X (device, n x 16 FP32, standardised
 * with cfg; cfg NULL = raw features; removed particles get zeros).
 * Errors: FPIC_EINVAL. */
int fpic_features(fpic_ctx *ctx, const fpic_particles *p, const double *const fields[6], double dt,
                  const fpic_learned_cfg *cfg, float *X, void *stream);

/* Training samples from the plain method itself, leaving the particles
 * unchanged; every alive particle takes the RK4 trial, the plain test and
 * then the implicit solve from the trial.  Labels S (1 if the plain hybrid
 * test (prm) rejects the trial) and targets T (16 floats per sample: outputs
 * 0-5 as the form's outputs, output 7 = (iterations - 8)/4).
 *   cfg->mode FPIC_LEARN_SKIP: row p = particle p; X as fpic_features;
 *     targets (z_IMR - z^n) / inc_scale; removed particles get zero rows.
 *   cfg->mode FPIC_LEARN_CORRECT: row = the particle's slot in the implicit
 *     queue (rows 0 .. n_alive - 1, the order is not deterministic; X, T
 *     and S rows match); X = the trial features; targets
 *     (z_IMR - z_RK4 - g)_i / (s_i inc_scale_i) clamped to [-4, 4].
 * cfg NULL = FPIC_LEARN_SKIP with raw features.  prm->scheme must be
 * FPIC_HYB1 or FPIC_HYB2 with the IMR partner.
 * Errors: FPIC_EINVAL, FPIC_ENOMEM. */
int fpic_learn_sample(fpic_ctx *ctx, fpic_particles *p, const double *const fields[6], const fpic_push_params *prm,
                      const fpic_learned_cfg *cfg, float *X, float *T, float *S, void *stream);

/* Hybrid push with the learned guess (cfg->mode):
 *   FPIC_LEARN_SKIP: features -> network -> particles predicted to be
 *     rejected go straight to the IMR (started from the predicted step), the
 *     others take the RK4 trial and the plain test (rejected ones -> IMR from
 *     the trial);
 *   FPIC_LEARN_CORRECT: RK4 trial and plain test for every particle; the
 *     rejected ones' trial features -> network (tensor cores, rows = implicit
 *     queue, count read on the device) -> IMR from the corrected trial.
 * Every step is accepted only by the plain method's own tests: the H test for
 * RK4 steps, convergence for implicit ones (so in FPIC_LEARN_CORRECT the
 * scheme choices are exactly the plain ones).  prm as fpic_push (scheme
 * FPIC_HYB1/HYB2, implicit FPIC_IMR).  stats: as fpic_push; n_implicit
 * includes the skipped ones.  Errors: FPIC_EINVAL, FPIC_ENOMEM, FPIC_ECUDA. */
int fpic_push_learned(fpic_ctx *ctx, fpic_mlp *m, fpic_particles *p, const double *const fields[6],
                      const fpic_push_params *prm, const fpic_learned_cfg *cfg, fpic_push_stats *stats,
                      void *stream);

/* fpic_push_batched with the learned guess: the corrector form of
 * fpic_push_learned (cfg->mode = FPIC_LEARN_CORRECT, dt_implicit 0 or dt,
 * scheme FPIC_HYB1/HYB2) on every run of the batch in the same launches:
 * RK4 trial + plain test for all particles, the network on the rejected ones
 * of every run, the implicit solves from the corrected trials.  One network
 * serves all runs (its features are run independent).  runs, p, prm, stats
 * as fpic_push_batched; the scratch is runs[0].ctx's.  Scheme choices are
 * exactly fpic_push_batched's.  Errors: FPIC_EINVAL, FPIC_ENOMEM, FPIC_ECUDA,
 * FPIC_ENOTCONVERGED (stats only). */
int fpic_push_batched_learned(const fpic_run *runs, int nruns, fpic_mlp *m, fpic_particles *p,
                              const fpic_push_params *prm, const fpic_learned_cfg *cfg, fpic_push_stats *stats,
                              void *stream);

/* Reads the handle's error word (synchronous): FPIC_ETIMEOUT if a bounded
 * tensor-core wait of an earlier launch ran out, else FPIC_OK. */
int fpic_mlp_status(fpic_mlp *m, int *status);

#ifdef __cplusplus
}
#endif
#endif /* FPIC_H */
