// C ABI: context, grid, field and particle initialisation, diagnostics.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "fpic_internal.h"

namespace fpic {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int check_cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return 0;
    if (e == cudaErrorMemoryAllocation) return set_error(FPIC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(FPIC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void retire(fpic_ctx* c, void** p, bool host)
{
    if (*p) (host ? c->retired_host : c->retired_dev).push_back(*p);
    *p = nullptr;
}

// Scratch grows and never shrinks; the superseded buffer is retired, not
// freed, so a graph captured over it stays valid until fpic_destroy.
int ensure_scratch(fpic_ctx* c, size_t bytes)
{
    if (bytes <= c->scratch_bytes) return 0;
    retire(c, &c->d_scratch);
    c->scratch_bytes = 0;
    size_t b = bytes + bytes / 8;
    FPIC_CUDA(cudaMalloc(&c->d_scratch, b));
    c->scratch_bytes = b;
    return 0;
}

int ensure_scratch2(fpic_ctx* c, size_t bytes)
{
    if (bytes <= c->scratch2_bytes) return 0;
    retire(c, &c->d_scratch2);
    c->scratch2_bytes = 0;
    size_t b = bytes + bytes / 8;
    FPIC_CUDA(cudaMalloc(&c->d_scratch2, b));
    c->scratch2_bytes = b;
    return 0;
}

int ensure_copy_stream(fpic_ctx* c)
{
    if (c->copy_stream) return 0;
    FPIC_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : c->copy_ev) FPIC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return 0;
}

bool particles_ok(const fpic_particles* p, bool need_state)
{
    if (p->n == 0) return true;
    const void* ptrs[] = {p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn,
                          p->alive, p->scheme, p->iters};
    for (const void* q : ptrs)
        if (!q) return false;
    (void)need_state;
    return true;
}

// ---- Wald field (Appendix B.1), derived from the potential of Eq. (Amu) ----
// A_0 = B0 a M r (1 + c^2)/rho^2 (+ const), A_r = (B0/2)(-a s^2 + 2aMr(1+c^2)/rho^2),
// A_ph = (B0/2) s^2 [r^2 + a^2 - 2 M a^2 r (1 + c^2)/rho^2];
// B^i = eta^ijk d_j A_k / sqrt(gamma), E_i = d_i A_0.
__device__ void wald_point(const BH& bh, double B0, double r, double th, double D[3], double B[3])
{
    double s, c;
    sincos(th, &s, &c);
    wald_point_sc(bh, B0, r, s, c, D, B);
}

__global__ void k_wald(BH bh, GridDev G, double B0, double* F0, double* F1, double* F2, double* F3,
                       double* F4, double* F5)
{
    double* F[6] = {F0, F1, F2, F3, F4, F5};
    const int i = blockIdx.y;
    for (int j = threadIdx.x; j <= G.Nth; j += blockDim.x) {
#pragma unroll 1
        for (int k = 0; k < 6; ++k) {
            const bool ro = (k == 0 || k == 4 || k == 5);
            const bool to = (k == 1 || k == 3 || k == 5);
            if ((ro && i >= G.Nr) || (to && j >= G.Nth)) continue;
            const double r = ro ? G.rh[i] : G.rn[i];
            const double t = to ? G.th[j] : G.tn[j];
            double D[3], B[3];
            wald_point(bh, B0, r, t, D, B);
            F[k][i * G.ld + j] = k < 3 ? D[k] : B[k - 3];
        }
    }
}

// Split-monopole initial field (Sec. 3.4, App. B.2): B^r = d_th Psi / sqrt(gamma)
// at the B^r Yee points, Psi = 4 M^2 B0 zeta(th) (1 - cos th), zeta =
// (2/pi) arctan[zeta0 (th - pi/2)]; every other component zero.
__global__ void k_split_monopole(BH bh, GridDev G, double B0, double zeta0, double* F0, double* F1, double* F2,
                                 double* F3, double* F4, double* F5)
{
    double* F[6] = {F0, F1, F2, F3, F4, F5};
    const int i = blockIdx.y;
    for (int j = threadIdx.x; j <= G.Nth; j += blockDim.x) {
        const size_t o = (size_t)i * G.ld + j;
        for (int k = 0; k < 6; ++k)
            if (k != 3) F[k][o] = 0.0;
        if (j >= G.Nth) {
            F[3][o] = 0.0;
            continue;
        }
        const double t = G.th[j], x = t - 0.5 * M_PI;
        double s, c;
        sincos(t, &s, &c);
        const double zeta = (2.0 / M_PI) * atan(zeta0 * x);
        const double dzeta = (2.0 / M_PI) * zeta0 / fma(zeta0 * zeta0, x * x, 1.0);
        const double dpsi = 4.0 * bh.M * bh.M * B0 * fma(dzeta, 1.0 - c, zeta * s);
        Geo g;
        geo_eval(bh, G.rn[i], s, c, g);
        F[3][o] = dpsi / g.sqrtg;
    }
}

struct PInit {
    double *r, *th, *ph, *ur, *uth, *uph, *qm, *H0, *D0, *Hn;
    uint8_t *alive, *scheme, *iters;
};

__device__ void set_energy(const BH& bh, const PInit& P, long long p, const double z[6], double B0pot)
{
    double kin, pot;
    h_parts(bh, z, P.qm[p], B0pot, kin, pot);
    P.H0[p] = kin - pot;
    P.Hn[p] = kin - pot;
    P.D0[p] = fabs(kin) + fabs(pot);
}

__global__ void k_seed_orbit(BH bh, PInit P, long long n, const double* __restrict__ cand, int K, double B0pot)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    bool done = false;
    double z[6];
    for (int k = 0; k < K && !done; ++k) {
        const double* cc = cand + ((size_t)p * K + k) * 5;
        const double r = cc[0], th = cc[1], E = cc[2], L = cc[3], sg = cc[4];
        double s, c;
        sincos(th, &s, &c);
        Geo g;
        geo_eval(bh, r, s, c, g);
        const double al2 = g.alpha * g.alpha;
        const double A = al2 * g.gurr - g.beta * g.beta;
        const double Bq = al2 * g.gurp * L - E * g.beta;
        const double C = al2 * (1.0 + g.gupp * L * L) - E * E;
        const double disc = Bq * Bq - A * C;
        if (!(disc >= 0.0) || !(A > 0.0)) continue;
        const double ur = (-Bq + (sg >= 0.0 ? 1.0 : -1.0) * sqrt(disc)) / A;
        if (!(E + g.beta * ur > 0.0)) continue;
        z[0] = r; z[1] = th; z[2] = 0.0; z[3] = ur; z[4] = 0.0; z[5] = L;
        done = true;
    }
    if (!done) {
        for (int i = 0; i < 6; ++i) z[i] = nan("");
    }
    P.r[p] = z[0]; P.th[p] = z[1]; P.ph[p] = z[2];
    P.ur[p] = z[3]; P.uth[p] = z[4]; P.uph[p] = z[5];
    P.alive[p] = done ? 1 : 0;
    P.scheme[p] = 0;
    P.iters[p] = 0;
    if (done) set_energy(bh, P, p, z, B0pot);
}

__global__ void k_seed_fido(BH bh, PInit P, long long n, const double* __restrict__ d6, double B0pot)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double* d = d6 + 6 * p;
    double s, c;
    sincos(d[1], &s, &c);
    Geo g;
    geo_eval(bh, d[0], s, c, g);
    const double L11 = sqrt(g.grr);
    const double L31 = g.grp / L11;
    const double L22 = sqrt(g.gtt);
    const double L33 = sqrt(fma(-L31, L31, g.gpp));
    double z[6] = {d[0], d[1], d[2], L11 * d[3], L22 * d[4], fma(L31, d[3], L33 * d[5])};
    P.r[p] = z[0]; P.th[p] = z[1]; P.ph[p] = z[2];
    P.ur[p] = z[3]; P.uth[p] = z[4]; P.uph[p] = z[5];
    P.alive[p] = 1;
    P.scheme[p] = 0;
    P.iters[p] = 0;
    set_energy(bh, P, p, z, B0pot);
}

__global__ void k_hamiltonian(BH bh, PInit P, long long n, double B0pot, double* Hout, double* Lout)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double z[6] = {P.r[p], P.th[p], P.ph[p], P.ur[p], P.uth[p], P.uph[p]};
    const double qm = P.qm[p];
    if (Hout) Hout[p] = eval_H(bh, z, qm, B0pot);
    if (Lout) {
        double L = z[5];
        if (B0pot != 0.0 && qm != 0.0) {
            double s, c;
            sincos(z[1], &s, &c);
            const double rho2 = fma(bh.a2, c * c, z[0] * z[0]);
            // A_ph = (B0/2) s^2 [r^2 + a^2 - 2 M a^2 r (1 + c^2)/rho^2]   (Sec. 3.1.3)
            const double Aph = 0.5 * B0pot * s * s *
                               (z[0] * z[0] + bh.a2 - 2.0 * bh.M * bh.a2 * z[0] * (1.0 + c * c) / rho2);
            L = fma(qm, Aph, L);
        }
        Lout[p] = L;
    }
}

__global__ void k_cell(GridDev G, const double* r, const double* th, uint32_t* cell, long long n)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int i, j;
    double w;
    const double rr = r[p];
    double tt, thv;
    int mh;
    theta_views(G, th[p], tt, thv, mh);
    const float lr = __logf((float)rr);
    locate(G.rn, G.irn, G.Nr + 1, rr, (lr - G.lr0) * G.ilr, i, w);
    locate(G.tn, G.itn, G.Nth + 1, tt, ((float)tt - G.t0) * G.it, j, w);
    cell[p] = (uint32_t)i * (uint32_t)G.Nth + (uint32_t)j;
}

int build_metric_tables(fpic_ctx* c);   // pic.cu

}  // namespace fpic

using namespace fpic;

extern "C" const char* fpic_last_error(void) { return g_err.c_str(); }

extern "C" int fpic_init_metric(fpic_ctx** out, double M, double a)
{
    if (!out) return set_error(FPIC_EINVAL, "fpic_init_metric: ctx is NULL");
    *out = nullptr;
    if (!(M > 0.0) || !std::isfinite(M)) return set_error(FPIC_EINVAL, "fpic_init_metric: M must be > 0");
    if (!(fabs(a) <= M)) return set_error(FPIC_EINVAL, "fpic_init_metric: need |a| <= M");
    fpic_ctx* c = new fpic_ctx();
    c->M = M;
    c->a = a;
    c->bh = BH{M, a, a * a, 2.0 * M};
    c->r_h = M + sqrt(M * M - a * a);
    int rc = check_cuda(cudaGetDevice(&c->device), "cudaGetDevice");
    if (!rc) rc = check_cuda(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device),
                             "cudaDeviceGetAttribute");
    // the counters, then room for one fpic_push_stats assembled on the device (FPIC_TUNE_ASYNC)
    if (!rc) rc = check_cuda(cudaMalloc(&c->d_cnt, CNT_N * sizeof(long long) + sizeof(fpic_push_stats)),
                             "cudaMalloc(counters)");
    if (!rc) rc = check_cuda(cudaMallocHost(&c->h_cnt, CNT_N * sizeof(long long)), "cudaMallocHost");
    if (rc) {
        fpic_destroy(c);
        return rc;
    }
    *out = c;
    return FPIC_OK;
}

extern "C" void fpic_destroy(fpic_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->d_nodes) cudaFree(c->d_nodes);
    if (c->d_metric) cudaFree(c->d_metric);
    if (c->d_cnt) cudaFree(c->d_cnt);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->d_scratch) cudaFree(c->d_scratch);
    if (c->d_scratch2) cudaFree(c->d_scratch2);
    if (c->d_runs) cudaFree(c->d_runs);
    if (c->h_runs) cudaFreeHost(c->h_runs);
    for (cudaEvent_t e : c->copy_ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->clean_exec) cudaGraphExecDestroy(c->clean_exec);
    if (c->d_fcoef) cudaFree(c->d_fcoef);
    if (c->d_slope) cudaFree(c->d_slope);
    if (c->d_stage_maps) cudaFree(c->d_stage_maps);
    for (void* q : c->retired_dev) cudaFree(q);
    for (void* q : c->retired_host) cudaFreeHost(q);
    delete c;
}

static bool increasing(const double* x, int m)
{
    for (int i = 0; i < m; ++i)
        if (!std::isfinite(x[i])) return false;
    for (int i = 1; i < m; ++i)
        if (!(x[i] > x[i - 1])) return false;
    return true;
}

extern "C" int fpic_set_grid(fpic_ctx* c, int Nr, int Nth, const double* rn, const double* rh,
                             const double* tn, const double* th)
{
    if (!c || !rn || !rh || !tn || !th) return set_error(FPIC_EINVAL, "fpic_set_grid: NULL argument");
    if (Nr < 2 || Nth < 2 || Nr > (1 << 20) || Nth > (1 << 20) || (double)(Nr + 1) * (Nth + 1) > 2e9)
        return set_error(FPIC_EINVAL, "fpic_set_grid: Nr, Nth must be in [2, 2^20]");
    if (!increasing(rn, Nr + 1) || !increasing(rh, Nr) || !increasing(tn, Nth + 1) || !increasing(th, Nth))
        return set_error(FPIC_EINVAL, "fpic_set_grid: node tables must be finite and strictly increasing");
    if (!(rn[0] > 0.0)) return set_error(FPIC_EINVAL, "fpic_set_grid: r nodes must be positive");
    FPIC_CUDA(cudaSetDevice(c->device));
    // the half-th list carries one more node, th[Nth] = th[0] + (tn[Nth] - tn[0]):
    // the upper end of the full-theta wrap cell (unused in the half-theta domain)
    const size_t tot = 3 * ((size_t)(Nr + 1) + Nr + (Nth + 1) + (Nth + 1));
    std::vector<double> h(tot);
    double* p = h.data();
    size_t o_rn = 0, o_rh = o_rn + Nr + 1, o_tn = o_rh + Nr, o_th = o_tn + Nth + 1;
    size_t o_irn = o_th + Nth + 1, o_irh = o_irn + Nr + 1, o_itn = o_irh + Nr, o_ith = o_itn + Nth + 1;
    size_t o_brn = o_ith + Nth + 1, o_brh = o_brn + Nr + 1, o_btn = o_brh + Nr, o_bth = o_btn + Nth + 1;
    memcpy(p + o_rn, rn, (Nr + 1) * sizeof(double));
    memcpy(p + o_rh, rh, Nr * sizeof(double));
    memcpy(p + o_tn, tn, (Nth + 1) * sizeof(double));
    memcpy(p + o_th, th, Nth * sizeof(double));
    p[o_th + Nth] = th[0] + (tn[Nth] - tn[0]);
    auto inv = [](const double* X, int m, double* out) {
        for (int i = 0; i < m - 1; ++i) out[i] = 1.0 / (X[i + 1] - X[i]);
        out[m - 1] = 0.0;
    };
    inv(rn, Nr + 1, p + o_irn);
    inv(rh, Nr, p + o_irh);
    inv(tn, Nth + 1, p + o_itn);
    inv(p + o_th, Nth + 1, p + o_ith);
    // -X[i] / (X[i+1] - X[i]): a gather's cell weight (x - X[i]) / (X[i+1] - X[i])
    // as one fused multiply-add, x iX[i] + B[i]
    auto off = [](const double* X, const double* iX, int m, double* out) {
        for (int i = 0; i < m; ++i) out[i] = -(X[i] * iX[i]);
    };
    off(p + o_rn, p + o_irn, Nr + 1, p + o_brn);
    off(p + o_rh, p + o_irh, Nr, p + o_brh);
    off(p + o_tn, p + o_itn, Nth + 1, p + o_btn);
    off(p + o_th, p + o_ith, Nth + 1, p + o_bth);
    retire(c, (void**)&c->d_nodes);
    FPIC_CUDA(cudaMalloc(&c->d_nodes, tot * sizeof(double)));
    FPIC_CUDA(cudaMemcpy(c->d_nodes, p, tot * sizeof(double), cudaMemcpyHostToDevice));
    c->h_nodes.assign((const char*)p, (o_irn) * sizeof(double));
    double* d = c->d_nodes;
    GridDev& G = c->G;
    G.Nr = Nr;
    G.Nth = Nth;
    G.ld = Nth + 1;
    G.rn = d + o_rn; G.rh = d + o_rh; G.tn = d + o_tn; G.th = d + o_th;
    G.irn = d + o_irn; G.irh = d + o_irh; G.itn = d + o_itn; G.ith = d + o_ith;
    G.brn = d + o_brn; G.brh = d + o_brh; G.btn = d + o_btn; G.bth = d + o_bth;
    // FP32 index estimates (corrected exactly against the tables on device)
    const double l0 = log(rn[0]), l1 = log(rn[Nr]);
    G.lr0 = (float)l0;
    G.lrh0 = (float)log(rh[0]);
    G.ilr = (float)(Nr / (l1 - l0));
    G.t0 = (float)tn[0];
    G.th0 = (float)th[0];
    G.it = (float)(Nth / (tn[Nth] - tn[0]));
    G.full = 0;                      // half-theta until fpic_set_theta_mode says otherwise
    G.tlo = tn[0];
    G.tper = tn[Nth] - tn[0];
    G.thlo = th[0];
    c->Nr = Nr;
    c->Nth = Nth;
    c->ld = Nth + 1;
    c->has_grid = true;
    for (int i = 0; i < 6; ++i) c->fcoef_src[i] = nullptr;   // coefficients belong to the old grid
    ++c->grid_gen;                                            // and so do cached slopes
    int rc = build_metric_tables(c);
    if (rc) return rc;
    FPIC_CUDA(cudaDeviceSynchronize());
    return FPIC_OK;
}

extern "C" int fpic_set_theta_mode(fpic_ctx* c, int mode)
{
    if (!c) return set_error(FPIC_EINVAL, "fpic_set_theta_mode: NULL ctx");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_set_theta_mode: no grid set");
    if (mode != FPIC_THETA_HALF && mode != FPIC_THETA_FULL)
        return set_error(FPIC_EINVAL, "fpic_set_theta_mode: mode must be FPIC_THETA_HALF or FPIC_THETA_FULL");
    if (mode == FPIC_THETA_FULL && !(fabs(c->G.tper - 2.0 * M_PI) <= 1e-12 * 2.0 * M_PI))
        return set_error(FPIC_EINVAL, "fpic_set_theta_mode: a full-theta grid needs tn[Nth] - tn[0] = 2 pi (got %.17g)",
                         c->G.tper);
    c->G.full = mode == FPIC_THETA_FULL ? 1 : 0;
    for (int i = 0; i < 6; ++i) c->fcoef_src[i] = nullptr;   // the wrap cell's coefficients
    ++c->grid_gen;                                            // cached slopes belong to the old mode
    return FPIC_OK;
}

// Full-theta domain: column Nth of each component array is the image of
// column 0 (copied, so the two are equal bit for bit).
__global__ void k_theta_image(GridDev G, double* F0, double* F1, double* F2, double* F3, double* F4, double* F5)
{
    double* F[6] = {F0, F1, F2, F3, F4, F5};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= G.Nr; i += gridDim.x * blockDim.x)
        for (int k = 0; k < 6; ++k) {
            const bool ro = (k == 0 || k == 4 || k == 5);
            if (ro && i >= G.Nr) continue;
            F[k][(size_t)i * G.ld + G.Nth] = F[k][(size_t)i * G.ld];
        }
}

extern "C" int fpic_init_split_monopole(fpic_ctx* c, double* const fields[6], double B0, double zeta0,
                                        void* stream)
{
    if (!c || !fields) return set_error(FPIC_EINVAL, "fpic_init_split_monopole: NULL argument");
    for (int i = 0; i < 6; ++i)
        if (!fields[i]) return set_error(FPIC_EINVAL, "fpic_init_split_monopole: fields[%d] is NULL", i);
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_init_split_monopole: no grid set");
    if (c->G.full) return set_error(FPIC_EINVAL, "fpic_init_split_monopole: not in the full-theta domain");
    if (!std::isfinite(B0) || !std::isfinite(zeta0) || !(zeta0 > 0.0))
        return set_error(FPIC_EINVAL, "fpic_init_split_monopole: need finite B0 and zeta0 > 0");
    FPIC_CUDA(cudaSetDevice(c->device));
    dim3 grid(1, c->Nr + 1);
    k_split_monopole<<<grid, 256, 0, (cudaStream_t)stream>>>(c->bh, c->G, B0, zeta0, fields[0], fields[1],
                                                             fields[2], fields[3], fields[4], fields[5]);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_init_wald(fpic_ctx* c, double* const fields[6], double B0, void* stream)
{
    if (!c || !fields) return set_error(FPIC_EINVAL, "fpic_init_wald: NULL argument");
    for (int i = 0; i < 6; ++i)
        if (!fields[i]) return set_error(FPIC_EINVAL, "fpic_init_wald: fields[%d] is NULL", i);
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_init_wald: no grid set");
    if (!std::isfinite(B0)) return set_error(FPIC_EINVAL, "fpic_init_wald: B0 not finite");
    FPIC_CUDA(cudaSetDevice(c->device));
    dim3 grid(1, c->Nr + 1);
    k_wald<<<grid, 256, 0, (cudaStream_t)stream>>>(c->bh, c->G, B0, fields[0], fields[1], fields[2], fields[3],
                                                   fields[4], fields[5]);
    if (c->G.full)
        k_theta_image<<<(unsigned)((c->Nr + 1 + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
            c->G, fields[0], fields[1], fields[2], fields[3], fields[4], fields[5]);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_init_particles(fpic_ctx* c, fpic_particles* p, int kind, const double* draws, int K,
                                   double B0pot, void* stream)
{
    if (!c || !p) return set_error(FPIC_EINVAL, "fpic_init_particles: NULL argument");
    if (p->n < 0) return set_error(FPIC_EINVAL, "fpic_init_particles: n < 0");
    if (p->n == 0) return FPIC_OK;
    if (!particles_ok(p, true) || !draws) return set_error(FPIC_EINVAL, "fpic_init_particles: NULL array");
    if (kind == FPIC_SEED_ORBIT && K < 1) return set_error(FPIC_EINVAL, "fpic_init_particles: K must be >= 1");
    if (kind != FPIC_SEED_ORBIT && kind != FPIC_SEED_FIDO)
        return set_error(FPIC_EINVAL, "fpic_init_particles: unknown kind %d", kind);
    FPIC_CUDA(cudaSetDevice(c->device));
    PInit P{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->H0, p->D0, p->Hn, p->alive, p->scheme, p->iters};
    const unsigned nb = (unsigned)((p->n + 127) / 128);
    if (kind == FPIC_SEED_ORBIT)
        k_seed_orbit<<<nb, 128, 0, (cudaStream_t)stream>>>(c->bh, P, p->n, draws, K, B0pot);
    else
        k_seed_fido<<<nb, 128, 0, (cudaStream_t)stream>>>(c->bh, P, p->n, draws, B0pot);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_hamiltonian(fpic_ctx* c, const fpic_particles* p, double B0pot, double* H_out,
                                double* L_out, void* stream)
{
    if (!c || !p) return set_error(FPIC_EINVAL, "fpic_hamiltonian: NULL argument");
    if (p->n < 0) return set_error(FPIC_EINVAL, "fpic_hamiltonian: n < 0");
    if (p->n == 0) return FPIC_OK;
    if (!p->r || !p->th || !p->ph || !p->ur || !p->uth || !p->uph || !p->qm)
        return set_error(FPIC_EINVAL, "fpic_hamiltonian: NULL state array");
    FPIC_CUDA(cudaSetDevice(c->device));
    PInit P{p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const unsigned nb = (unsigned)((p->n + 127) / 128);
    k_hamiltonian<<<nb, 128, 0, (cudaStream_t)stream>>>(c->bh, P, p->n, B0pot, H_out, L_out);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_cell_index(fpic_ctx* c, fpic_particles* p, void* stream)
{
    if (!c || !p) return set_error(FPIC_EINVAL, "fpic_cell_index: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_cell_index: no grid set");
    if (p->n < 0) return set_error(FPIC_EINVAL, "fpic_cell_index: n < 0");
    if (p->n == 0) return FPIC_OK;
    if (!p->r || !p->th || !p->cell) return set_error(FPIC_EINVAL, "fpic_cell_index: NULL array");
    FPIC_CUDA(cudaSetDevice(c->device));
    const unsigned nb = (unsigned)((p->n + 255) / 256);
    k_cell<<<nb, 256, 0, (cudaStream_t)stream>>>(c->G, p->r, p->th, p->cell, p->n);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}
