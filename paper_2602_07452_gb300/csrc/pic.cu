// Grid side of the PIC step: metric tables at the Yee points (Sec. 2.1),
// the stable sort of particles by cell, the deterministic volume-weighted
// deposit (Sec. 2.3) and the FDTD leapfrog (Sec. 2.1, 2.5).
//
// Deposit pipeline (no floating-point atomics, bitwise reproducible):
//   k_dep_particle  one thread per particle (in cell order): the 4x4
//                   trapezoidal subvolumes of sqrt(gamma) on each sub-grid
//                   -> 16 node shares (rho, j^ph, j^r, j^th);
//   k_dep_cell      one warp per cell, one lane per record row and
//                   particle parity: fixed-order sums of the cell's
//                   particles' shares into its 20 stencil slots;
//   k_dep_node      one thread per node: fixed-order sum of the slots of the
//                   (up to six) cells touching it, / (2 pi V_dual).
// The FDTD is HBM-bound; its metric factors come from tables built once.
#include <math.h>

#include "ff.cuh"
#include "fpic_internal.h"

namespace fpic {

// ---------------------------------------------------------------------------
// Metric tables
// ---------------------------------------------------------------------------
// type t: 0 (i, j), 1 (i+1/2, j), 2 (i, j+1/2), 3 (i+1/2, j+1/2)
// quantity q: 0 alpha, 1 beta, 2 sqrt(gamma), 3 g_rr, 4 g_rp, 5 g_tt, 6 g_pp,
// 7 1/sqrt(gamma) (the FDTD multiplies by it instead of dividing)
// tables 32..34: 2 pi x dual-cell volume of the (i,j), (i+1/2,j), (i,j+1/2) grids
// then sin/cos of the integer and half th nodes.
enum { MT_Q = 8, MT_DUAL = 32, MT_N = 35 };

struct Tabs {
    const double* m;   // MT_N tables of size sz, then 2 (Nth+1) + 2 Nth trig values
    size_t sz;
    int ld;
    __device__ __forceinline__ double at(int t, int q, int i, int j) const
    {
        return m[(size_t)(t * MT_Q + q) * sz + (size_t)i * ld + j];
    }
    __device__ __forceinline__ double dual(int t, int i, int j) const
    {
        return m[(size_t)(MT_DUAL + t) * sz + (size_t)i * ld + j];
    }
};

__device__ __forceinline__ double sqrtg_sc(const BH& bh, double r, double s, double c)
{
    // sqrt(gamma) = rho^2 sqrt(xi) sin th = sin th sqrt(rho^2 (rho^2 + 2 M r))
    const double rho2 = fma(bh.a2, c * c, r * r);
    return s * sqrt(rho2 * fma(bh.twoM, r, rho2));
}

__device__ double trap16_dev(const BH& bh, double x0, double x1, double y0, double y1)
{
    const double wt[4] = {0.5, 1.0, 1.0, 0.5};
    const double hx = (x1 - x0) / 3.0, hy = (y1 - y0) / 3.0;
    double acc = 0.0;
    for (int l = 0; l < 4; ++l) {
        double s, c;
        sincos(y0 + l * hy, &s, &c);
        double row = 0.0;
        for (int k = 0; k < 4; ++k) row = fma(wt[k], sqrtg_sc(bh, x0 + k * hx, s, c), row);
        acc = fma(wt[l], row, acc);
    }
    return acc * hx * hy;
}

__global__ void k_metric_tables(BH bh, GridDev G, double* m, size_t sz)
{
    const int i = blockIdx.y;
    for (int j = threadIdx.x; j <= G.Nth; j += blockDim.x) {
        for (int t = 0; t < 4; ++t) {
            const bool ro = t & 1, to = t & 2;
            if ((ro && i >= G.Nr) || (to && j >= G.Nth)) continue;
            const double r = ro ? G.rh[i] : G.rn[i];
            const double th = to ? G.th[j] : G.tn[j];
            double s, c;
            sincos(th, &s, &c);
            Geo g;
            geo_eval(bh, r, s, c, g);
            const double v[MT_Q] = {g.alpha, g.beta, g.sqrtg, g.grr, g.grp, g.gtt, g.gpp, 1.0 / g.sqrtg};
            for (int q = 0; q < MT_Q; ++q) m[(size_t)(t * MT_Q + q) * sz + (size_t)i * G.ld + j] = v[q];
        }
        // dual-cell volumes of the (i,j), (i+1/2,j), (i,j+1/2) sub-grids
        for (int t = 0; t < 3; ++t) {
            const bool ro = (t == 1), to = (t == 2);
            if ((ro && i >= G.Nr) || (to && j >= G.Nth)) continue;
            double x0, x1, y0, y1;
            if (ro) { x0 = G.rn[i]; x1 = G.rn[i + 1]; }
            else { x0 = i == 0 ? G.rn[0] : G.rh[i - 1]; x1 = i == G.Nr ? G.rn[G.Nr] : G.rh[i]; }
            if (to) { y0 = G.tn[j]; y1 = G.tn[j + 1]; }
            else { y0 = j == 0 ? G.tn[0] : G.th[j - 1]; y1 = j == G.Nth ? G.tn[G.Nth] : G.th[j]; }
            m[(size_t)(MT_DUAL + t) * sz + (size_t)i * G.ld + j] = 2.0 * M_PI * trap16_dev(bh, x0, x1, y0, y1);
        }
    }
    if (i == 0) {
        double* trig = m + (size_t)MT_N * sz;
        for (int j = threadIdx.x; j <= G.Nth; j += blockDim.x) {
            double s, c;
            sincos(G.tn[j], &s, &c);
            trig[j] = s;
            trig[(G.Nth + 1) + j] = c;
            if (j < G.Nth) {
                sincos(G.th[j], &s, &c);
                trig[2 * (G.Nth + 1) + j] = s;
                trig[2 * (G.Nth + 1) + G.Nth + j] = c;
            }
        }
    }
}

int build_metric_tables(fpic_ctx* c)
{
    const size_t sz = (size_t)(c->Nr + 1) * c->ld;
    const size_t tot = (size_t)MT_N * sz + 2 * (size_t)(c->Nth + 1) + 2 * (size_t)c->Nth;
    retire(c, (void**)&c->d_metric);
    FPIC_CUDA(cudaMalloc(&c->d_metric, tot * sizeof(double)));
    c->metric_stride = sz;
    dim3 grid(1, c->Nr + 1);
    k_metric_tables<<<grid, 128>>>(c->bh, c->G, c->d_metric, sz);
    FPIC_CUDA(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------------------
// Stable sort by cell
// ---------------------------------------------------------------------------
struct SortBufs {
    uint32_t *key, *perm, *perm2, *count, *cursor, *off, *bsum;
    void* tmp;
};

// count[k] += 1 for each valid lane's key k, one atomic per distinct key of
// the warp (particles arrive nearly sorted by cell: most of a warp shares one
// key, and same-address atomics would serialise).  Every lane of the warp
// calls it; an invalid lane's 64-bit key matches no valid one.
__device__ __forceinline__ void count_key(uint32_t* count, uint32_t k, bool valid)
{
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? (unsigned long long)k : (1ull << 32));
    if (valid && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&count[k], (unsigned)__popc(peers));
}

__global__ void k_keys(GridDev G, const double* r, const double* th, const uint8_t* alive, uint32_t* key,
                       uint32_t* cell, uint32_t* count, long long n, uint32_t C)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool valid = p < n;
    uint32_t k = 0;
    if (valid) {
        int i, j;
        double w;
        const double rr = r[p];
        double tt, thv;
        int mh;
        theta_views(G, th[p], tt, thv, mh);
        const float lr = __logf((float)rr);
        locate(G.rn, G.irn, G.Nr + 1, rr, (lr - G.lr0) * G.ilr, i, w);
        locate(G.tn, G.itn, G.Nth + 1, tt, ((float)tt - G.t0) * G.it, j, w);
        const uint32_t c = (uint32_t)i * (uint32_t)G.Nth + (uint32_t)j;
        if (cell) cell[p] = c;
        k = alive[p] ? c : C;
        key[p] = k;
    }
    count_key(count, k, valid);
}

// exclusive scan of count[0..m) into off[0..m], m + 1 outputs; three phases
constexpr int SCAN_B = 1024, SCAN_PER = 4;
__global__ void k_scan_blocks(const uint32_t* in, uint32_t* out, uint32_t* bsum, long long m)
{
    __shared__ uint32_t sh[SCAN_B];
    const long long base = (long long)blockIdx.x * SCAN_B * SCAN_PER;
    uint32_t v[SCAN_PER], tot = 0;
    for (int k = 0; k < SCAN_PER; ++k) {
        const long long idx = base + (long long)threadIdx.x * SCAN_PER + k;
        v[k] = idx < m ? in[idx] : 0u;
        tot += v[k];
    }
    sh[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < SCAN_B; o <<= 1) {
        uint32_t t = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = sh[threadIdx.x] - tot;   // exclusive prefix of this thread
    for (int k = 0; k < SCAN_PER; ++k) {
        const long long idx = base + (long long)threadIdx.x * SCAN_PER + k;
        if (idx < m) out[idx] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_B - 1) bsum[blockIdx.x] = sh[SCAN_B - 1];
}

// In-place exclusive scan of bsum[0..nb), bsum[nb] = the total: one block of
// SCAN_B threads, each over a contiguous run of ceil(nb / SCAN_B) entries.
__global__ void __launch_bounds__(SCAN_B) k_scan_bsum(uint32_t* bsum, int nb)
{
    __shared__ uint32_t wsum[SCAN_B / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int per = (nb + SCAN_B - 1) / SCAN_B;
    const int lo = min(nb, t * per), hi = min(nb, lo + per);
    uint32_t tot = 0;
    for (int b = lo; b < hi; ++b) tot += bsum[b];
    uint32_t inc = tot;                 // inclusive scan of the thread totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = inc - tot + (wid > 0 ? wsum[wid - 1] : 0u);
    for (int b = lo; b < hi; ++b) {
        const uint32_t v = bsum[b];
        bsum[b] = run;
        run += v;
    }
    if (t == SCAN_B - 1) bsum[nb] = run;
}

__global__ void k_scan_add(uint32_t* out, const uint32_t* bsum, long long m, int nb)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < m) out[idx] += bsum[idx / (SCAN_B * SCAN_PER)];
    if (idx == 0) out[m] = bsum[nb];
}

__global__ void k_scatter(const uint32_t* key, const uint32_t* off, uint32_t* cursor, uint32_t* perm, long long n)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool valid = p < n;
    const uint32_t k = valid ? key[p] : 0u;
    // one atomic per distinct key of the warp; lanes of a key take
    // consecutive places in lane order (every lane takes part in the match)
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? (unsigned long long)k : (1ull << 32));
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&cursor[k], (unsigned)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) perm[off[k] + base + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = (uint32_t)p;
}

// Order every bucket by particle index (rank = number of smaller indices in
// the bucket): one warp per bucket.  Removed particles (last bucket) are
// handled by k_dead_rank.
__global__ void k_bucket_rank(const uint32_t* off, const uint32_t* perm, uint32_t* perm2, uint32_t C)
{
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= C) return;
    const uint32_t b0 = off[warp], b1 = off[warp + 1];
    // a bucket already in index order (the usual case: nearly sorted input,
    // whole warps placed in lane order) is copied as it is
    bool sorted = true;
    for (uint32_t a = b0 + lane; a + 1 < b1; a += 32) sorted = sorted && perm[a] < perm[a + 1];
    if (__all_sync(0xffffffffu, sorted)) {
        for (uint32_t a = b0 + lane; a < b1; a += 32) perm2[a] = perm[a];
        return;
    }
    for (uint32_t a = b0 + lane; a < b1; a += 32) {
        const uint32_t x = perm[a];
        uint32_t rank = 0;
        for (uint32_t b = b0; b < b1; ++b) rank += perm[b] < x ? 1u : 0u;
        perm2[b0 + rank] = x;
    }
}

// Removed particles keep their relative order: position = off[C] + number of
// removed particles with a smaller index.  Blocks of DEAD_T threads cover
// DEAD_PER x DEAD_T consecutive particles (thread t takes particles
// base + k DEAD_T + t); k_dead_count writes each block's count, an exclusive
// scan turns the counts into block offsets, and k_dead_place ranks the
// block's removed particles by ballots in index order.
constexpr int DEAD_T = 256, DEAD_PER = 16, DEAD_W = DEAD_T / 32;

__global__ void __launch_bounds__(DEAD_T) k_dead_count(const uint8_t* alive, uint32_t* bcnt, long long n)
{
    __shared__ uint32_t ws[DEAD_W];
    const long long base = (long long)blockIdx.x * DEAD_PER * DEAD_T;
    uint32_t d = 0;
#pragma unroll
    for (int k = 0; k < DEAD_PER; ++k) {
        const long long q = base + (long long)k * DEAD_T + threadIdx.x;
        d += (q < n && !alive[q]) ? 1u : 0u;
    }
    d = __reduce_add_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < DEAD_W; ++w) t += ws[w];
        bcnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(DEAD_T) k_dead_place(const uint8_t* alive, const uint32_t* boff,
                                                       const uint32_t* off, uint32_t* perm2, long long n, uint32_t C)
{
    __shared__ uint32_t pre[DEAD_PER * DEAD_W];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * DEAD_PER * DEAD_T;
    unsigned m[DEAD_PER];
#pragma unroll
    for (int k = 0; k < DEAD_PER; ++k) {
        const long long q = base + (long long)k * DEAD_T + threadIdx.x;
        m[k] = __ballot_sync(0xffffffffu, q < n && !alive[q]);
        if (lane == 0) pre[k * DEAD_W + wid] = (uint32_t)__popc(m[k]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {             // exclusive prefix in index order (k, then warp)
        uint32_t run = 0;
        for (int e = 0; e < DEAD_PER * DEAD_W; ++e) {
            const uint32_t v = pre[e];
            pre[e] = run;
            run += v;
        }
    }
    __syncthreads();
    const uint32_t at = off[C] + boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < DEAD_PER; ++k)
        if ((m[k] >> lane) & 1u) {
            const long long q = base + (long long)k * DEAD_T + threadIdx.x;
            perm2[at + pre[k * DEAD_W + wid] + (uint32_t)__popc(m[k] & ((1u << lane) - 1u))] = (uint32_t)q;
        }
}

template <typename T>
__global__ void k_gather_perm(const T* __restrict__ src, T* __restrict__ dst, const uint32_t* __restrict__ perm,
                              long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

// Every particle array permuted at once (the deposit's sort): one pass
// gathers them all through the permutation into a staging area (11 x n
// doubles, then n u32, then 3 x n bytes), reading the permutation once, and
// one pass copies them back, instead of a gather and a copy per array.
struct PermArrays {
    double* d[11];
    uint8_t* b[3];
    uint32_t* u;
};

__global__ void k_gather_all(PermArrays a, const uint32_t* __restrict__ perm, double* __restrict__ stage, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    uint32_t* su = (uint32_t*)(stage + 11 * n);
    uint8_t* sb = (uint8_t*)(su + n);
#pragma unroll
    for (int k = 0; k < 11; ++k)
        if (a.d[k]) stage[k * n + i] = a.d[k][j];
    if (a.u) su[i] = a.u[j];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (a.b[k]) sb[k * n + i] = a.b[k][j];
}

__global__ void k_copy_all(PermArrays a, const double* __restrict__ stage, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t* su = (const uint32_t*)(stage + 11 * n);
    const uint8_t* sb = (const uint8_t*)(su + n);
#pragma unroll
    for (int k = 0; k < 11; ++k)
        if (a.d[k]) a.d[k][i] = stage[k * n + i];
    if (a.u) a.u[i] = su[i];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (a.b[k]) a.b[k][i] = sb[k * n + i];
}

static int scan_u32(const uint32_t* in, uint32_t* out, uint32_t* bsum, long long m, cudaStream_t s)
{
    const int nb = (int)((m + SCAN_B * SCAN_PER - 1) / (SCAN_B * SCAN_PER));
    k_scan_blocks<<<nb, SCAN_B, 0, s>>>(in, out, bsum, m);
    k_scan_bsum<<<1, SCAN_B, 0, s>>>(bsum, nb);
    k_scan_add<<<(unsigned)((m + 255) / 256 + 1), 256, 0, s>>>(out, bsum, m, nb);
    return check_cuda(cudaGetLastError(), "scan");
}

// Scratch2 layout for sort + deposit.
struct Work {
    uint32_t *key, *perm, *perm2, *count, *cursor, *off, *bsum, *flag, *pos;
    double* tmp;        // n doubles (permutation buffer)
    double* rec;        // 16 x n deposit shares
    uint32_t* code;     // n stencil offsets
    double* part;       // 20 x C cell partials
};

static int work_layout(fpic_ctx* c, long long n, bool deposit, Work& w, size_t extra_bytes = 0,
                       void** extra = nullptr)
{
    const long long C = (long long)c->Nr * c->Nth;
    const long long nbs = (n > C + 2 ? n : C + 2) / (SCAN_B * SCAN_PER) + 2;
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
    size_t o_key = take(4 * n), o_perm = take(4 * n), o_perm2 = take(4 * n), o_count = take(4 * (C + 2)),
           o_cursor = take(4 * (C + 2)), o_off = take(4 * (C + 2)), o_bsum = take(4 * nbs), o_flag = take(4 * n),
           o_pos = take(4 * (n + 1)), o_tmp = take(8 * n);
    size_t o_rec = 0, o_code = 0, o_part = 0;
    if (deposit) {
        o_rec = take(16 * 8 * (size_t)n);
        o_code = take(4 * n);
        o_part = take(20 * 8 * (size_t)C);
    }
    const size_t o_extra = extra_bytes ? take(extra_bytes) : 0;
    int rc = ensure_scratch2(c, bytes);
    if (rc) return rc;
    char* b = (char*)c->d_scratch2;
    if (extra) *extra = extra_bytes ? (void*)(b + o_extra) : nullptr;
    w.key = (uint32_t*)(b + o_key);
    w.perm = (uint32_t*)(b + o_perm);
    w.perm2 = (uint32_t*)(b + o_perm2);
    w.count = (uint32_t*)(b + o_count);
    w.cursor = (uint32_t*)(b + o_cursor);
    w.off = (uint32_t*)(b + o_off);
    w.bsum = (uint32_t*)(b + o_bsum);
    w.flag = (uint32_t*)(b + o_flag);
    w.pos = (uint32_t*)(b + o_pos);
    w.tmp = (double*)(b + o_tmp);
    w.rec = deposit ? (double*)(b + o_rec) : nullptr;
    w.code = deposit ? (uint32_t*)(b + o_code) : nullptr;
    w.part = deposit ? (double*)(b + o_part) : nullptr;
    return 0;
}

// stage: nullable, room for 12 x n doubles (the deposit's record buffer,
// unused until the sort is done): every array is permuted in two passes.
static int sort_impl(fpic_ctx* c, fpic_particles* p, Work& w, cudaStream_t s, double* stage = nullptr)
{
    const long long n = p->n;
    const uint32_t C = (uint32_t)c->Nr * (uint32_t)c->Nth;
    const unsigned nb = (unsigned)((n + 255) / 256);
    FPIC_CUDA(cudaMemsetAsync(w.count, 0, 4 * ((size_t)C + 2), s));
    FPIC_CUDA(cudaMemsetAsync(w.cursor, 0, 4 * ((size_t)C + 2), s));
    k_keys<<<nb, 256, 0, s>>>(c->G, p->r, p->th, p->alive, w.key, p->cell, w.count, n, C);
    int rc = scan_u32(w.count, w.off, w.bsum, (long long)C + 1, s);
    if (rc) return rc;
    k_scatter<<<nb, 256, 0, s>>>(w.key, w.off, w.cursor, w.perm, n);
    k_bucket_rank<<<(unsigned)(((long long)C * 32 + 255) / 256), 256, 0, s>>>(w.off, w.perm, w.perm2, C);
    // removed particles: per-block counts in w.pos (nbd + 1 <= n + 1 entries)
    const unsigned nbd = (unsigned)((n + DEAD_PER * DEAD_T - 1) / (DEAD_PER * DEAD_T));
    k_dead_count<<<nbd, DEAD_T, 0, s>>>(p->alive, w.pos, n);
    k_scan_bsum<<<1, SCAN_B, 0, s>>>(w.pos, (int)nbd);
    k_dead_place<<<nbd, DEAD_T, 0, s>>>(p->alive, w.pos, w.off, w.perm2, n, C);
    FPIC_CUDA(cudaGetLastError());
    double* d8[] = {p->r, p->th, p->ph, p->ur, p->uth, p->uph, p->qm, p->w, p->H0, p->D0, p->Hn};
    if (stage) {
        PermArrays a;
        for (int k = 0; k < 11; ++k) a.d[k] = d8[k];
        a.b[0] = p->alive; a.b[1] = p->scheme; a.b[2] = p->iters;
        a.u = p->cell;
        k_gather_all<<<nb, 256, 0, s>>>(a, w.perm2, stage, n);
        k_copy_all<<<nb, 256, 0, s>>>(a, stage, n);
        FPIC_CUDA(cudaGetLastError());
        return 0;
    }
    for (double* a : d8) {
        if (!a) continue;
        k_gather_perm<double><<<nb, 256, 0, s>>>(a, w.tmp, w.perm2, n);
        FPIC_CUDA(cudaMemcpyAsync(a, w.tmp, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    uint8_t* d1[] = {p->alive, p->scheme, p->iters};
    for (uint8_t* a : d1) {
        if (!a) continue;
        k_gather_perm<uint8_t><<<nb, 256, 0, s>>>(a, (uint8_t*)w.tmp, w.perm2, n);
        FPIC_CUDA(cudaMemcpyAsync(a, w.tmp, (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    if (p->cell) {
        k_gather_perm<uint32_t><<<nb, 256, 0, s>>>(p->cell, (uint32_t*)w.tmp, w.perm2, n);
        FPIC_CUDA(cudaMemcpyAsync(p->cell, w.tmp, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    FPIC_CUDA(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------------------
// Deposit (Sec. 2.3)
// ---------------------------------------------------------------------------

// (s, c) of angle x + h from (s, c) of x and (sin h, cos h - 1).
__device__ __forceinline__ void rotate(double s, double c, double sh, double cm, double& so, double& co)
{
    so = fma(s, cm, fma(c, sh, s));
    co = fma(c, cm, fma(-s, sh, c));
}

// sin/cos at the 7 lattice th values of the th cell [y0, y1] split at t:
// y0 + l hc (l = 0..3, y0 + 3 hc = t), t + l hd (l = 1..3, t + 3 hd = y1).
// The end points come in (node tables, the particle's own sin/cos); the
// interior points are angle-addition rotations by hc, 2 hc, hd, 2 hd.
__device__ __forceinline__ void theta_lattice(double hc, double hd, double s0, double c0, double st, double ct,
                                              double s1, double c1, double sy[7], double cy[7])
{
    double sh, cm;
    sy[0] = s0; cy[0] = c0;
    sy[3] = st; cy[3] = ct;
    sy[6] = s1; cy[6] = c1;
    sincos_step(hc, sh, cm);
    rotate(s0, c0, sh, cm, sy[1], cy[1]);
    // double angle: sin 2h = 2 sin h cos h, cos 2h - 1 = 2 (cos h - 1)(cos h + 1)
    rotate(s0, c0, 2.0 * fma(sh, cm, sh), 2.0 * cm * (cm + 2.0), sy[2], cy[2]);
    sincos_step(hd, sh, cm);
    rotate(st, ct, sh, cm, sy[4], cy[4]);
    rotate(st, ct, 2.0 * fma(sh, cm, sh), 2.0 * cm * (cm + 2.0), sy[5], cy[5]);
}

// 4x4 trapezoid lattice of a sub-grid cell [x0, x1] x [y0, y1] split at
// (r, t): the four subvolumes V00 = [x0,r]x[y0,t], V10 = [r,x1]x[y0,t],
// V01 = [x0,r]x[t,y1], V11 = [r,x1]x[t,y1], each by its own 4 x 4 rule; the
// points of the 7 x 7 lattice are evaluated once.  With X = x^2,
// B = X + 2 M x and A = a^2 cos^2 th, sqrt(gamma) = sin th sqrt((X + A)(B + A))
// and the radicand is X B + A (X + B + A): two operations per point.  The
// sin th factor is applied once per lattice row.
// The three sub-grids of a particle share lattice lines: the split column
// x = r of the (i, j) and (i+1/2, j) lattices (same th rows) and the split
// row th = t of the (i, j) and (i, j+1/2) lattices (same r columns), when
// neither split point was clamped.  col / row carry those 7 values: written
// by every call, read instead of evaluated with COL_IN / ROW_IN.
template <bool COL_IN = false, bool ROW_IN = false>
__device__ __forceinline__ void subvolumes(const BH& bh, double x0, double x1, double r, double hc, double hd,
                                           const double sy[7], const double cy[7], double V[4], double col[7],
                                           double row[7])
{
    const double third = 1.0 / 3.0;
    const double ha = (r - x0) * third, hb = (x1 - r) * third;
    double P[7], Q[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const double x = k < 3 ? fma((double)k, ha, x0) : (k == 3 ? r : fma((double)(k - 3), hb, r));
        const double X = x * x, B = fma(bh.twoM, x, X);
        P[k] = X * B;
        Q[k] = X + B;
    }
    // the lattice values are 2 sqrt(...) (sqrt2_dep): a common factor of the
    // four subvolumes, which only enter as ratios
    double S00 = 0, S10 = 0, S01 = 0, S11 = 0;
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        const double A = bh.a2 * (cy[l] * cy[l]);
        double f[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            if (ROW_IN && l == 3) f[k] = row[k];
            else if (COL_IN && k == 3) f[k] = col[l];
            else f[k] = sqrt2_dep(fma(A, Q[k] + A, P[k]));
        }
        if (!COL_IN) col[l] = f[3];
        if (!ROW_IN && l == 3) {
#pragma unroll
            for (int k = 0; k < 7; ++k) row[k] = f[k];
        }
        // trapezoid weights 1/2, 1, 1, 1/2 along r on each half; the row's
        // th weight (1/2 at the ends and the split row) times sin th
        const double ra = fma(0.5, f[0] + f[3], f[1] + f[2]);
        const double rb = fma(0.5, f[3] + f[6], f[4] + f[5]);
        const double ws = (l == 0 || l == 3 || l == 6) ? 0.5 * sy[l] : sy[l];
        if (l <= 3) { S00 = fma(ws, ra, S00); S10 = fma(ws, rb, S10); }
        if (l >= 3) { S01 = fma(ws, ra, S01); S11 = fma(ws, rb, S11); }
    }
    V[0] = S00 * (ha * hc);
    V[1] = S10 * (hb * hc);
    V[2] = S01 * (ha * hd);
    V[3] = S11 * (hb * hd);
}

// The same lattices in paired-FP32 arithmetic (ff.cuh): the lattice
// coordinates and step sizes, the sin/cos rotations of the th lattice, the
// radicand, its square root, the trapezoid sums and the subvolumes run on
// the FP32 pipe (about 48 bits; the square root to about 2^-44, against
// 2^-39.6 for the FP64 form above), which issues 64 times the FP64 rate.
// The values are sqrt(...) itself (no factor 2).
struct BHff {
    ff twoM, a2, third;
};

__device__ __forceinline__ void rotate_ff(ff s, ff c, ff sh, ff cm, ff& so, ff& co)
{
    so = ff_add(s, ff_add(ff_mul(c, sh), ff_mul(s, cm)));
    co = ff_add(c, ff_add(ff_neg(ff_mul(s, sh)), ff_mul(c, cm)));
}

// sin and cos of th = x + d from those of a node x (table doubles) and an
// offset d under a cell (a double: the difference of two close doubles,
// formed in FP64).
__device__ __forceinline__ void sincos_from_node(double s0, double c0, double d, ff& s, ff& c)
{
    ff sh, cm;
    sincos_step_ff(d, sh, cm);
    rotate_ff(ff_from(s0), ff_from(c0), sh, cm, s, c);
}

// The 7 th values of the lattice of [y0, y1] split at t: y0 + l hc
// (l = 0..3), t + l hd (l = 1..3); the end points' sin/cos come in.
__device__ __forceinline__ void theta_lattice_ff(ff hc, ff hd, ff s0, ff c0, ff st, ff ct, ff s1, ff c1, ff sy[7],
                                                 ff cy[7])
{
    sy[0] = s0; cy[0] = c0;
    sy[3] = st; cy[3] = ct;
    sy[6] = s1; cy[6] = c1;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int b = 3 * half;
        ff sh, cm;
        sincos_step_ff(half ? hd : hc, sh, cm);
        rotate_ff(sy[b], cy[b], sh, cm, sy[b + 1], cy[b + 1]);
        // double angle: sin 2h = 2 sin h (1 + (cos h - 1)), cos 2h - 1 = 2 (cos h - 1)(cos h - 1 + 2)
        const ff sh2 = ff_scale(ff_add(sh, ff_mul(sh, cm)), 2.f);
        const ff cm2 = ff_scale(ff_mul(cm, ff_add(cm, ff_of(2.f))), 2.f);
        rotate_ff(sy[b], cy[b], sh2, cm2, sy[b + 2], cy[b + 2]);
    }
}

// One sub-grid lattice in paired FP32, row by row (the row loop is not
// unrolled: one copy of the code serves every row and, through
// k_dep_particle_ff's loop, every sub-grid): r columns x0 + k ha (k = 0..3,
// x0 + 3 ha = r), r + k hb (k = 1..3).  col_in / row_in: take the split
// column / row from col / row instead of evaluating them; put_shared: store
// this lattice's split column and row there.  V: the four subvolumes.
__device__ __forceinline__ void subvolumes_ff(const BHff& bh, ff x0f, ff rf, ff ha, ff hb, ff hc, ff hd,
                                              const ff* sy, const ff* cy, ff V[4], ff* col, ff row[7],
                                              bool col_in, bool row_in, bool put_shared)
{
    ff P[7], Q[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        ff x;
        if (k == 0) x = x0f;
        else if (k < 3) x = ff_add(x0f, k == 1 ? ha : ff_scale(ha, 2.f));
        else if (k == 3) x = rf;
        else x = ff_add(rf, k == 4 ? hb : (k == 5 ? ff_scale(hb, 2.f) : ff_mulf(hb, 3.f)));
        const ff X = ff_sqr(x), B = ff_add(X, ff_mul(bh.twoM, x));
        P[k] = ff_mul(X, B);
        Q[k] = ff_add_ge(B, X);                        // B = X + 2 M x >= X
    }
    ff S00 = ff_of(0.f), S10 = ff_of(0.f), S01 = ff_of(0.f), S11 = ff_of(0.f);
#pragma unroll 1
    for (int l = 0; l < 7; ++l) {
        ff f[7];
        if (row_in && l == 3) {
#pragma unroll
            for (int k = 0; k < 7; ++k) f[k] = row[k];
        } else {
            const ff A = ff_mul(bh.a2, ff_sqr(cy[l]));
#pragma unroll
            for (int k = 0; k < 7; ++k)
                if (k != 3 || !col_in) f[k] = ff_sqrt(ff_add(P[k], ff_mul(A, ff_add(Q[k], A))));
            if (col_in) f[3] = col[l];
        }
        if (put_shared) {
            col[l] = f[3];
            if (l == 3) {
#pragma unroll
                for (int k = 0; k < 7; ++k) row[k] = f[k];
            }
        }
        // trapezoid weights 1/2, 1, 1, 1/2 along r on each half; the row's
        // th weight (1/2 at the ends and the split row) times sin th.  Along
        // a row sqrt(gamma) grows with r (both factors of the radicand do),
        // so f[k] <= f[k'] for k < k': the pair sums take the fast two-sum
        const ff ra = ff_add(ff_scale(ff_add_ge(f[3], f[0]), 0.5f), ff_add_ge(f[2], f[1]));
        const ff rb = ff_add(ff_scale(ff_add_ge(f[6], f[3]), 0.5f), ff_add_ge(f[5], f[4]));
        const ff ws = ff_scale(sy[l], (l == 0 || l == 3 || l == 6) ? 0.5f : 1.f);
        if (l <= 3) { S00 = ff_add(S00, ff_mul(ws, ra)); S10 = ff_add(S10, ff_mul(ws, rb)); }
        if (l >= 3) { S01 = ff_add(S01, ff_mul(ws, ra)); S11 = ff_add(S11, ff_mul(ws, rb)); }
    }
    V[0] = ff_mul(S00, ff_mul(ha, hc));
    V[1] = ff_mul(S10, ff_mul(hb, hc));
    V[2] = ff_mul(S01, ff_mul(ha, hd));
    V[3] = ff_mul(S11, ff_mul(hb, hd));
}

struct DepK {
    BH bh;
    BHff bhf;        // 2M and a^2 as paired floats
    GridDev G;
    const double* trig;  // sin tn[0..Nth], cos tn[0..Nth], sin th[0..Nth-1], cos th[0..Nth-1]
    const double *r, *th, *ur, *uth, *uph, *qm, *w;
    long long n_alive;
    double* rec;     // 16 x n
    uint32_t* code;  // (i1 - i0 + 1) | (j1 - j0 + 1) << 2
};

__device__ __forceinline__ double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

__global__ void __launch_bounds__(256) k_dep_particle(DepK k)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= k.n_alive) return;
    const GridDev& G = k.G;
    const double r = k.r[p], t = k.th[p];
    // FIDO three-velocity v^i = gamma^ij u_j / Gamma at the particle
    double s, c;
    sincos(t, &s, &c);
    Geo g;
    geo_eval(k.bh, r, s, c, g);
    const double ur = k.ur[p], ut = k.uth[p], up = k.uph[p];
    const double Ur = fma(g.gurr, ur, g.gurp * up), Ut = g.gutt * ut, Up = fma(g.gurp, ur, g.gupp * up);
    const double iG = rsqrt_nr(fma(ur, Ur, fma(ut, Ut, fma(up, Up, 1.0))));
    const double Q = k.w[p] * k.qm[p];
    const double vr = Ur * iG, vt = Ut * iG, vp = Up * iG;
    // clamped positions and cells on the integer and half node lists
    const double rn_c = clampd(r, G.rn[0], G.rn[G.Nr]), rh_c = clampd(r, G.rh[0], G.rh[G.Nr - 1]);
    const double tn_c = clampd(t, G.tn[0], G.tn[G.Nth]), th_c = clampd(t, G.th[0], G.th[G.Nth - 1]);
    int i0, i1, j0, j1;
    double wd;
    const float lr = __logf((float)r);
    locate(G.rn, G.irn, G.Nr + 1, rn_c, (lr - G.lr0) * G.ilr, i0, wd);
    locate(G.rh, G.irh, G.Nr, rh_c, (lr - G.lrh0) * G.ilr, i1, wd);
    locate(G.tn, G.itn, G.Nth + 1, tn_c, ((float)t - G.t0) * G.it, j0, wd);
    locate(G.th, G.ith, G.Nth, th_c, ((float)t - G.th0) * G.it, j1, wd);
    // sin/cos at the clamped th (the particle's own unless clamped at an edge)
    double stn = s, ctn = c, sth = s, cth = c;
    if (tn_c != t) sincos(tn_c, &stn, &ctn);
    if (th_c != t) sincos(th_c, &sth, &cth);
    const double* sn = k.trig;
    const double* cn = k.trig + (G.Nth + 1);
    const double* sh = k.trig + 2 * (G.Nth + 1);
    const double* ch = sh + G.Nth;
    const double third = 1.0 / 3.0;
    double sy[7], cy[7], V[4], col[7], row[7];
    const long long n = k.n_alive;
    // the split column / row are shared between the sub-grids unless clamped
    const bool share = (rn_c == rh_c) && (tn_c == th_c);
    // (i, j): rho and j^ph
    const double y0 = G.tn[j0], y1 = G.tn[j0 + 1];
    double hc = (tn_c - y0) * third, hd = (y1 - tn_c) * third;
    theta_lattice(hc, hd, sn[j0], cn[j0], stn, ctn, sn[j0 + 1], cn[j0 + 1], sy, cy);
    subvolumes(k.bh, G.rn[i0], G.rn[i0 + 1], rn_c, hc, hd, sy, cy, V, col, row);
    double iV = rcp_nr(V[0] + V[1] + V[2] + V[3]);
    // share of node (i+a, j+b) = V(opposite corner) / V
    const double w00 = V[3] * iV, w10 = V[2] * iV, w01 = V[1] * iV, w11 = V[0] * iV;
    k.rec[0 * n + p] = Q * w00; k.rec[1 * n + p] = Q * w10; k.rec[2 * n + p] = Q * w01; k.rec[3 * n + p] = Q * w11;
    const double Qp = Q * vp;
    k.rec[4 * n + p] = Qp * w00; k.rec[5 * n + p] = Qp * w10; k.rec[6 * n + p] = Qp * w01; k.rec[7 * n + p] = Qp * w11;
    // (i+1/2, j): j^r  (same th lattice)
    {
        double row_rh[7];   // this lattice's split row (r columns of the half grid): not shared
        if (share) subvolumes<true, false>(k.bh, G.rh[i1], G.rh[i1 + 1], rh_c, hc, hd, sy, cy, V, col, row_rh);
        else subvolumes(k.bh, G.rh[i1], G.rh[i1 + 1], rh_c, hc, hd, sy, cy, V, col, row_rh);
    }
    iV = rcp_nr(V[0] + V[1] + V[2] + V[3]);
    const double Qr = Q * vr;
    k.rec[8 * n + p] = Qr * (V[3] * iV); k.rec[9 * n + p] = Qr * (V[2] * iV);
    k.rec[10 * n + p] = Qr * (V[1] * iV); k.rec[11 * n + p] = Qr * (V[0] * iV);
    // (i, j+1/2): j^th
    const double z0 = G.th[j1], z1 = G.th[j1 + 1];
    hc = (th_c - z0) * third;
    hd = (z1 - th_c) * third;
    theta_lattice(hc, hd, sh[j1], ch[j1], sth, cth, sh[j1 + 1], ch[j1 + 1], sy, cy);
    if (share) subvolumes<false, true>(k.bh, G.rn[i0], G.rn[i0 + 1], rn_c, hc, hd, sy, cy, V, col, row);
    else subvolumes(k.bh, G.rn[i0], G.rn[i0 + 1], rn_c, hc, hd, sy, cy, V, col, row);
    iV = rcp_nr(V[0] + V[1] + V[2] + V[3]);
    const double Qt = Q * vt;
    k.rec[12 * n + p] = Qt * (V[3] * iV); k.rec[13 * n + p] = Qt * (V[2] * iV);
    k.rec[14 * n + p] = Qt * (V[1] * iV); k.rec[15 * n + p] = Qt * (V[0] * iV);
    k.code[p] = (uint32_t)(i1 - i0 + 1) | ((uint32_t)(j1 - j0 + 1) << 2);
}

// x clamped to [lo, hi] by integer compares of the order-preserving keys:
// the value the FP64 compares give for non-NaN x (a -0 below lo = +0 comes
// back as +0), without FP64-pipe instructions.
__device__ __forceinline__ double clamp_key(double x, double lo, double hi)
{
    const long long kx = okey(x);
    return kx < okey(lo) ? lo : (kx > okey(hi) ? hi : x);
}

__device__ __forceinline__ bool same_bits(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// The deposit's per-particle pass: the sin/cos of the lattices' split
// points (angle addition from the node tables by the in-cell offset), the
// three sub-grid lattices, their subvolumes, weights and the charge products
// in paired FP32; FP64 keeps the particle's sin/cos th and FIDO velocity,
// the node-coordinate differences (the step sizes) and the final sum of
// each share's two floats.
__global__ void __launch_bounds__(256) k_dep_particle_ff(DepK k)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= k.n_alive) return;
    const GridDev& G = k.G;
    const BHff& bh = k.bhf;
    const double r = k.r[p], t = k.th[p];
    // clamped positions and cells on the integer and half node lists
    const double rn_c = clamp_key(r, G.rn[0], G.rn[G.Nr]), rh_c = clamp_key(r, G.rh[0], G.rh[G.Nr - 1]);
    const double tn_c = clamp_key(t, G.tn[0], G.tn[G.Nth]), th_c = clamp_key(t, G.th[0], G.th[G.Nth - 1]);
    int i0, i1, j0, j1;
    double wd;
    const float lr = __logf(f32_est(r)), tf = f32_est(t);
    locate(G.rn, G.irn, G.Nr + 1, rn_c, (lr - G.lr0) * G.ilr, i0, wd);
    locate(G.rh, G.irh, G.Nr, rh_c, (lr - G.lrh0) * G.ilr, i1, wd);
    locate(G.tn, G.itn, G.Nth + 1, tn_c, (tf - G.t0) * G.it, j0, wd);
    locate(G.th, G.ith, G.Nth, th_c, (tf - G.th0) * G.it, j1, wd);
    const double* sn = k.trig;
    const double* cn = k.trig + (G.Nth + 1);
    const double* sh = k.trig + 2 * (G.Nth + 1);
    const double* ch = sh + G.Nth;
    // sin/cos th of the particle in FP64 by angle addition from a node of
    // its cell: the lower node where cos >= 0, the upper one elsewhere, so
    // that sin(x + d) = sin x + (sin x (cos d - 1) + cos x sin d) adds terms
    // of one sign and sin th keeps its relative accuracy up to the poles
    // (g^pp = 1 / (rho^2 sin^2 th) in the velocity needs it); the offset's
    // sin / cos - 1 by the series (libm beyond a cell: a clamped th).
    const int jn = j0 + (__double2hiint(cn[j0]) < 0 ? 1 : 0);
    double s, c;
    {
        double sd, cm;
        sincos_step(t - G.tn[jn], sd, cm);
        s = fma(sn[jn], cm, fma(cn[jn], sd, sn[jn]));
        c = fma(cn[jn], cm, fma(-sn[jn], sd, cn[jn]));
    }
    // ... and at the split points of the two th lattices in paired FP32 (the
    // integer lattice's is the particle's own th unless clamped)
    ff stn, ctn, sth, cth;
    if (same_bits(tn_c, t)) {
        stn = ff_from(s);
        ctn = ff_from(c);
    } else {
        sincos_from_node(sn[jn], cn[jn], tn_c - G.tn[jn], stn, ctn);
    }
    sincos_from_node(sh[j1], ch[j1], th_c - G.th[j1], sth, cth);
    // FIDO three-velocity v^i = gamma^ij u_j / Gamma, in FP64 (the 1/sin^2 th
    // of g^pp and the cancellation between the two terms of U^r and U^ph
    // want more than paired FP32's 46 bits)
    Geo g;
    geo_eval(k.bh, r, s, c, g);
    const double ur = k.ur[p], ut = k.uth[p], up = k.uph[p];
    const double Ur = fma(g.gurr, ur, g.gurp * up), Ut = g.gutt * ut, Up = fma(g.gurp, ur, g.gupp * up);
    const double Qd = k.w[p] * k.qm[p];
    const double QiG = Qd * rsqrt_nr(fma(ur, Ur, fma(ut, Ut, fma(up, Up, 1.0))));
    const ff Q = ff_from(Qd), Qr = ff_from(QiG * Ur), Qt = ff_from(QiG * Ut), Qp = ff_from(QiG * Up);
    const long long n = k.n_alive;
    // the split column / row are shared between the sub-grids unless clamped
    const bool share = same_bits(rn_c, rh_c) && same_bits(tn_c, th_c);
    ff sy[7], cy[7], col[7], row[7];
    ff hc = ff_of(0.f), hd = ff_of(0.f);
    // sub-grid 0: (i, j), rho and j^ph; 1: (i+1/2, j), j^r (the th lattice of
    // 0); 2: (i, j+1/2), j^th.  One copy of the lattice code serves all three.
#pragma unroll 1
    for (int sg = 0; sg < 3; ++sg) {
        if (sg != 1) {
            const bool hth = sg == 2;
            const int jj = hth ? j1 : j0;
            const double* Y = hth ? G.th : G.tn;
            const double* sY = hth ? sh : sn;
            const double* cY = hth ? ch : cn;
            const double tc = hth ? th_c : tn_c;
            hc = ff_mul(ff_from(tc - Y[jj]), bh.third);
            hd = ff_mul(ff_from(Y[jj + 1] - tc), bh.third);
            theta_lattice_ff(hc, hd, ff_from(sY[jj]), ff_from(cY[jj]), hth ? sth : stn, hth ? cth : ctn,
                             ff_from(sY[jj + 1]), ff_from(cY[jj + 1]), sy, cy);
        }
        const bool hr = sg == 1;
        const double x0 = hr ? G.rh[i1] : G.rn[i0], x1 = hr ? G.rh[i1 + 1] : G.rn[i0 + 1];
        const double rc = hr ? rh_c : rn_c;
        const ff ha = ff_mul(ff_from(rc - x0), bh.third), hb = ff_mul(ff_from(x1 - rc), bh.third);
        ff V[4];
        subvolumes_ff(bh, ff_from(x0), ff_from(rc), ha, hb, hc, hd, sy, cy, V, col, row, share && sg == 1,
                      share && sg == 2, sg == 0);
        const ff iV = ff_rcp(ff_add(ff_add(V[0], V[1]), ff_add(V[2], V[3])));
        // share of node (i+a, j+b) = V(opposite corner) / V
        const ff w00 = ff_mul(V[3], iV), w10 = ff_mul(V[2], iV), w01 = ff_mul(V[1], iV), w11 = ff_mul(V[0], iV);
        const int b = sg == 0 ? 0 : 4 + 4 * sg;
        const ff Qs = sg == 0 ? Q : (sg == 1 ? Qr : Qt);
        k.rec[(b + 0) * n + p] = ff_to(ff_mul(Qs, w00)); k.rec[(b + 1) * n + p] = ff_to(ff_mul(Qs, w10));
        k.rec[(b + 2) * n + p] = ff_to(ff_mul(Qs, w01)); k.rec[(b + 3) * n + p] = ff_to(ff_mul(Qs, w11));
        if (sg == 0) {
            k.rec[4 * n + p] = ff_to(ff_mul(Qp, w00)); k.rec[5 * n + p] = ff_to(ff_mul(Qp, w10));
            k.rec[6 * n + p] = ff_to(ff_mul(Qp, w01)); k.rec[7 * n + p] = ff_to(ff_mul(Qp, w11));
        }
    }
    k.code[p] = (uint32_t)(i1 - i0 + 1) | ((uint32_t)(j1 - j0 + 1) << 2);
}

// Slots of a cell (i0, j0): rho[a + 2b] (0..3), j^ph[a + 2b] (4..7),
// j^r[k + 3b] at half-r node i0 - 1 + k (8..13), j^th[a + 2k] at half-th
// node j0 - 1 + k (14..19).  A particle with offsets (ko, kt) (each 0 or 1)
// puts record rows 0..7 in slots 0..7, rows 8 + 2b and 9 + 2b in slots
// 8 + 3b + ko and 9 + 3b + ko, rows 12 + a and 14 + a in slots 14 + a + 2 kt
// and 16 + a + 2 kt.
//
// One warp per cell, its particles 32 at a time: every lane loads one
// particle's 16 shares and code (coalesced, no load depending on another)
// into shared memory; then lane l sums record row l / 2 over the group's
// particles of parity l & 1, into one of two accumulators chosen by the
// particle's offset bit (ko for the j^r rows, kt for the j^th rows, none
// for rows 0..7): 16 FP64 additions per particle, each lane busy.  The
// accumulator is chosen by integer selects, so each addition is one FP64
// instruction.  At the end the two parities are added and lane q < 20
// assembles slot q from at most two (row, accumulator) pairs.  Every
// addition has a fixed order: bitwise reproducible.
constexpr int DEP_CELL_WARPS = 8, DEP_CELL_LD = 33;   // row stride 33: conflict-free shared-memory columns

__device__ __forceinline__ double sel_bits(bool p, double a, double b)
{
    double r;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\tselp.b64 %0, %1, %2, q;\n\t}"
        : "=d"(r) : "d"(a), "d"(b), "r"((unsigned)p));
    return r;
}

__global__ void __launch_bounds__(32 * DEP_CELL_WARPS) k_dep_cell(const double* __restrict__ rec,
                                                                   const uint32_t* __restrict__ code,
                                                                   const uint32_t* __restrict__ off,
                                                                   double* __restrict__ part, long long n, uint32_t C)
{
    __shared__ double sv[DEP_CELL_WARPS][16 * DEP_CELL_LD];
    __shared__ uint32_t sc[DEP_CELL_WARPS][32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long cell = blockIdx.x * (long long)DEP_CELL_WARPS + wid;
    if (cell >= C) return;                  // whole warps: one cell per warp
    double* v = sv[wid];
    uint32_t* cw = sc[wid];
    const uint32_t b0 = off[cell], b1 = off[cell + 1];
    const int row = lane >> 1, par = lane & 1;
    const int bsh = row >= 12 ? 2 : 0;      // the offset bit this row splits on
    const uint32_t bmask = row >= 8 ? 1u : 0u;
    double acc0 = 0.0, acc1 = 0.0;
    for (uint32_t base = b0; base < b1; base += 32) {
        const uint32_t cnt = min(32u, b1 - base);
        const bool live = (uint32_t)lane < cnt;
        const size_t a = (size_t)base + lane;
        double x[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = live ? __ldg(rec + (size_t)q * n + a) : 0.0;
        const uint32_t cd = live ? __ldg(code + a) : 0u;
        __syncwarp();                       // the previous group's reads are done
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q * DEP_CELL_LD + lane] = x[q];
        cw[lane] = cd;
        __syncwarp();
        const int kend = (int)(cnt + 1) >> 1;
        for (int k = 0; k < kend; ++k) {
            const int pp = 2 * k + par;     // a particle past the group's end holds zeros
            const double y = v[row * DEP_CELL_LD + pp];
            const bool bit = ((cw[pp] >> bsh) & bmask) != 0u;
            const double s = sel_bits(bit, acc1, acc0) + y;
            acc1 = sel_bits(bit, s, acc1);
            acc0 = sel_bits(bit, acc0, s);
        }
    }
    acc0 += __shfl_xor_sync(0xffffffffu, acc0, 1);
    acc1 += __shfl_xor_sync(0xffffffffu, acc1, 1);
    // slot q = lane: rows ra (accumulator ua) and rb (accumulator 0, if any)
    int ra = lane, rb = -1;
    bool ua = false;
    if (lane >= 8 && lane < 14) {
        const int b = (lane - 8) / 3, kk = (lane - 8) % 3;
        ra = kk == 2 ? 9 + 2 * b : 8 + 2 * b;
        ua = kk != 0;
        rb = kk == 1 ? 9 + 2 * b : -1;
    } else if (lane >= 14 && lane < 20) {
        const int aa = (lane - 14) & 1, kk = (lane - 14) >> 1;
        ra = kk == 2 ? 14 + aa : 12 + aa;
        ua = kk != 0;
        rb = kk == 1 ? 14 + aa : -1;
    }
    const int la = 2 * (ra & 15), lb = 2 * (rb & 15);
    const double xa0 = __shfl_sync(0xffffffffu, acc0, la), xa1 = __shfl_sync(0xffffffffu, acc1, la);
    const double xb0 = __shfl_sync(0xffffffffu, acc0, lb);
    if (lane < 20) part[(size_t)lane * C + cell] = (ua ? xa1 : xa0) + (rb >= 0 ? xb0 : 0.0);
}

struct NodeK {
    int Nr, Nth, ld;
    const double* part;
    uint32_t C;
    Tabs T;
    double *rho, *jr, *jt, *jp;
};

__global__ void k_dep_node(NodeK k)
{
    const int i = blockIdx.y;
    const int Nr = k.Nr, Nth = k.Nth;
    auto P = [&](int q, int ci, int cj) -> double {
        return k.part[(size_t)q * k.C + (size_t)ci * Nth + cj];
    };
    for (int j = threadIdx.x; j <= Nth; j += blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        // rho, j^ph at (i, j): cells (i - a, j - b), slot a + 2b
        double sr = 0.0, sp = 0.0;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int ci = i - a, cj = j - b;
                if (ci < 0 || ci >= Nr || cj < 0 || cj >= Nth) continue;
                sr += P(a + 2 * b, ci, cj);
                sp += P(4 + a + 2 * b, ci, cj);
            }
        k.rho[o] = sr / k.T.dual(0, i, j);
        k.jp[o] = sp / k.T.dual(0, i, j);
        // j^r at (i+1/2, j): cells (i + 1 - kk, j - b), slot kk + 3b
        if (i < Nr) {
            double sj = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int kk = 0; kk < 3; ++kk) {
                    const int ci = i + 1 - kk, cj = j - b;
                    if (ci < 0 || ci >= Nr || cj < 0 || cj >= Nth) continue;
                    sj += P(8 + kk + 3 * b, ci, cj);
                }
            k.jr[o] = sj / k.T.dual(1, i, j);
        }
        // j^th at (i, j+1/2): cells (i - a, j + 1 - kk), slot a + 2 kk
        if (j < Nth) {
            double sj = 0.0;
            for (int kk = 0; kk < 3; ++kk)
                for (int a = 0; a < 2; ++a) {
                    const int ci = i - a, cj = j + 1 - kk;
                    if (ci < 0 || ci >= Nr || cj < 0 || cj >= Nth) continue;
                    sj += P(14 + a + 2 * kk, ci, cj);
                }
            k.jt[o] = sj / k.T.dual(2, i, j);
        }
    }
}

// ---------------------------------------------------------------------------
// FDTD (Sec. 2.1, Eqs. m3, m4, Ei; Sec. 2.5)
// ---------------------------------------------------------------------------
struct FK {
    int Nr, Nth, ld;
    GridDev G;
    Tabs T;
    double dt, chi0, lam, r_abs, r_max;
    int conserving;     // sources are coordinate currents J (fpic_deposit_conserving)
};

__device__ __forceinline__ double damp(const FK& k, double r)
{
    if (k.chi0 <= 0.0 || r <= k.r_abs) return 1.0;
    const double x = (r - k.r_abs) / (k.r_max - k.r_abs);
    return exp(-k.chi0 * pow(x, k.lam) * k.dt);
}

// metric-weighted average of F (staggering ro, to) to the point of the other
// r staggering at index i2 (zero-gradient beyond the ends)
__device__ __forceinline__ double avg_r(const FK& k, const double* F, int ro, int to, int i2, int j)
{
    int ia = ro ? i2 - 1 : i2, ib = ro ? i2 : i2 + 1;
    const int m = ro ? k.Nr : k.Nr + 1;
    if (ia < 0) ia = ib;
    if (ib > m - 1) ib = ia;
    const int tF = (ro ? 1 : 0) | (to ? 2 : 0), tT = (ro ? 0 : 1) | (to ? 2 : 0);
    const double sa = k.T.at(tF, 2, ia, j), sb = k.T.at(tF, 2, ib, j), ist = k.T.at(tT, 7, i2, j);
    return fma(sa, F[(size_t)ia * k.ld + j], sb * F[(size_t)ib * k.ld + j]) * (0.5 * ist);
}

struct F3 {
    const double *a[3], *b[3];   // value = b ? 0.5 (a + b) : a  (pointwise level average)
    __device__ __forceinline__ double v(int c, size_t o) const
    {
        return b[c] ? 0.5 * (a[c][o] + b[c][o]) : a[c][o];
    }
};

struct O3 {
    double* p[3];
};

__global__ void k_avg3(F3 in, O3 out, size_t sz)
{
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < sz; o += (size_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) out.p[c][o] = in.v(c, o);
}

// Eq. (Ei): E_r (i+1/2,j) = alpha (g_rr D^r + g_rp <D^ph>);
// E_th (i,j+1/2) = alpha g_tt D^th - sqrtg beta <B^ph>;
// E_ph (i,j) = alpha (g_rp <D^r> + g_pp D^ph) + sqrtg beta <B^th>.
// Full-theta domain (Sec. 2.5, periodic in th): columns 0..Nth-1 are the
// distinct points; the thread of column 0 also stores its values in column
// Nth, the image the seam's stencils and the push's gather read.
__device__ __forceinline__ void put(double* F, size_t o, int j, const FK& k, double v)
{
    F[o] = v;
    if (k.G.full && j == 0) F[o + k.Nth] = v;
}

__global__ void k_make_E(FK k, F3 D, F3 B, O3 E)
{
    const int i = blockIdx.y;
    const int jend = k.G.full ? k.Nth - 1 : k.Nth;
    for (int j = threadIdx.x; j <= jend; j += blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        if (i < k.Nr) {
            const double Dp = avg_r(k, D.a[2], 0, 0, i, j);
            put(E.p[0], o, j, k, k.T.at(1, 0, i, j) * fma(k.T.at(1, 3, i, j), D.a[0][o], k.T.at(1, 4, i, j) * Dp));
        }
        if (j < k.Nth) {
            const double Bp = avg_r(k, B.a[2], 1, 1, i, j);
            put(E.p[1], o, j, k, fma(k.T.at(2, 0, i, j) * k.T.at(2, 5, i, j), D.a[1][o],
                                     -k.T.at(2, 2, i, j) * k.T.at(2, 1, i, j) * Bp));
        }
        const double Dr = avg_r(k, D.a[0], 1, 0, i, j);
        const double Bt = avg_r(k, B.a[1], 1, 0, i, j);
        put(E.p[2], o, j, k, fma(k.T.at(0, 0, i, j), fma(k.T.at(0, 4, i, j), Dr, k.T.at(0, 6, i, j) * D.a[2][o]),
                                 k.T.at(0, 2, i, j) * k.T.at(0, 1, i, j) * Bt));
    }
}

// H_r (i,j+1/2) = alpha (g_rr B^r + g_rp <B^ph>);  H_th (i+1/2,j) = alpha g_tt
// B^th + sqrtg beta <D^ph>;  H_ph (i+1/2,j+1/2) = alpha (g_rp <B^r> + g_pp B^ph)
// - sqrtg beta <D^th>.
__global__ void k_make_H(FK k, F3 D, F3 B, O3 H)
{
    const int i = blockIdx.y;
    const int jend = k.G.full ? k.Nth - 1 : k.Nth;
    for (int j = threadIdx.x; j <= jend; j += blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        if (j < k.Nth) {
            const double Bp = avg_r(k, B.a[2], 1, 1, i, j);
            put(H.p[0], o, j, k, k.T.at(2, 0, i, j) * fma(k.T.at(2, 3, i, j), B.a[0][o], k.T.at(2, 4, i, j) * Bp));
        }
        if (i < k.Nr) {
            const double Dp = avg_r(k, D.a[2], 0, 0, i, j);
            put(H.p[1], o, j, k, fma(k.T.at(1, 0, i, j) * k.T.at(1, 5, i, j), B.a[1][o],
                                     k.T.at(1, 2, i, j) * k.T.at(1, 1, i, j) * Dp));
        }
        if (i < k.Nr && j < k.Nth) {
            const double Br = avg_r(k, B.a[0], 0, 1, i, j);
            const double Dt = avg_r(k, D.a[1], 0, 1, i, j);
            put(H.p[2], o, j, k, fma(k.T.at(3, 0, i, j), fma(k.T.at(3, 4, i, j), Br, k.T.at(3, 6, i, j) * B.a[2][o]),
                                     -k.T.at(3, 2, i, j) * k.T.at(3, 1, i, j) * Dt));
        }
    }
}

// Eq. (m4) + (abs0): B_out = (B_in - dt curl E / sqrtg) exp(-chi dt).
// The forward th differences at j = Nth-1 read column Nth: the image of
// column 0 in the full-theta domain.
__global__ void k_update_B(FK k, F3 Bin, O3 E, O3 Bout)
{
    const int i = blockIdx.y;
    const GridDev& G = k.G;
    const int jend = G.full ? k.Nth - 1 : k.Nth;
    // the damping factor depends on the row only; 1/dr of the row
    const double dn = damp(k, G.rn[i]), dh = i < k.Nr ? damp(k, G.rh[i]) : 1.0;
    const double idr = i < k.Nr ? G.irn[i] : 0.0;
    for (int j = threadIdx.x; j <= jend; j += blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        if (j < k.Nth) {   // B^r (i, j+1/2)
            const double curl = (E.p[2][o + 1] - E.p[2][o]) * G.itn[j];
            put(Bout.p[0], o, j, k, (Bin.v(0, o) - k.dt * curl * k.T.at(2, 7, i, j)) * dn);
        }
        if (i < k.Nr) {    // B^th (i+1/2, j)
            const double curl = -(E.p[2][o + k.ld] - E.p[2][o]) * idr;
            put(Bout.p[1], o, j, k, (Bin.v(1, o) - k.dt * curl * k.T.at(1, 7, i, j)) * dh);
        }
        if (i < k.Nr && j < k.Nth) {   // B^ph (i+1/2, j+1/2)
            const double dEt = (E.p[1][o + k.ld] - E.p[1][o]) * idr;
            const double dEr = (E.p[0][o + 1] - E.p[0][o]) * G.itn[j];
            put(Bout.p[2], o, j, k, (Bin.v(2, o) - k.dt * (dEt - dEr) * k.T.at(3, 7, i, j)) * dh);
        }
    }
}

struct Src {
    const double *j[3], *rho;
    double w;
};

// J = alpha j - rho beta at the J^k point (rho averaged to J^r's point)
__device__ __forceinline__ double jsrc(const FK& k, const Src& S, int comp, int i, int j)
{
    if (S.w == 0.0) return 0.0;
    const size_t o = (size_t)i * k.ld + j;
    if (k.conserving) return S.w * S.j[comp][o];
    if (comp == 0) {
        const double rb = avg_r(k, S.rho, 0, 0, i, j);
        return S.w * fma(k.T.at(1, 0, i, j), S.j[0][o], -rb * k.T.at(1, 1, i, j));
    }
    if (comp == 1) return S.w * (k.T.at(2, 0, i, j) * S.j[1][o]);
    return S.w * (k.T.at(0, 0, i, j) * S.j[2][o]);
}

// Eq. (m3) + (abs1): D_out = (D_in + dt [curl H / sqrtg - 4 pi J]) exp(-chi dt),
// interior points only (boundaries: k_bc_D).  Full-theta domain: D^r and D^ph
// at j = 0 too, their backward th difference across the seam (half node
// Nth-1, one period below: spacing th[Nth] - th[Nth-1], th[Nth] = th[0] + P).
__global__ void k_update_D(FK k, F3 Din, O3 H, Src S0, Src S1, O3 Dout)
{
    const int i = blockIdx.y;
    const GridDev& G = k.G;
    const double fpi = 4.0 * M_PI;
    const int jlo = G.full ? 0 : 1;
    // the damping factor depends on the row only; 1/dr of the row
    const double dn = damp(k, G.rn[i]), dh = i < k.Nr ? damp(k, G.rh[i]) : 1.0;
    const double idr = (i >= 1 && i < k.Nr) ? G.irh[i - 1] : 0.0;
    for (int j = threadIdx.x; j < k.Nth; j += blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        const size_t om = j > 0 ? o - 1 : o + (k.Nth - 1);
        const double idth = G.ith[j > 0 ? j - 1 : k.Nth - 1];     // 1/(th[j] - th[j-1]), across the seam at j = 0
        if (i < k.Nr && j >= jlo) {    // D^r (i+1/2, j)
            const double curl = (H.p[2][o] - H.p[2][om]) * idth;
            const double J = jsrc(k, S0, 0, i, j) + jsrc(k, S1, 0, i, j);
            put(Dout.p[0], o, j, k, (Din.v(0, o) + k.dt * fma(curl, k.T.at(1, 7, i, j), -fpi * J)) * dh);
        }
        if (i >= 1 && i < k.Nr) {    // D^th (i, j+1/2)
            const double curl = -(H.p[2][o] - H.p[2][o - k.ld]) * idr;
            const double J = jsrc(k, S0, 1, i, j) + jsrc(k, S1, 1, i, j);
            put(Dout.p[1], o, j, k, (Din.v(1, o) + k.dt * fma(curl, k.T.at(2, 7, i, j), -fpi * J)) * dn);
        }
        if (i >= 1 && i < k.Nr && j >= jlo) {   // D^ph (i, j)
            const double dHt = (H.p[1][o] - H.p[1][o - k.ld]) * idr;
            const double dHr = (H.p[0][o] - H.p[0][om]) * idth;
            const double J = jsrc(k, S0, 2, i, j) + jsrc(k, S1, 2, i, j);
            put(Dout.p[2], o, j, k, (Din.v(2, o) + k.dt * fma(dHt - dHr, k.T.at(0, 7, i, j), -fpi * J)) * dn);
        }
    }
}

// Sec. 2.5 (reading): zero gradient where a stencil is one-sided, D^ph = 0 on
// the axis rows (k_axis_D).  Full-theta domain: no th boundary; the radial
// boundary rows copy every column, the image column Nth included.
__global__ void k_bc_D(FK k, O3 D)
{
    const int i = blockIdx.y;
    const int Nr = k.Nr, Nth = k.Nth, ld = k.ld;
    const bool full = k.G.full;
    if (threadIdx.x == 0 && !full) {
        if (i < Nr) {
            D.p[0][(size_t)i * ld + 0] = D.p[0][(size_t)i * ld + 1];
            D.p[0][(size_t)i * ld + Nth] = D.p[0][(size_t)i * ld + Nth - 1];
        }
    }
    const int jt = full ? Nth : Nth - 1, jp0 = full ? 0 : 1, jp1 = full ? Nth : Nth - 1;
    for (int j = threadIdx.x; j <= Nth; j += blockDim.x) {
        if (i == 0 && j <= jt) D.p[1][j] = D.p[1][(size_t)ld + j];
        if (i == Nr && j <= jt) D.p[1][(size_t)Nr * ld + j] = D.p[1][(size_t)(Nr - 1) * ld + j];
        if (i == 0 && j >= jp0 && j <= jp1) D.p[2][j] = D.p[2][(size_t)ld + j];
        if (i == Nr && j >= jp0 && j <= jp1) D.p[2][(size_t)Nr * ld + j] = D.p[2][(size_t)(Nr - 1) * ld + j];
    }
}

__global__ void k_axis_D(FK k, O3 D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= k.Nr) {
        D.p[2][(size_t)i * k.ld + 0] = 0.0;
        D.p[2][(size_t)i * k.ld + k.Nth] = 0.0;
    }
}

}  // namespace fpic

using namespace fpic;

static Tabs tabs_of(const fpic_ctx* c)
{
    return Tabs{c->d_metric, c->metric_stride, c->ld};
}

extern "C" int fpic_sort(fpic_ctx* c, fpic_particles* p, void* stream)
{
    if (!c || !p) return set_error(FPIC_EINVAL, "fpic_sort: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_sort: no grid set");
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_sort: n out of range");
    if (p->n == 0) return FPIC_OK;
    if (!particles_ok(p, true) || !p->w) return set_error(FPIC_EINVAL, "fpic_sort: NULL particle array");
    FPIC_CUDA(cudaSetDevice(c->device));
    Work w;
    int rc = work_layout(c, p->n, false, w);
    if (rc) return rc;
    return sort_impl(c, p, w, (cudaStream_t)stream);
}

namespace fpic {
static ff ff_host(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

static BHff bh_ff(const BH& bh)
{
    return {ff_host(bh.twoM), ff_host(bh.a2), ff_host(1.0 / 3.0)};
}
}  // namespace fpic

extern "C" int fpic_deposit(fpic_ctx* c, fpic_particles* p, double* rho, double* jr, double* jth, double* jph,
                            void* stream)
{
    if (c && c->G.full) return set_error(FPIC_EINVAL, "fpic_deposit: not built for the full-theta domain");
    if (!c || !p || !rho || !jr || !jth || !jph) return set_error(FPIC_EINVAL, "fpic_deposit: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_deposit: no grid set");
    if (p->n < 0 || p->n >= (1LL << 31)) return set_error(FPIC_EINVAL, "fpic_deposit: n out of range");
    if (p->n > 0 && (!particles_ok(p, true) || !p->w)) return set_error(FPIC_EINVAL, "fpic_deposit: NULL particle array");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = p->n;
    const uint32_t C = (uint32_t)c->Nr * (uint32_t)c->Nth;
    Work w;
    int rc = work_layout(c, n > 0 ? n : 1, true, w);
    if (rc) return rc;
    if (n > 0) {
        rc = sort_impl(c, p, w, s, w.rec);
        if (rc) return rc;
    } else {
        FPIC_CUDA(cudaMemsetAsync(w.off, 0, 4 * ((size_t)C + 2), s));
    }
    // alive particles occupy [0, off[C]) after the sort; the count is read on the device
    DepK k{c->bh, bh_ff(c->bh), c->G, c->d_metric + (size_t)MT_N * c->metric_stride, p->r, p->th, p->ur, p->uth, p->uph, p->qm, p->w, n, w.rec, w.code};
    if (n > 0) {
        // rec/code for all n slots; removed particles (past off[C]) are never summed
        const int dt_ = c->dep_threads;
        const unsigned nb = (unsigned)((n + dt_ - 1) / dt_);
        if (c->dep_lattice) k_dep_particle_ff<<<nb, dt_, 0, s>>>(k);
        else k_dep_particle<<<nb, dt_, 0, s>>>(k);
    }
    k_dep_cell<<<(unsigned)(((long long)C + DEP_CELL_WARPS - 1) / DEP_CELL_WARPS), 32 * DEP_CELL_WARPS, 0, s>>>(
        w.rec, w.code, w.off, w.part, n > 0 ? n : 1, C);
    NodeK nk{c->Nr, c->Nth, c->ld, w.part, C, tabs_of(c), rho, jr, jth, jph};
    k_dep_node<<<dim3(1, c->Nr + 1), 256, 0, s>>>(nk);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

namespace fpic {
// ---------------------------------------------------------------------------
// Charge-conserving deposit (an extension; the paper's deposit is not and
// relies on the cleaning of Sec. 2.4)
// ---------------------------------------------------------------------------
// A move from x^n to x^{n+1} with linear (area) node weights S = S_r S_th,
// split Esirkepov's way on the 3 x 3 window of integer nodes spanned by the
// two stencils: W_r = dS_r <S_th>, W_th = <S_r> dS_th (<.> the mean of old
// and new), charge crossing the dual face between window nodes x and x+1 in
// +r: -Q sum_{x' <= x} W_r(x', y) (alike in th).  Window partials (30 per
// particle: Q S^new and Q <S> (dph/dt)_mid on 3 x 3 nodes, 2 x 3 r faces,
// 3 x 2 th faces) are summed per window-base cell by one warp over the cell's
// particles in index order (fixed shuffle tree), then gathered per node /
// face in a fixed order: bitwise reproducible.  Normalised by the Yee cell
// (2 pi sqrtg dr_dual dth_dual) so that sqrtg (rho^{n+1} - rho^n) + dt
// Yee-div(sqrtg J) = 0 at every node.
enum { CD_Q = 0, CD_P = 9, CD_R = 18, CD_T = 24, CD_SLOTS = 30 };

struct CDepK {
    int Nr, Nth, ld;
    GridDev G;
    BH bh;
    long long n;
    const double *r0, *t0, *ur0, *ut0, *up0;
    const uint8_t* alive0;
    const double *r1, *t1, *ur1, *ut1, *up1, *qm, *w;
    const double* trig;      // sin tn[0..Nth], then cos tn[0..Nth]
};

__device__ __forceinline__ void cd_lin(const GridDev& G, double r, double t, int& i, double& fr, int& j, double& ft)
{
    const float lr = __logf(f32_est(r));
    locate(G.rn, G.irn, G.Nr + 1, r, (lr - G.lr0) * G.ilr, i, fr);
    locate(G.tn, G.itn, G.Nth + 1, t, (f32_est(t) - G.t0) * G.it, j, ft);
}

// window base cell of each particle alive before the move (C: skipped / removed)
__global__ void k_cdep_keys(CDepK k, uint32_t* key, uint32_t* count, uint32_t C, long long* n_skip)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool valid = p < k.n;
    uint32_t kk = C;
    if (valid && k.alive0[p]) {
        int ia, ja, ib, jb;
        double f;
        cd_lin(k.G, k.r0[p], k.t0[p], ia, f, ja, f);
        cd_lin(k.G, k.r1[p], k.t1[p], ib, f, jb, f);
        if (abs(ia - ib) > 1 || abs(ja - jb) > 1) atomicAdd((unsigned long long*)n_skip, 1ull);
        else kk = (uint32_t)min(ia, ib) * (uint32_t)k.Nth + (uint32_t)min(ja, jb);
    }
    if (valid) key[p] = kk;
    count_key(count, kk, valid);
}

// coordinate dph/dt = alpha gamma^{ph j} u_j / Gamma.  sin/cos th by angle
// addition from the tabulated node tn[j] of the particle's cell (the step
// t - tn[j] is under a cell, so its sin / cos - 1 come from the series), and
// 1/Gamma as one reciprocal square root.
__device__ __forceinline__ double cd_phdot(const BH& bh, const GridDev& G, const double* trig, int j, double r,
                                           double t, double ur, double ut, double up)
{
    double sh, cm;
    sincos_step(t - G.tn[j], sh, cm);
    const double s0 = trig[j], c0 = trig[G.Nth + 1 + j];
    const double s = fma(s0, cm, fma(c0, sh, s0)), c = fma(c0, cm, fma(-s0, sh, c0));
    Geo g;
    geo_eval(bh, r, s, c, g);
    const double iG = rsqrt_nr(fma(g.gurr * ur, ur, fma(2.0 * g.gurp * ur, up, fma(g.gutt * ut, ut, fma(g.gupp * up, up, 1.0)))));
    return g.alpha * fma(g.gurp, ur, g.gupp * up) * iG;
}

// one warp per window-base cell: its particles' 30 window partials, summed
__global__ void k_cdep_cell(CDepK k, const uint32_t* __restrict__ off, const uint32_t* __restrict__ perm,
                            double* __restrict__ part, uint32_t C)
{
    const long long cell = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= C) return;
    const uint32_t b0 = off[cell], b1 = off[cell + 1];
    const int i0 = (int)(cell / k.Nth), j0 = (int)(cell - (long long)i0 * k.Nth);
    double acc = 0.0;           // lane q: slot q of the cell (q < CD_SLOTS)
    for (uint32_t base = b0; base < b1; base += 32) {
        double v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = 0.0;
        const uint32_t a = base + lane;
        if (a < b1) {
            const uint32_t p = perm[a];
            int ia, ja, ib, jb;
            double fra, fta, frb, ftb;
            cd_lin(k.G, k.r0[p], k.t0[p], ia, fra, ja, fta);
            cd_lin(k.G, k.r1[p], k.t1[p], ib, frb, jb, ftb);
            // window weights by selects (registers, no indexed local arrays)
            const int da = ia - i0, db = ib - i0, ea = ja - j0, eb = jb - j0;
            double Sra[3], Srb[3], Sta[3], Stb[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                Sra[x] = x == da ? 1.0 - fra : (x == da + 1 ? fra : 0.0);
                Srb[x] = x == db ? 1.0 - frb : (x == db + 1 ? frb : 0.0);
                Sta[x] = x == ea ? 1.0 - fta : (x == ea + 1 ? fta : 0.0);
                Stb[x] = x == eb ? 1.0 - ftb : (x == eb + 1 ? ftb : 0.0);
            }
            const double Q = k.w[p] * k.qm[p];
            const double phd = 0.5 * (cd_phdot(k.bh, k.G, k.trig, ja, k.r0[p], k.t0[p], k.ur0[p], k.ut0[p], k.up0[p]) +
                                      cd_phdot(k.bh, k.G, k.trig, jb, k.r1[p], k.t1[p], k.ur1[p], k.ut1[p], k.up1[p]));
            // factors shared by the slots: Q S_r^{n+1}, Q (dph/dt) / 2, the
            // half differences and sums of the weights
            const double Qh = 0.5 * Q * phd;
            double QSrb[3], dSr[2], aSr[3], dSt[2], sSt[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                QSrb[x] = Q * Srb[x];
                aSr[x] = 0.5 * (Sra[x] + Srb[x]);
                sSt[x] = Sta[x] + Stb[x];
            }
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                dSr[x] = 0.5 * (Srb[x] - Sra[x]);
                dSt[x] = Stb[x] - Sta[x];
            }
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) {
                    v[CD_Q + 3 * x + y] = QSrb[x] * Stb[y];
                    v[CD_P + 3 * x + y] = Qh * fma(Sra[x], Sta[y], Srb[x] * Stb[y]);
                }
#pragma unroll
            for (int y = 0; y < 3; ++y) {
                double s_ = 0.0;
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    s_ = fma(dSr[x], sSt[y], s_);
                    v[CD_R + 3 * x + y] = -Q * s_;
                }
            }
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                double s_ = 0.0;
#pragma unroll
                for (int y = 0; y < 2; ++y) {
                    s_ = fma(aSr[x], dSt[y], s_);
                    v[CD_T + 2 * x + y] = -Q * s_;
                }
            }
        }
        // reduce-scatter across the warp (recursive halving): each step a lane
        // keeps half of its slots and adds its partner's copy of them; after
        // five steps lane q holds the warp's sum of slot q (31 adds per lane)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int q = 0; q < o; ++q) {
                const double send = upper ? v[q] : v[q + o];
                const double keep = upper ? v[q + o] : v[q];
                v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        acc += v[0];
    }
    if (lane < CD_SLOTS) part[(size_t)lane * C + cell] = acc;
}

__device__ __forceinline__ double cd_dual_r(const GridDev& G, int i)
{
    return (i == G.Nr ? G.rn[G.Nr] : G.rh[i]) - (i == 0 ? G.rn[0] : G.rh[i - 1]);
}

__device__ __forceinline__ double cd_dual_t(const GridDev& G, int j)
{
    return (j == G.Nth ? M_PI : G.th[j]) - (j == 0 ? 0.0 : G.th[j - 1]);
}

// per node / face: the partials of the window cells covering it, fixed order
__global__ void k_cdep_node(CDepK k, Tabs T, const double* __restrict__ part, uint32_t C, double dt, double* rho,
                            double* Jr, double* Jt, double* Jp)
{
    const int i = blockIdx.y;
    const GridDev& G = k.G;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= k.Nth; j += gridDim.x * blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        double Q = 0.0, Pp = 0.0, Fr = 0.0, Ft = 0.0;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) {
                const int ci = i - x, cj = j - y;
                if (ci < 0 || ci >= k.Nr || cj < 0 || cj >= k.Nth) continue;
                const size_t cell = (size_t)ci * k.Nth + cj;
                Q += part[(size_t)(CD_Q + 3 * x + y) * C + cell];
                Pp += part[(size_t)(CD_P + 3 * x + y) * C + cell];
                if (x < 2) Fr += part[(size_t)(CD_R + 3 * x + y) * C + cell];
                if (y < 2) Ft += part[(size_t)(CD_T + 2 * x + y) * C + cell];
            }
        const double drd = cd_dual_r(G, i), dtd = cd_dual_t(G, j);
        const double vol = 2.0 * M_PI * T.at(0, 2, i, j) * drd * dtd;
        rho[o] = vol > 0.0 ? Q / vol : 0.0;
        Jp[o] = vol > 0.0 ? Pp / vol : 0.0;
        if (i < k.Nr) Jr[o] = Fr / (dt * 2.0 * M_PI * T.at(1, 2, i, j) * dtd);
        else Jr[o] = 0.0;
        if (j < k.Nth) Jt[o] = Ft / (dt * 2.0 * M_PI * T.at(2, 2, i, j) * drd);
        else Jt[o] = 0.0;
    }
}
}  // namespace fpic

extern "C" int fpic_deposit_conserving(fpic_ctx* c, const fpic_particles* before, const fpic_particles* after,
                                       double dt, double* rho, double* jr, double* jth, double* jph,
                                       long long* n_skipped, void* stream)
{
    if (c && c->G.full) return set_error(FPIC_EINVAL, "fpic_deposit_conserving: not built for the full-theta domain");
    if (!c || !before || !after || !rho || !jr || !jth || !jph)
        return set_error(FPIC_EINVAL, "fpic_deposit_conserving: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_deposit_conserving: no grid set");
    if (before->n != after->n || after->n < 0) return set_error(FPIC_EINVAL, "fpic_deposit_conserving: n mismatch");
    if (!(std::isfinite(dt)) || dt == 0.0) return set_error(FPIC_EINVAL, "fpic_deposit_conserving: dt must be finite and nonzero");
    const long long n = after->n;
    if (n > 0 && (!before->r || !before->th || !before->ur || !before->uth || !before->uph || !before->alive ||
                  !after->r || !after->th || !after->ur || !after->uth || !after->uph || !after->qm || !after->w))
        return set_error(FPIC_EINVAL, "fpic_deposit_conserving: NULL particle array");
    if (n >= (1LL << 32)) return set_error(FPIC_EINVAL, "fpic_deposit_conserving: more than 2^32 particles");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long C = (long long)c->Nr * c->Nth;
    Work w;
    void* part_v = nullptr;     // per-cell window partials, CD_SLOTS x C doubles
    int rc = work_layout(c, n > 0 ? n : 1, false, w, (size_t)CD_SLOTS * C * sizeof(double), &part_v);
    if (rc) return rc;
    double* part = (double*)part_v;
    CDepK k{c->Nr, c->Nth, c->ld, c->G, c->bh, n, before->r, before->th, before->ur, before->uth, before->uph,
            before->alive, after->r, after->th, after->ur, after->uth, after->uph, after->qm, after->w,
            c->d_metric + (size_t)MT_N * c->metric_stride};
    FPIC_CUDA(cudaMemsetAsync(w.count, 0, 4 * ((size_t)C + 2), s));
    FPIC_CUDA(cudaMemsetAsync(w.cursor, 0, 4 * ((size_t)C + 2), s));
    FPIC_CUDA(cudaMemsetAsync(c->d_cnt + CNT_ERR, 0, sizeof(long long), s));
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) k_cdep_keys<<<nb, 256, 0, s>>>(k, w.key, w.count, (uint32_t)C, c->d_cnt + CNT_ERR);
    rc = scan_u32(w.count, w.off, w.bsum, C + 1, s);
    if (rc) return rc;
    if (n > 0) k_scatter<<<nb, 256, 0, s>>>(w.key, w.off, w.cursor, w.perm, n);
    k_bucket_rank<<<(unsigned)((C * 32 + 255) / 256), 256, 0, s>>>(w.off, w.perm, w.perm2, (uint32_t)C);
    k_cdep_cell<<<(unsigned)((C * 32 + 255) / 256), 256, 0, s>>>(k, w.off, w.perm2, part, (uint32_t)C);
    k_cdep_node<<<dim3((unsigned)((c->Nth + 1 + 255) / 256), c->Nr + 1), 256, 0, s>>>(k, tabs_of(c), part,
                                                                                     (uint32_t)C, dt, rho, jr,
                                                                                     jth, jph);
    FPIC_CUDA(cudaGetLastError());
    if (n_skipped) {
        long long v = 0;
        FPIC_CUDA(cudaMemcpyAsync(&v, c->d_cnt + CNT_ERR, sizeof(long long), cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        *n_skipped = v;
    }
    return FPIC_OK;
}

namespace fpic {
// ---------------------------------------------------------------------------
// Divergence cleaning (Sec. 2.4, Eq. phi)
// ---------------------------------------------------------------------------
// (1/sqrtg) d_k (sqrtg gamma^kl d_l phi) = (1/sqrtg) d_j (sqrtg D^j) - 4 pi rho at
// the integer nodes i = 1 .. Nr-1, j = 0 .. Nth, multiplied by sqrtg at the
// node: the left side is the sum over the four faces of sqrtg gamma^kk d_k phi
// differences over the dual widths (the Yee divergence's own fluxes), the
// pole faces carry no flux, phi = 0 on the radial end rows.  Jacobi form
// phi <- sum_f c_f phi_f - b with c_f = face coefficient / sum of the face
// coefficients and b = right side / the same sum, both built once.
struct CleanK {
    int Nr, Nth, ld;
    GridDev G;
    Tabs T;                                  // metric tables at the Yee points
    double *c_r1, *c_r0, *c_t1, *c_t0, *b;   // per node (library scratch)
};

// Inverse spatial metric from the tabulated lower one: the th block is
// diagonal, the (r, ph) block a 2 x 2 inverse.
__device__ __forceinline__ double tab_gu_rr(const Tabs& T, int t, int i, int j)
{
    const double grr = T.at(t, 3, i, j), grp = T.at(t, 4, i, j), gpp = T.at(t, 6, i, j);
    return gpp / fma(grr, gpp, -grp * grp);
}

__device__ __forceinline__ double tab_gu_rp(const Tabs& T, int t, int i, int j)
{
    const double grr = T.at(t, 3, i, j), grp = T.at(t, 4, i, j), gpp = T.at(t, 6, i, j);
    return -grp / fma(grr, gpp, -grp * grp);
}

__global__ void k_clean_setup(CleanK k, const double* __restrict__ Dr, const double* __restrict__ Dt,
                              const double* __restrict__ rho)
{
    const int i = blockIdx.y + 1;                   // 1 .. Nr-1
    const GridDev& G = k.G;
    const Tabs& T = k.T;
    const double dr = G.rh[i] - G.rh[i - 1];
    const double ir1 = 1.0 / ((G.rn[i + 1] - G.rn[i]) * dr), ir0 = 1.0 / ((G.rn[i] - G.rn[i - 1]) * dr);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= k.Nth; j += gridDim.x * blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        const double dth = (j < k.Nth ? G.th[j] : M_PI) - (j > 0 ? G.th[j - 1] : 0.0);
        const double sr1 = T.at(1, 2, i, j), sr0 = T.at(1, 2, i - 1, j);
        const double st1 = j < k.Nth ? T.at(2, 2, i, j) : 0.0, st0 = j > 0 ? T.at(2, 2, i, j - 1) : 0.0;
        const double rhs = (sr1 * Dr[o] - sr0 * Dr[o - k.ld]) / dr +
                           ((j < k.Nth ? st1 * Dt[o] : 0.0) - (j > 0 ? st0 * Dt[o - 1] : 0.0)) / dth -
                           4.0 * M_PI * T.at(0, 2, i, j) * rho[o];
        const double cr1 = sr1 * tab_gu_rr(T, 1, i, j) * ir1;
        const double cr0 = sr0 * tab_gu_rr(T, 1, i - 1, j) * ir0;
        const double ct1 = j < k.Nth ? st1 / (T.at(2, 5, i, j) * (G.tn[j + 1] - G.tn[j]) * dth) : 0.0;
        const double ct0 = j > 0 ? st0 / (T.at(2, 5, i, j - 1) * (G.tn[j] - G.tn[j - 1]) * dth) : 0.0;
        const double inv = 1.0 / (cr1 + cr0 + ct1 + ct0);
        k.c_r1[o] = cr1 * inv;
        k.c_r0[o] = cr0 * inv;
        k.c_t1[o] = ct1 * inv;
        k.c_t0[o] = ct0 * inv;
        k.b[o] = rhs * inv;
    }
}

// One Jacobi sweep over the interior nodes (phi_in -> phi_out); the radial
// end rows stay zero in both buffers.  A thread walks JAC_ROWS rows of one
// theta column keeping the column's three radial neighbours in registers,
// so each phi value comes from L2 about once per sweep; the theta
// neighbours are the same row's loads of the adjacent threads (L1).
constexpr int JAC_ROWS = 8, JAC_THREADS = 128;
__global__ void __launch_bounds__(JAC_THREADS) k_jacobi(CleanK k, const double* __restrict__ phi_in,
                                                        double* __restrict__ phi_out)
{
    const int j = blockIdx.x * JAC_THREADS + threadIdx.x;
    if (j > k.Nth) return;
    const int i0 = 1 + blockIdx.y * JAC_ROWS;
    const int i1 = min(i0 + JAC_ROWS, k.Nr);        // exclusive
    size_t o = (size_t)i0 * k.ld + j;
    double dn = phi_in[o - k.ld], mid = phi_in[o];
    for (int i = i0; i < i1; ++i, o += k.ld) {
        const double up = phi_in[o + k.ld];
        double s = fma(k.c_r1[o], up, k.c_r0[o] * dn);
        if (j < k.Nth) s = fma(k.c_t1[o], phi_in[o + 1], s);
        if (j > 0) s = fma(k.c_t0[o], phi_in[o - 1], s);
        phi_out[o] = s - k.b[o];
        dn = mid;
        mid = up;
    }
}

// D^i -= gamma^ij d_j phi: D^r at (i+1/2, j), D^th at (i, j+1/2), D^ph at
// (i, j) with d_r phi the mean of the two adjacent half-point differences
// (one-sided on the end rows).
__global__ void k_clean_correct(CleanK k, const double* __restrict__ phi, double* Dr, double* Dt, double* Dp)
{
    const int i = blockIdx.y;                       // 0 .. Nr
    const GridDev& G = k.G;
    const Tabs& T = k.T;
    const double iu = i < k.Nr ? 1.0 / (G.rn[i + 1] - G.rn[i]) : 0.0;
    const double id = i > 0 ? 1.0 / (G.rn[i] - G.rn[i - 1]) : 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= k.Nth; j += gridDim.x * blockDim.x) {
        const size_t o = (size_t)i * k.ld + j;
        const double up = i < k.Nr ? (phi[o + k.ld] - phi[o]) * iu : 0.0;
        const double dn = i > 0 ? (phi[o] - phi[o - k.ld]) * id : 0.0;
        const double mean = (i > 0 && i < k.Nr) ? 0.5 * (up + dn) : up + dn;
        if (i < k.Nr) Dr[o] -= tab_gu_rr(T, 1, i, j) * up;
        if (j < k.Nth) Dt[o] -= (phi[o + 1] - phi[o]) / (T.at(2, 5, i, j) * (G.tn[j + 1] - G.tn[j]));
        Dp[o] -= tab_gu_rp(T, 0, i, j) * mean;
    }
}

}  // namespace fpic

namespace fpic {
// ---------------------------------------------------------------------------
// Pair injection (Sec. 3.3, 3.4)
// ---------------------------------------------------------------------------
// Every cell whose centre radius lies in [r_lo, r_hi] gets an e-/e+ pair
// when e n < mult e n_GJ: e n = sum of w |q/m| over the cell's alive
// particles (taken in particle-index order from the stable bucket order, so
// the sum is the same on every run) over the cell's proper volume V,
// e n_GJ = |Omega_h B^z| / 4 pi with B^z = B^r cos th - r sin th B^th at the
// centre.  The pair sits at one point of the cell, each particle with the
// weight that makes the pair's density n0 n_GJ; pairs are appended in cell
// order, e- then e+, while they fit.
struct InjK {
    int Nr, Nth, ld;
    GridDev G;
    BH bh;
    double Om, r_lo, r_hi, mult, n0, qm_e, B0pot;
    const double *Br, *Bth, *draws;
    const double *w, *qm;                    // existing particles
    const uint32_t *off, *perm;              // cell buckets, particle-index order
    uint32_t* flag;                          // per cell 0 / 1
    uint8_t* flags8;                         // optional copy for the caller
    double* wpair;                           // per cell: weight of each new particle
};

__global__ void k_inject_flag(InjK k)
{
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= (long long)k.Nr * k.Nth) return;
    const int i = (int)(c / k.Nth), j = (int)(c - (long long)i * k.Nth);
    uint32_t inj = 0;
    double wp = 0.0;
    const double rc = k.G.rh[i];
    if (rc >= k.r_lo && rc <= k.r_hi) {
        double S = 0.0;
        for (uint32_t q = k.off[c]; q < k.off[c + 1]; ++q) {
            const uint32_t p = k.perm[q];
            S = __dadd_rn(S, __dmul_rn(k.w[p], fabs(k.qm[p])));   // product rounded, then added
        }
        const double V = 2.0 * M_PI * trap16_dev(k.bh, k.G.rn[i], k.G.rn[i + 1], k.G.tn[j], k.G.tn[j + 1]);
        const size_t o = (size_t)i * k.ld + j;
        const double br = 0.5 * (k.Br[o] + k.Br[o + k.ld]);
        const double bt = 0.5 * (k.Bth[o] + k.Bth[o + 1]);
        double sn, cs;
        sincos(k.G.th[j], &sn, &cs);
        const double Bz = br * cs - rc * sn * bt;
        const double gj = fabs(k.Om * Bz) / (4.0 * M_PI);
        inj = S / V < k.mult * gj ? 1u : 0u;
        wp = k.n0 * gj * V / (2.0 * k.qm_e);
    }
    k.flag[c] = inj;
    if (k.flags8) k.flags8[c] = (uint8_t)inj;
    k.wpair[c] = wp;
}

__global__ void k_inject_write(InjK k, fpic_particles P, const uint32_t* __restrict__ pos, long long cap)
{
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= (long long)k.Nr * k.Nth || !k.flag[c]) return;
    const long long m = P.n + 2LL * pos[c];
    if (m + 2 > cap) return;
    const int i = (int)(c / k.Nth), j = (int)(c - (long long)i * k.Nth);
    const double* d = k.draws + 9 * c;
    const double r = k.G.rn[i] + d[0] * (k.G.rn[i + 1] - k.G.rn[i]);
    const double t = k.G.tn[j] + d[1] * (k.G.tn[j + 1] - k.G.tn[j]);
    const double ph = 2.0 * M_PI * d[2];
    double sn, cs;
    sincos(t, &sn, &cs);
    Geo g;
    geo_eval(k.bh, r, sn, cs, g);
    const double L11 = sqrt(g.grr), L31 = g.grp / L11, L22 = sqrt(g.gtt);
    const double L33 = sqrt(fma(-L31, L31, g.gpp));
    const double wp = k.wpair[c];
    for (int s = 0; s < 2; ++s) {
        const double* u = d + 3 + 3 * s;
        const double z[6] = {r, t, ph, L11 * u[0], L22 * u[1], fma(L31, u[0], L33 * u[2])};
        const long long q = m + s;
        const double qm = s == 0 ? -k.qm_e : k.qm_e;
        P.r[q] = z[0]; P.th[q] = z[1]; P.ph[q] = z[2];
        P.ur[q] = z[3]; P.uth[q] = z[4]; P.uph[q] = z[5];
        P.qm[q] = qm;
        P.w[q] = wp;
        P.alive[q] = 1;
        P.scheme[q] = 0;
        P.iters[q] = 0;
        if (P.cell) P.cell[q] = (uint32_t)c;
        double kin, pot;
        h_parts(k.bh, z, qm, k.B0pot, kin, pot);
        P.H0[q] = kin - pot;
        P.Hn[q] = kin - pot;
        P.D0[q] = fabs(kin) + fabs(pot);
    }
}
}  // namespace fpic

extern "C" int fpic_inject_pairs(fpic_ctx* c, fpic_particles* p, long long capacity, const double* Br,
                                 const double* Bth, const fpic_inject_params* prm, const double* draws,
                                 unsigned char* flags, long long* wanted, long long* n_new, void* stream)
{
    if (c && c->G.full) return set_error(FPIC_EINVAL, "fpic_inject_pairs: not built for the full-theta domain");
    if (!c || !p || !Br || !Bth || !prm || !draws || !n_new)
        return set_error(FPIC_EINVAL, "fpic_inject_pairs: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_inject_pairs: no grid set");
    if (p->n < 0 || capacity < p->n) return set_error(FPIC_EINVAL, "fpic_inject_pairs: need 0 <= n <= capacity");
    if (!particles_ok(p, true) || !p->w) return set_error(FPIC_EINVAL, "fpic_inject_pairs: NULL particle array");
    if (!(prm->qm_e > 0.0) || !(prm->n0 > 0.0) || !(prm->multiplicity >= 0.0) || !(prm->r_lo <= prm->r_hi))
        return set_error(FPIC_EINVAL, "fpic_inject_pairs: need qm_e > 0, n0 > 0, multiplicity >= 0, r_lo <= r_hi");
    const long long n = p->n;
    const long long C = (long long)c->Nr * c->Nth;
    if (n + 2 * C > 0xffffffffLL) return set_error(FPIC_EINVAL, "fpic_inject_pairs: more than 2^32 particles");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    Work w;
    int rc = work_layout(c, n > C + 2 ? n : C + 2, false, w);
    if (rc) return rc;
    FPIC_CUDA(cudaMemsetAsync(w.count, 0, 4 * ((size_t)C + 2), s));
    FPIC_CUDA(cudaMemsetAsync(w.cursor, 0, 4 * ((size_t)C + 2), s));
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) k_keys<<<nb, 256, 0, s>>>(c->G, p->r, p->th, p->alive, w.key, nullptr, w.count, n, (uint32_t)C);
    rc = scan_u32(w.count, w.off, w.bsum, C + 1, s);
    if (rc) return rc;
    if (n > 0) k_scatter<<<nb, 256, 0, s>>>(w.key, w.off, w.cursor, w.perm, n);
    k_bucket_rank<<<(unsigned)((C * 32 + 255) / 256), 256, 0, s>>>(w.off, w.perm, w.perm2, (uint32_t)C);
    const double r_h = c->r_h;
    InjK k{c->Nr, c->Nth, c->ld, c->G, c->bh, c->a / (2.0 * c->M * r_h), prm->r_lo, prm->r_hi, prm->multiplicity,
           prm->n0, prm->qm_e, prm->B0pot, Br, Bth, draws, p->w, p->qm, w.off, w.perm2, w.flag, flags, w.tmp};
    const unsigned cb = (unsigned)((C + 255) / 256);
    k_inject_flag<<<cb, 256, 0, s>>>(k);
    rc = scan_u32(w.flag, w.pos, w.bsum, C, s);
    if (rc) return rc;
    k_inject_write<<<cb, 256, 0, s>>>(k, *p, w.pos, capacity);
    FPIC_CUDA(cudaGetLastError());
    uint32_t K = 0;
    FPIC_CUDA(cudaMemcpyAsync(&K, w.pos + C, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    FPIC_CUDA(cudaStreamSynchronize(s));
    const long long room = (capacity - n) / 2;
    if (wanted) *wanted = (long long)K;
    *n_new = n + 2 * ((long long)K < room ? (long long)K : room);
    return FPIC_OK;
}

namespace fpic {
// Eq. (Pbz) on the sphere r = rh[i]: P = (1/2) sum_j (E_th H_ph - E_ph H_th)
// dth_j with each product at the cell centre (rh[i], th_{j+1/2}) from its
// staggered neighbours (E_th averaged in r, H_th in th, E_ph over the four
// nodes).  One block; each thread sums a fixed stride of cells and the block
// sums in a fixed tree, so the result is bitwise reproducible.
__global__ void __launch_bounds__(256) k_bz_power(int Nth, int ld, const double* __restrict__ tn, const double* Eth,
                                                  const double* Eph, const double* Hth, const double* Hph, int i,
                                                  double* out)
{
    __shared__ double part[256];
    double acc = 0.0;
    for (int j = threadIdx.x; j < Nth; j += 256) {
        const size_t o = (size_t)i * ld + j, o1 = o + ld;
        const double et = 0.5 * (Eth[o] + Eth[o1]);
        const double ep = 0.25 * ((Eph[o] + Eph[o + 1]) + (Eph[o1] + Eph[o1 + 1]));
        const double ht = 0.5 * (Hth[o] + Hth[o + 1]);
        acc = fma(fma(et, Hph[o], -ep * ht), tn[j + 1] - tn[j], acc);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * part[0];
}
}  // namespace fpic

extern "C" int fpic_bz_power(fpic_ctx* c, const fpic_fields* f, int i, double* out, void* stream)
{
    if (c && c->G.full) return set_error(FPIC_EINVAL, "fpic_bz_power: not built for the full-theta domain");
    if (!c || !f || !out) return set_error(FPIC_EINVAL, "fpic_bz_power: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_bz_power: no grid set");
    if (i < 0 || i >= c->Nr) return set_error(FPIC_EINVAL, "fpic_bz_power: half-r index %d outside [0, %d)", i, c->Nr);
    if (!f->E[1] || !f->E[2] || !f->H[1] || !f->H[2]) return set_error(FPIC_EINVAL, "fpic_bz_power: NULL E or H array");
    FPIC_CUDA(cudaSetDevice(c->device));
    k_bz_power<<<1, 256, 0, (cudaStream_t)stream>>>(c->Nth, c->ld, c->G.tn, f->E[1], f->E[2], f->H[1], f->H[2], i,
                                                    out);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_div_clean(fpic_ctx* c, double* const D[3], const double* rho, int n_iter, double* phi,
                              void* stream)
{
    if (c && c->G.full) return set_error(FPIC_EINVAL, "fpic_div_clean: not built for the full-theta domain");
    if (!c || !D || !D[0] || !D[1] || !D[2] || !rho) return set_error(FPIC_EINVAL, "fpic_div_clean: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_div_clean: no grid set");
    if (n_iter < 0) return set_error(FPIC_EINVAL, "fpic_div_clean: n_iter < 0");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sz = (size_t)(c->Nr + 1) * c->ld;
    // scratch: 5 coefficient arrays and two phi buffers
    int rc = ensure_scratch2(c, 7 * sz * sizeof(double) + 256);
    if (rc) return rc;
    double* base = (double*)c->d_scratch2;
    CleanK k{c->Nr, c->Nth, c->ld, c->G, tabs_of(c), base, base + sz, base + 2 * sz, base + 3 * sz, base + 4 * sz};
    double* pa = base + 5 * sz;
    double* pb = base + 6 * sz;
    FPIC_CUDA(cudaMemsetAsync(pa, 0, 2 * sz * sizeof(double), s));
    if (c->Nr >= 2) {
        const unsigned gx = (unsigned)((c->Nth + 1 + 255) / 256);
        k_clean_setup<<<dim3(gx, c->Nr - 1), 256, 0, s>>>(k, D[0], D[1], rho);
        const dim3 jg((unsigned)((c->Nth + 1 + JAC_THREADS - 1) / JAC_THREADS),
                      (unsigned)((c->Nr - 1 + JAC_ROWS - 1) / JAC_ROWS));
        auto sweeps = [&](cudaStream_t st) {
            double *x = base + 5 * sz, *y = base + 6 * sz;
            for (int it = 0; it < n_iter; ++it) {
                k_jacobi<<<jg, JAC_THREADS, 0, st>>>(k, x, y);
                double* t = x;
                x = y;
                y = t;
            }
        };
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        FPIC_CUDA(cudaStreamIsCapturing(s, &cap));
        if (n_iter < 8 || cap != cudaStreamCaptureStatusNone) {
            sweeps(s);       // short chains, or the caller is recording a graph itself
        } else {
            // hundreds of short launches: replay them as one graph
            if (!c->clean_exec || c->clean_key_base != base || c->clean_key_Nr != c->Nr ||
                c->clean_key_Nth != c->Nth || c->clean_key_iter != n_iter) {
                if (c->clean_exec) FPIC_CUDA(cudaGraphExecDestroy(c->clean_exec));
                c->clean_exec = nullptr;
                int rc2 = ensure_copy_stream(c);
                if (rc2) return rc2;
                cudaGraph_t g = nullptr;
                FPIC_CUDA(cudaStreamBeginCapture(c->copy_stream, cudaStreamCaptureModeThreadLocal));
                sweeps(c->copy_stream);
                FPIC_CUDA(cudaStreamEndCapture(c->copy_stream, &g));
                cudaError_t e = cudaGraphInstantiate(&c->clean_exec, g, 0);
                cudaGraphDestroy(g);
                FPIC_CUDA(e);
                c->clean_key_base = base;
                c->clean_key_Nr = c->Nr;
                c->clean_key_Nth = c->Nth;
                c->clean_key_iter = n_iter;
            }
            FPIC_CUDA(cudaGraphLaunch(c->clean_exec, s));
        }
        if (n_iter & 1) {
            double* t = pa;
            pa = pb;
            pb = t;
        }
    }
    k_clean_correct<<<dim3((unsigned)((c->Nth + 1 + 255) / 256), c->Nr + 1), 256, 0, s>>>(k, pa, D[0], D[1], D[2]);
    if (phi) FPIC_CUDA(cudaMemcpyAsync(phi, pa, sz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_fdtd_step(fpic_ctx* c, fpic_fields* f, const fpic_fdtd_params* prm, int stage, void* stream)
{
    if (!c || !f || !prm) return set_error(FPIC_EINVAL, "fpic_fdtd_step: NULL argument");
    if (!c->has_grid) return set_error(FPIC_EINVAL, "fpic_fdtd_step: no grid set");
    if (stage != 1 && stage != 2) return set_error(FPIC_EINVAL, "fpic_fdtd_step: stage must be 1 or 2");
    if (!std::isfinite(prm->dt) || !std::isfinite(prm->chi0) || prm->chi0 < 0.0 ||
        (prm->chi0 > 0.0 && !(prm->r_max > prm->r_abs)))
        return set_error(FPIC_EINVAL, "fpic_fdtd_step: bad dt or absorbing-layer parameters");
    for (int k = 0; k < 3; ++k) {
        const void* need[] = {f->B0[k], f->B1[k], f->D0[k], f->D1[k], f->j0[k], f->j1[k], f->E[k], f->H[k],
                              f->Bh[k], f->Dw[k]};
        for (const void* q : need)
            if (!q) return set_error(FPIC_EINVAL, "fpic_fdtd_step: NULL field array");
    }
    if (!f->rho0 || !f->rho1) return set_error(FPIC_EINVAL, "fpic_fdtd_step: NULL rho array");
    FPIC_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    FK k{c->Nr, c->Nth, c->ld, c->G, tabs_of(c), prm->dt, prm->chi0, prm->lambda, prm->r_abs, prm->r_max,
         prm->conserving};
    const size_t sz = (size_t)(c->Nr + 1) * c->ld;
    const dim3 g2(1, c->Nr + 1);
    const int TB = 256;
    auto f3 = [](double* const a[3], double* const b[3]) {
        F3 r;
        for (int q = 0; q < 3; ++q) { r.a[q] = a[q]; r.b[q] = b ? b[q] : nullptr; }
        return r;
    };
    auto o3 = [](double* const a[3]) { O3 r; for (int q = 0; q < 3; ++q) r.p[q] = a[q]; return r; };
    if (stage == 1) {
        // [1] E^{n+1} = alpha <D>^{n+1} + beta x B^{n+1}, <D> materialised in Dw
        k_avg3<<<1024, TB, 0, s>>>(f3(f->D0, f->D1), o3(f->Dw), sz);
        k_make_E<<<g2, TB, 0, s>>>(k, f3(f->Dw, nullptr), f3(f->B1, nullptr), o3(f->E));
        // [2] B^{n+3/2} = <B>^{n+1/2} - dt curl E^{n+1}
        k_update_B<<<g2, TB, 0, s>>>(k, f3(f->B0, f->B1), o3(f->E), o3(f->Bh));
        // [3] E^{n+3/2}
        k_make_E<<<g2, TB, 0, s>>>(k, f3(f->D1, nullptr), f3(f->Bh, nullptr), o3(f->E));
        // [4] B^{n+2} = B^{n+1} - dt curl E^{n+3/2}  (into B0)
        k_update_B<<<g2, TB, 0, s>>>(k, f3(f->B1, nullptr), o3(f->E), o3(f->B0));
    } else {
        // [7] H^{n+3/2} = alpha B^{n+3/2} - beta x D^{n+3/2}
        k_make_H<<<g2, TB, 0, s>>>(k, f3(f->D1, nullptr), f3(f->Bh, nullptr), o3(f->H));
        // [8] D^{n+2} = <D>^{n+1} + dt [curl H - 4 pi <J>^{n+3/2}]  (into Dw)
        Src S0{{f->j0[0], f->j0[1], f->j0[2]}, f->rho0, 0.5}, S1{{f->j1[0], f->j1[1], f->j1[2]}, f->rho1, 0.5};
        k_update_D<<<g2, TB, 0, s>>>(k, f3(f->D0, f->D1), o3(f->H), S0, S1, o3(f->Dw));
        k_bc_D<<<g2, TB, 0, s>>>(k, o3(f->Dw));
        if (!c->G.full) k_axis_D<<<(c->Nr + 1 + 255) / 256, 256, 0, s>>>(k, o3(f->Dw));
        // [9] H^{n+2} = alpha B^{n+2} - beta x D^{n+2}
        k_make_H<<<g2, TB, 0, s>>>(k, f3(f->Dw, nullptr), f3(f->B0, nullptr), o3(f->H));
        // [10] D^{n+5/2} = D^{n+3/2} + dt [curl H - 4 pi J^{n+2}]  (into D0)
        S0.w = 0.0;
        S1.w = 1.0;
        k_update_D<<<g2, TB, 0, s>>>(k, f3(f->D1, nullptr), o3(f->H), S0, S1, o3(f->D0));
        k_bc_D<<<g2, TB, 0, s>>>(k, o3(f->D0));
        if (!c->G.full) k_axis_D<<<(c->Nr + 1 + 255) / 256, 256, 0, s>>>(k, o3(f->D0));
    }
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}
