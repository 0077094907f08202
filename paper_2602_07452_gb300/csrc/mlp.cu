// Learned implicit guess: the MLP 14 -> 128 -> 128 -> 128 -> 9 (ReLU) on the
// fifth-generation tensor cores (tcgen05, BF16 operands, FP32 accumulators
// in tensor memory).
//
//   k_gemm_bf16  generic C (+)= A B^T, one 128-row block per CTA, K staged
//                through shared memory in 64-wide slices; used for every
//                backward GEMM of training.
//   k_mlp_fwd    fused persistent forward: the four weight matrices stay in
//                shared memory, each 128-sample tile runs layer after layer
//                through one TMEM accumulator, the epilogue (bias, ReLU,
//                bf16 rounding) writes the next layer's A operand back to
//                shared memory.
// Parameter layout (FP32 master copy, as the oracle): W1 [128][14] b1 W2
// [128][128] b2 W3 [128][128] b3 W4 [9][128] b4.  Every wait on an mbarrier
// is bounded; a timeout sets an error word and the kernel frees its tensor
// memory and returns.
#include <math.h>

#include <vector>

#include "fpic_internal.h"
#include "mlp_dev.cuh"
#include "tc.cuh"

namespace fpic {

constexpr long long MLP_NPARAM = 128LL * 14 + 128 + 2 * (128LL * 128 + 128) + 9LL * 128 + 9;

// ---------------------------------------------------------------------------
// Generic GEMM
// ---------------------------------------------------------------------------
constexpr int GK = 64;   // K slice staged per round

__global__ void __launch_bounds__(128) k_gemm_bf16(const uint16_t* __restrict__ A, int lda,
                                                   const uint16_t* __restrict__ B, int ldb, float* __restrict__ C,
                                                   int ldc, int M, int N, int K, int accumulate, int* err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;                        // 128 x 64 bf16 = 16 KB
    uint8_t* sB = smem + 16384;                // N x 64 bf16 <= 32 KB
    uint64_t* mbar = (uint64_t*)(smem + 16384 + 32768);
    uint32_t* tslot = (uint32_t*)(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tid == 0) tc::mbar_init(mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    uint32_t phase = 0;
    int ok = 1;
    for (int k0 = 0; k0 < K && ok; k0 += GK) {
        const int kc = min(GK, K - k0);
        const int nv = kc / 8;
        for (int v = tid; v < 128 * nv; v += 128) {
            const int r = v / nv, g = v % nv;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (m0 + r < M) val = *(const uint4*)(A + (size_t)(m0 + r) * lda + k0 + g * 8);
            *(uint4*)(sA + tc::kmajor_off(r, g * 8, 128)) = val;
        }
        for (int v = tid; v < N * nv; v += 128) {
            const int r = v / nv, g = v % nv;
            *(uint4*)(sB + tc::kmajor_off(r, g * 8, N)) = *(const uint4*)(B + (size_t)r * ldb + k0 + g * 8);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t idesc = tc::idesc_bf16(128, N);
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
            for (int kk = 0; kk < kc / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a0 + kk * 2 * (128 * 16), 128 * 16, 128);
                const uint64_t bd = tc::smem_desc(b0 + kk * 2 * (N * 16), N * 16, 128);
                tc::mma_bf16(tbase, ad, bd, idesc, (k0 > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(mbar);
        }
        const int done = tc::mbar_wait(mbar, phase) ? 1 : 0;
        phase ^= 1u;
        ok = __syncthreads_and(done);
    }
    tc::fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            const uint32_t ta = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            int w = min(32, N - c0);
            if (w == 32) tc::tmem_ld32(ta, v);
            else tc::tmem_ld16(ta, v);
            if (row < M) {
                float* cr = C + (size_t)row * ldc + c0;
                for (int i = 0; i < w; ++i) cr[i] = accumulate ? cr[i] + v[i] : v[i];
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// ---------------------------------------------------------------------------
// Parameter packing: FP32 master -> padded bf16 matrices (and transposes)
// ---------------------------------------------------------------------------

__global__ void k_mlp_pack(const float* __restrict__ P, MlpDev d)
{
    const long long oW1 = 0, ob1 = oW1 + 128 * 14, oW2 = ob1 + 128, ob2 = oW2 + 128 * 128, oW3 = ob2 + 128,
                    ob3 = oW3 + 128 * 128, oW4 = ob3 + 128, ob4 = oW4 + 9 * 128;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 128 * 128; t += gridDim.x * blockDim.x) {
        const int o = t / 128, i = t % 128;
        const uint16_t w2 = tc::f2bf(P[oW2 + t]), w3 = tc::f2bf(P[oW3 + t]);
        d.W2[t] = w2;
        d.W3[t] = w3;
        d.W2t[i * 128 + o] = w2;
        d.W3t[i * 128 + o] = w3;
        if (i < 16) d.W1[o * 16 + i] = i < 14 ? tc::f2bf(P[oW1 + o * 14 + i]) : (uint16_t)0;
        if (o < 16) {
            const uint16_t w4 = o < 9 ? tc::f2bf(P[oW4 + o * 128 + i]) : (uint16_t)0;
            d.W4[o * 128 + i] = w4;
            d.W4t[i * 16 + o] = w4;
        }
        if (t < 128) {
            d.b1[t] = P[ob1 + t];
            d.b2[t] = P[ob2 + t];
            d.b3[t] = P[ob3 + t];
        }
        if (t < 16) d.b4[t] = t < 9 ? P[ob4 + t] : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Fused forward (building blocks in mlp_dev.cuh)
// ---------------------------------------------------------------------------
struct FwdK {
    MlpDev w;
    const float* X;      // B x 16 FP32 features (standardised, padded with zeros)
    float* Y;            // B x 16 FP32 outputs (9 used)
    uint16_t* H;         // nullable: 3 x B x 128 bf16 hidden activations
    long long B;         // rows (bound of the launch)
    const long long* count;   // nullable: rows = min(B, *count), read on the device
    int* err;
};

// Fused persistent forward, 256 threads: thread t owns row t % 128 of each
// 128-row tile and half t / 128 of its 16 inputs and of the hidden columns.
// The next tile's inputs are loaded into registers while the current tile
// runs through the four layers.
__global__ void __launch_bounds__(FW_THREADS) k_mlp_fwd(FwdK k)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    long long B = k.B;
    if (k.count) {
        const long long c = *k.count;
        B = c < 0 ? 0 : (c < B ? c : B);
    }
    const long long ntiles = (B + 127) / 128;
    if ((long long)blockIdx.x >= ntiles) return;     // whole block, before any allocation
    float* sb = (float*)(smem + FW_B);
    const int tid = threadIdx.x, warp = tid >> 5, r = tid & 127, half = tid >> 7;
    uint64_t* mbar;
    const uint32_t tbase = mlp_cta_setup(k.w, smem, &mbar);
    uint32_t phase = 0;
    int ok = 1;
    // this thread's 8 inputs of the first tile
    float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
    {
        const long long row = (long long)blockIdx.x * 128 + r;
        if (row < B) {
            xa = *(const float4*)(k.X + row * 16 + 8 * half);
            xb = *(const float4*)(k.X + row * 16 + 8 * half + 4);
        }
    }
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long row = tile * 128 + r;
        *(uint4*)(smem + FW_X + tc::kmajor_off(r, 8 * half, 128)) =
            make_uint4(tc::pack_bf2(xa.x, xa.y), tc::pack_bf2(xa.z, xa.w), tc::pack_bf2(xb.x, xb.y),
                       tc::pack_bf2(xb.z, xb.w));
        {
            const long long nrow = (tile + gridDim.x) * 128 + r;
            xa = make_float4(0.f, 0.f, 0.f, 0.f);
            xb = xa;
            if (nrow < B) {
                xa = *(const float4*)(k.X + nrow * 16 + 8 * half);
                xb = *(const float4*)(k.X + nrow * 16 + 8 * half + 4);
            }
        }
        ok = mlp_tile_layers(tbase, smem, mbar, phase, k.H, row, B);
        if (!ok) break;
        if (half == 0) {
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16), v);
            if (row < B) {
                float4* y = (float4*)(k.Y + row * 16);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    y[q] = make_float4(v[4 * q] + sb[384 + 4 * q], v[4 * q + 1] + sb[385 + 4 * q],
                                       v[4 * q + 2] + sb[386 + 4 * q], v[4 * q + 3] + sb[387 + 4 * q]);
            }
        }
    }
    mlp_cta_teardown(tbase, ok, k.err);
}


// ---------------------------------------------------------------------------
// Training: loss gradient, ReLU backward, transposes, split-K sums, Adam
// ---------------------------------------------------------------------------
struct LossW {
    float m[16];     // regression weights per output (entry 6: the logit, unused)
};

// d loss / d y (scaled by 1/B) for the 9 outputs: 2 m_k (y_k - t_k) and, for
// the logit, sigmoid(y_6) - s; writes dY (FP32), its bf16 copy and the
// per-row loss.
__global__ void k_dloss(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ S,
                        LossW lw, long long B, float invB, float* __restrict__ dY, uint16_t* __restrict__ dYb,
                        float* __restrict__ rowloss)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= B) return;
    float L = 0.f;
    for (int k = 0; k < 16; ++k) {
        float d = 0.f;
        if (k == 6) {
            const float v = Y[b * 16 + 6], sv = S[b];
            const float sp = v > 0.f ? v + log1pf(expf(-v)) : log1pf(expf(v));
            L += sp - sv * v;
            d = 1.f / (1.f + expf(-v)) - sv;
        } else if (k < 9) {
            const float e = Y[b * 16 + k] - T[b * 16 + k];
            L += lw.m[k] * e * e;
            d = 2.f * lw.m[k] * e;
        }
        d *= invB;
        dY[b * 16 + k] = d;
        dYb[b * 16 + k] = tc::f2bf(d);
    }
    rowloss[b] = L;
}

// dZ = dH * (H > 0) in place (FP32) and its bf16 copy [B][128].
__global__ void k_relu_bwd(float* __restrict__ dH, const uint16_t* __restrict__ H, uint16_t* __restrict__ dZb,
                           long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float h = __uint_as_float((uint32_t)H[i] << 16);
        const float d = h > 0.f ? dH[i] : 0.f;
        dH[i] = d;
        dZb[i] = tc::f2bf(d);
    }
}

// out [C][R] = in [R][C] (bf16), 32 x 32 tiles through shared memory.
__global__ void k_transpose_bf16(const uint16_t* __restrict__ in, uint16_t* __restrict__ out, long long R, int Ccols)
{
    __shared__ uint16_t t[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const long long r = r0 + y;
        const int c = c0 + threadIdx.x;
        t[y][threadIdx.x] = (r < R && c < Ccols) ? in[r * Ccols + c] : (uint16_t)0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y;
        const long long r = r0 + threadIdx.x;
        if (c < Ccols && r < R) out[(long long)c * R + r] = t[threadIdx.x][y];
    }
}

// FP32 -> bf16 of X [B][16] (the GEMM operand of dW1).
__global__ void k_to_bf16(const float* __restrict__ x, uint16_t* __restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = tc::f2bf(x[i]);
}

// Column sums of an FP32 [B][C] array (fixed order per column; FP64 accumulate).
__global__ void k_colsum(const float* __restrict__ a, long long B, int Ccols, double* __restrict__ out)
{
    const int c = blockIdx.x;
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long b = threadIdx.x; b < B; b += blockDim.x) acc += (double)a[b * Ccols + c];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// Sum of nsplit partial [M][N] FP32 blocks in a fixed order.
__global__ void k_sum_partials(const float* __restrict__ part, int nsplit, long long MN, float* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < nsplit; ++s) acc += part[(long long)s * MN + i];
        out[i] = acc;
    }
}

struct GradParts {
    const float *dW1, *dW2, *dW3, *dW4t;   // [128][16], [128][128], [128][128], [128][16]
    const double *db1, *db2, *db3, *db4;   // 128, 128, 128, 16
};

// Flat gradient in the parameter layout (W1 b1 W2 b2 W3 b3 W4 b4).
__global__ void k_assemble_grad(GradParts g, float* __restrict__ out)
{
    const long long oW1 = 0, ob1 = 128 * 14, oW2 = ob1 + 128, ob2 = oW2 + 128 * 128, oW3 = ob2 + 128,
                    ob3 = oW3 + 128 * 128, oW4 = ob3 + 128, ob4 = oW4 + 9 * 128;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 128 * 128; t += gridDim.x * blockDim.x) {
        const int o = t / 128, i = t % 128;
        out[oW2 + t] = g.dW2[t];
        out[oW3 + t] = g.dW3[t];
        if (i < 14) out[oW1 + o * 14 + i] = g.dW1[o * 16 + i];
        if (o < 9) out[oW4 + o * 128 + i] = g.dW4t[i * 16 + o];
        if (t < 128) {
            out[ob1 + t] = (float)g.db1[t];
            out[ob2 + t] = (float)g.db2[t];
            out[ob3 + t] = (float)g.db3[t];
        }
        if (t < 9) out[ob4 + t] = (float)g.db4[t];
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters.
__global__ void k_adam(float* __restrict__ P, float* __restrict__ mom, float* __restrict__ vel,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float m = b1 * mom[k] + (1.0f - b1) * gk;
        const float v = b2 * vel[k] + (1.0f - b2) * gk * gk;
        mom[k] = m;
        vel[k] = v;
        P[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

}  // namespace fpic

using namespace fpic;

struct fpic_mlp {
    int device = 0, sm_count = 0;
    void* buf = nullptr;     // device: bf16 weights + biases + error word
    MlpDev d{};
    int* err = nullptr;
};

namespace fpic {
const MlpDev& mlp_weights(const fpic_mlp* m) { return m->d; }
int* mlp_err(const fpic_mlp* m) { return m->err; }
int mlp_sm_count(const fpic_mlp* m) { return m->sm_count; }
}  // namespace fpic

static bool g_fwd_attr_set = false;

extern "C" int fpic_mma_bf16(const uint16_t* A, int lda, const uint16_t* B, int ldb, float* C, int ldc, int M,
                             int N, int K, int accumulate, int* err, void* stream)
{
    if (!A || !B || !C || !err) return set_error(FPIC_EINVAL, "fpic_mma_bf16: NULL argument");
    if (M < 1 || N < 16 || N > 256 || N % 16 || K < 16 || K % 16 || lda % 8 || ldb % 8 || lda < K || ldb < K ||
        ldc < N)
        return set_error(FPIC_EINVAL, "fpic_mma_bf16: need N in [16, 256] and K multiples of 16, lda/ldb >= K "
                                      "and multiples of 8, ldc >= N");
    if (((uintptr_t)A | (uintptr_t)B) & 15) return set_error(FPIC_EINVAL, "fpic_mma_bf16: A, B must be 16-byte aligned");
    // 48 KB are used; asking for 100 KB keeps at most two CTAs per SM, so
    // their tensor-memory allocations (<= 256 columns each) always fit.
    const int smem = 100 * 1024;
    static bool attr = false;
    if (!attr) {
        FPIC_CUDA(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    k_gemm_bf16<<<(M + 127) / 128, 128, smem, (cudaStream_t)stream>>>(A, lda, B, ldb, C, ldc, M, N, K, accumulate, err);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_mlp_create(fpic_mlp** out)
{
    if (!out) return set_error(FPIC_EINVAL, "fpic_mlp_create: NULL");
    *out = nullptr;
    fpic_mlp* m = new fpic_mlp();
    int rc = check_cuda(cudaGetDevice(&m->device), "cudaGetDevice");
    if (!rc) rc = check_cuda(cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device), "attr");
    const size_t w_elems = 128 * 16 + 2 * 128 * 128 + 16 * 128 + 2 * 128 * 128 + 128 * 16;
    const size_t bytes = w_elems * 2 + (3 * 128 + 16) * 4 + 256;
    if (!rc) rc = check_cuda(cudaMalloc(&m->buf, bytes), "cudaMalloc(mlp)");
    if (rc) {
        delete m;
        return rc;
    }
    uint16_t* p = (uint16_t*)m->buf;
    m->d.W1 = p; p += 128 * 16;
    m->d.W2 = p; p += 128 * 128;
    m->d.W3 = p; p += 128 * 128;
    m->d.W4 = p; p += 16 * 128;
    m->d.W2t = p; p += 128 * 128;
    m->d.W3t = p; p += 128 * 128;
    m->d.W4t = p; p += 128 * 16;
    float* f = (float*)p;
    m->d.b1 = f; f += 128;
    m->d.b2 = f; f += 128;
    m->d.b3 = f; f += 128;
    m->d.b4 = f; f += 16;
    m->err = (int*)f;
    cudaMemset(m->err, 0, sizeof(int));
    *out = m;
    return FPIC_OK;
}

extern "C" void fpic_mlp_destroy(fpic_mlp* m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    if (m->buf) cudaFree(m->buf);
    delete m;
}

extern "C" long long fpic_mlp_nparams(void) { return MLP_NPARAM; }

extern "C" int fpic_mlp_set_params(fpic_mlp* m, const float* P, void* stream)
{
    if (!m || !P) return set_error(FPIC_EINVAL, "fpic_mlp_set_params: NULL argument");
    k_mlp_pack<<<64, 256, 0, (cudaStream_t)stream>>>(P, m->d);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

static int mlp_forward_impl(fpic_mlp* m, const float* X, float* Y, uint16_t* H, long long B,
                            const long long* count, cudaStream_t s)
{
    if (!g_fwd_attr_set) {
        FPIC_CUDA(cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
        g_fwd_attr_set = true;
    }
    if (B == 0) return FPIC_OK;
    FwdK k{m->d, X, Y, H, B, count, m->err};
    const long long ntiles = (B + 127) / 128;
    // two CTAs per SM (~110 KB of shared memory and 128 TMEM columns each) so
    // one CTA's epilogue overlaps the other's MMAs
    const long long cap = 2LL * m->sm_count;
    const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
    k_mlp_fwd<<<grid, FW_THREADS, FW_SMEM, s>>>(k);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

namespace fpic {
int mlp_forward_dev(fpic_mlp* m, const float* X, float* Y, long long B, cudaStream_t s)
{
    return mlp_forward_impl(m, X, Y, nullptr, B, nullptr, s);
}

int mlp_forward_dev_count(fpic_mlp* m, const float* X, float* Y, long long B, const long long* count,
                          cudaStream_t s)
{
    return mlp_forward_impl(m, X, Y, nullptr, B, count, s);
}
}  // namespace fpic

extern "C" int fpic_mlp_forward(fpic_mlp* m, const float* X, float* Y, long long B, void* stream)
{
    if (!m || (B > 0 && (!X || !Y))) return set_error(FPIC_EINVAL, "fpic_mlp_forward: NULL argument");
    if (B < 0) return set_error(FPIC_EINVAL, "fpic_mlp_forward: B < 0");
    FPIC_CUDA(cudaSetDevice(m->device));
    return mlp_forward_impl(m, X, Y, nullptr, B, nullptr, (cudaStream_t)stream);
}

extern "C" int fpic_mlp_status(fpic_mlp* m, int* status)
{
    if (!m || !status) return set_error(FPIC_EINVAL, "fpic_mlp_status: NULL argument");
    FPIC_CUDA(cudaMemcpy(status, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    return *status ? set_error(FPIC_ETIMEOUT, "a tensor-core wait timed out") : FPIC_OK;
}


namespace {

struct TrainBufs {
    long long B = 0;
    void* buf = nullptr;
    size_t bytes = 0;
    float *Y, *dY, *dH, *rowloss, *part, *dW1, *dW2, *dW3, *dW4t, *grad;
    double *db;
    uint16_t *H, *Ht, *Xb, *Xt, *dYb, *dYt, *dZb, *dZt;
};

TrainBufs g_tb;   // one training workspace per process (training is serial)

constexpr int SPLITS = 16;

int train_bufs(long long B)
{
    if (g_tb.buf && g_tb.B == B) return 0;
    if (g_tb.buf) FPIC_CUDA(cudaFree(g_tb.buf));
    g_tb.buf = nullptr;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += (b + 255) & ~(size_t)255; return o; };
    size_t oY = take(B * 16 * 4), odY = take(B * 16 * 4), odH = take(B * 128 * 4), orl = take(B * 4),
           opart = take((size_t)SPLITS * 128 * 128 * 4), odW1 = take(128 * 16 * 4), odW2 = take(128 * 128 * 4),
           odW3 = take(128 * 128 * 4), odW4 = take(128 * 16 * 4), ograd = take(MLP_NPARAM * 4),
           odb = take(400 * 8), oH = take(3 * B * 128 * 2), oHt = take(3 * B * 128 * 2), oXb = take(B * 16 * 2),
           oXt = take(16 * B * 2), odYb = take(B * 16 * 2), odYt = take(16 * B * 2), odZb = take(B * 128 * 2),
           odZt = take(128 * B * 2);
    FPIC_CUDA(cudaMalloc(&g_tb.buf, off));
    char* b = (char*)g_tb.buf;
    g_tb.B = B;
    g_tb.bytes = off;
    g_tb.Y = (float*)(b + oY); g_tb.dY = (float*)(b + odY); g_tb.dH = (float*)(b + odH);
    g_tb.rowloss = (float*)(b + orl); g_tb.part = (float*)(b + opart);
    g_tb.dW1 = (float*)(b + odW1); g_tb.dW2 = (float*)(b + odW2); g_tb.dW3 = (float*)(b + odW3);
    g_tb.dW4t = (float*)(b + odW4); g_tb.grad = (float*)(b + ograd); g_tb.db = (double*)(b + odb);
    g_tb.H = (uint16_t*)(b + oH); g_tb.Ht = (uint16_t*)(b + oHt); g_tb.Xb = (uint16_t*)(b + oXb);
    g_tb.Xt = (uint16_t*)(b + oXt); g_tb.dYb = (uint16_t*)(b + odYb); g_tb.dYt = (uint16_t*)(b + odYt);
    g_tb.dZb = (uint16_t*)(b + odZb); g_tb.dZt = (uint16_t*)(b + odZt);
    return 0;
}

int gemm(const uint16_t* A, int lda, const uint16_t* Bm, int ldb, float* C, int ldc, int M, int N, int K, int* err,
         cudaStream_t s)
{
    return fpic_mma_bf16(A, lda, Bm, ldb, C, ldc, M, N, K, 0, err, s);
}

// C [128][N] = A [128][K] Bm[N][K]^T with K split across CTAs (partials
// summed in a fixed order); K a multiple of 16 * SPLITS.
int gemm_splitk(const uint16_t* A, long long lda, const uint16_t* Bm, long long ldb, float* C, int N, long long K,
                int* err, cudaStream_t s)
{
    const long long ks = K / SPLITS;
    for (int sp = 0; sp < SPLITS; ++sp) {
        int rc = fpic_mma_bf16(A + sp * ks, (int)lda, Bm + sp * ks, (int)ldb, g_tb.part + (size_t)sp * 128 * N, N,
                               128, N, (int)ks, 0, err, s);
        if (rc) return rc;
    }
    k_sum_partials<<<64, 256, 0, s>>>(g_tb.part, SPLITS, 128LL * N, C);
    return check_cuda(cudaGetLastError(), "k_sum_partials");
}

void transpose(const uint16_t* in, uint16_t* out, long long R, int Cc, cudaStream_t s)
{
    dim3 grid((unsigned)((R + 31) / 32), (unsigned)((Cc + 31) / 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(in, out, R, Cc);
}

}  // namespace

// Gradient of the batch loss (in the parameter layout) and the loss value.
static int mlp_grad_impl(fpic_mlp* m, const float* X, const float* T, const float* S, const float* lossw, long long B,
                         float* grad, float* loss_host, cudaStream_t s)
{
    int rc = train_bufs(B);
    if (rc) return rc;
    TrainBufs& t = g_tb;
    const long long BH = B * 128;
    rc = mlp_forward_impl(m, X, t.Y, t.H, B, nullptr, s);
    if (rc) return rc;
    LossW lw;
    for (int k = 0; k < 16; ++k) lw.m[k] = k < 9 ? lossw[k] : 0.f;
    const unsigned nb = (unsigned)((B + 255) / 256);
    k_dloss<<<nb, 256, 0, s>>>(t.Y, T, S, lw, B, 1.0f / (float)B, t.dY, t.dYb, t.rowloss);
    k_to_bf16<<<256, 256, 0, s>>>(X, t.Xb, B * 16);
    transpose(t.Xb, t.Xt, B, 16, s);
    transpose(t.dYb, t.dYt, B, 16, s);
    for (int l = 0; l < 3; ++l) transpose(t.H + l * BH, t.Ht + l * BH, B, 128, s);
    int* err = m->err;
    double* db1 = t.db; double* db2 = t.db + 128; double* db3 = t.db + 256; double* db4 = t.db + 384;
    // layer 4
    k_colsum<<<16, 256, 0, s>>>(t.dY, B, 16, db4);
    if ((rc = gemm_splitk(t.Ht + 2 * BH, B, t.dYt, B, t.dW4t, 16, B, err, s))) return rc;
    if ((rc = gemm(t.dYb, 16, m->d.W4t, 16, t.dH, 128, (int)B, 128, 16, err, s))) return rc;
    // layer 3
    k_relu_bwd<<<1024, 256, 0, s>>>(t.dH, t.H + 2 * BH, t.dZb, BH);
    k_colsum<<<128, 256, 0, s>>>(t.dH, B, 128, db3);
    transpose(t.dZb, t.dZt, B, 128, s);
    if ((rc = gemm_splitk(t.dZt, B, t.Ht + BH, B, t.dW3, 128, B, err, s))) return rc;
    if ((rc = gemm(t.dZb, 128, m->d.W3t, 128, t.dH, 128, (int)B, 128, 128, err, s))) return rc;
    // layer 2
    k_relu_bwd<<<1024, 256, 0, s>>>(t.dH, t.H + BH, t.dZb, BH);
    k_colsum<<<128, 256, 0, s>>>(t.dH, B, 128, db2);
    transpose(t.dZb, t.dZt, B, 128, s);
    if ((rc = gemm_splitk(t.dZt, B, t.Ht, B, t.dW2, 128, B, err, s))) return rc;
    if ((rc = gemm(t.dZb, 128, m->d.W2t, 128, t.dH, 128, (int)B, 128, 128, err, s))) return rc;
    // layer 1
    k_relu_bwd<<<1024, 256, 0, s>>>(t.dH, t.H, t.dZb, BH);
    k_colsum<<<128, 256, 0, s>>>(t.dH, B, 128, db1);
    transpose(t.dZb, t.dZt, B, 128, s);
    if ((rc = gemm_splitk(t.dZt, B, t.Xt, B, t.dW1, 16, B, err, s))) return rc;
    GradParts gp{t.dW1, t.dW2, t.dW3, t.dW4t, db1, db2, db3, db4};
    k_assemble_grad<<<64, 256, 0, s>>>(gp, grad);
    FPIC_CUDA(cudaGetLastError());
    if (loss_host) {
        std::vector<float> h(B);
        FPIC_CUDA(cudaMemcpyAsync(h.data(), t.rowloss, B * 4, cudaMemcpyDeviceToHost, s));
        FPIC_CUDA(cudaStreamSynchronize(s));
        double L = 0.0;
        for (long long b = 0; b < B; ++b) L += h[b];
        *loss_host = (float)(L / (double)B);
    }
    return FPIC_OK;
}

static bool mlp_batch_ok(long long B)
{
    return B >= 16 * SPLITS && (B & (B - 1)) == 0 && B <= (1LL << 24);
}

extern "C" int fpic_mlp_grad(fpic_mlp* m, const float* X, const float* T, const float* S, const float* lossw,
                             long long B, float* grad, float* loss, void* stream)
{
    if (!m || !X || !T || !S || !lossw || !grad) return set_error(FPIC_EINVAL, "fpic_mlp_grad: NULL argument");
    if (!mlp_batch_ok(B)) return set_error(FPIC_EINVAL, "fpic_mlp_grad: B must be a power of two in [256, 2^24]");
    FPIC_CUDA(cudaSetDevice(m->device));
    return mlp_grad_impl(m, X, T, S, lossw, B, grad, loss, (cudaStream_t)stream);
}

extern "C" int fpic_mlp_train_step(fpic_mlp* m, float* P, float* mom, float* vel, const float* X, const float* T,
                                   const float* S, const float* lossw, long long B, int step, float lr, float beta1,
                                   float beta2, float eps, float* loss, void* stream)
{
    if (!m || !P || !mom || !vel || !X || !T || !S || !lossw) return set_error(FPIC_EINVAL, "fpic_mlp_train_step: NULL argument");
    if (!mlp_batch_ok(B)) return set_error(FPIC_EINVAL, "fpic_mlp_train_step: B must be a power of two in [256, 2^24]");
    if (step < 1 || !(lr > 0.f)) return set_error(FPIC_EINVAL, "fpic_mlp_train_step: step >= 1 and lr > 0 required");
    FPIC_CUDA(cudaSetDevice(m->device));
    cudaStream_t s = (cudaStream_t)stream;
    int rc = train_bufs(B);
    if (rc) return rc;
    rc = mlp_grad_impl(m, X, T, S, lossw, B, g_tb.grad, loss, s);
    if (rc) return rc;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<64, 256, 0, s>>>(P, mom, vel, g_tb.grad, MLP_NPARAM, lr, beta1, beta2, eps, c1, c2);
    FPIC_CUDA(cudaGetLastError());
    return fpic_mlp_set_params(m, P, stream);
}
