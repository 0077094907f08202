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

#include "fpic_internal.h"
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
struct MlpDev {
    // bf16 weights, row-major [out][in] padded: W1 [128][16], W2, W3 [128][128], W4 [16][128]
    uint16_t *W1, *W2, *W3, *W4;
    // transposes for the backward: W2t, W3t [128][128] (= [in][out]), W4t [128][16]
    uint16_t *W2t, *W3t, *W4t;
    float *b1, *b2, *b3, *b4;    // b4 padded to 16
};

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
// Fused forward
// ---------------------------------------------------------------------------
// shared memory map (bytes)
constexpr int FW_W1 = 0, FW_W2 = FW_W1 + 128 * 16 * 2, FW_W3 = FW_W2 + 128 * 128 * 2, FW_W4 = FW_W3 + 128 * 128 * 2,
              FW_X = FW_W4 + 16 * 128 * 2, FW_H = FW_X + 128 * 16 * 2, FW_BAR = FW_H + 128 * 128 * 2,
              FW_SMEM = FW_BAR + 64;

__device__ __forceinline__ void load_tile_kmajor(uint8_t* dst, const uint16_t* __restrict__ src, int R, int Kd)
{
    const int nv = Kd / 8;
    for (int v = threadIdx.x; v < R * nv; v += blockDim.x) {
        const int r = v / nv, g = v % nv;
        *(uint4*)(dst + tc::kmajor_off(r, g * 8, R)) = *(const uint4*)(src + (size_t)r * Kd + g * 8);
    }
}

// Run one layer's MMAs (A: 128 x K in sA, B: N x K in sB) into TMEM and wait.
__device__ __forceinline__ int layer_mma(uint32_t tbase, const uint8_t* sA, const uint8_t* sB, int N, int K,
                                         uint64_t* mbar, uint32_t& phase)
{
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after();
        const uint32_t idesc = tc::idesc_bf16(128, N);
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(a0 + kk * 2 * (128 * 16), 128 * 16, 128);
            const uint64_t bd = tc::smem_desc(b0 + kk * 2 * (N * 16), N * 16, 128);
            tc::mma_bf16(tbase, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
        tc::mma_commit(mbar);
    }
    const int done = tc::mbar_wait(mbar, phase) ? 1 : 0;
    phase ^= 1u;
    const int ok = __syncthreads_and(done);
    tc::fence_after();
    return ok;
}

// Epilogue of a hidden layer: z = acc + b; a = bf16(relu(z)) into sH (row r
// = thread), optionally to global H (bf16 [B][128]).
__device__ __forceinline__ void hidden_epilogue(uint32_t tbase, const float* __restrict__ b, uint8_t* sH,
                                                uint16_t* Hg, long long row, long long B)
{
    const int r = threadIdx.x, warp = r >> 5;
    for (int c0 = 0; c0 < 128; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + g * 8 + 2 * q;
                const float z0 = v[g * 8 + 2 * q] + b[c], z1 = v[g * 8 + 2 * q + 1] + b[c + 1];
                pk[q] = tc::pack_bf2(z0 > 0.f ? z0 : 0.f, z1 > 0.f ? z1 : 0.f);
            }
            const uint4 u = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *(uint4*)(sH + tc::kmajor_off(r, c0 + g * 8, 128)) = u;
            if (Hg && row < B) *(uint4*)(Hg + (size_t)row * 128 + c0 + g * 8) = u;
        }
    }
}

struct FwdK {
    MlpDev w;
    const float* X;      // B x 16 FP32 features (standardised, padded with zeros)
    float* Y;            // B x 16 FP32 outputs (9 used)
    uint16_t* H;         // nullable: 3 x B x 128 bf16 hidden activations
    long long B;
    int* err;
};

__global__ void __launch_bounds__(128) k_mlp_fwd(FwdK k)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* mbar = (uint64_t*)(smem + FW_BAR);
    uint32_t* tslot = (uint32_t*)(smem + FW_BAR + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    load_tile_kmajor(smem + FW_W1, k.w.W1, 128, 16);
    load_tile_kmajor(smem + FW_W2, k.w.W2, 128, 128);
    load_tile_kmajor(smem + FW_W3, k.w.W3, 128, 128);
    load_tile_kmajor(smem + FW_W4, k.w.W4, 16, 128);
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    if (tid == 0) tc::mbar_init(mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    uint32_t phase = 0;
    int ok = 1;
    const long long ntiles = (k.B + 127) / 128;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long row = tile * 128 + tid;
        // input tile: one row per thread, 16 features -> bf16
        {
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float a = 0.f, b = 0.f;
                if (row < k.B) {
                    a = k.X[row * 16 + 2 * q];
                    b = k.X[row * 16 + 2 * q + 1];
                }
                pk[q] = tc::pack_bf2(a, b);
            }
            *(uint4*)(smem + FW_X + tc::kmajor_off(tid, 0, 128)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *(uint4*)(smem + FW_X + tc::kmajor_off(tid, 8, 128)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        ok = layer_mma(tbase, smem + FW_X, smem + FW_W1, 128, 16, mbar, phase);
        if (!ok) break;
        hidden_epilogue(tbase, k.w.b1, smem + FW_H, k.H ? k.H : nullptr, row, k.B);
        ok = layer_mma(tbase, smem + FW_H, smem + FW_W2, 128, 128, mbar, phase);
        if (!ok) break;
        hidden_epilogue(tbase, k.w.b2, smem + FW_H, k.H ? k.H + (size_t)k.B * 128 : nullptr, row, k.B);
        ok = layer_mma(tbase, smem + FW_H, smem + FW_W3, 128, 128, mbar, phase);
        if (!ok) break;
        hidden_epilogue(tbase, k.w.b3, smem + FW_H, k.H ? k.H + (size_t)2 * k.B * 128 : nullptr, row, k.B);
        ok = layer_mma(tbase, smem + FW_H, smem + FW_W4, 16, 128, mbar, phase);
        if (!ok) break;
        float v[16];
        tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16), v);
        if (row < k.B) {
#pragma unroll
            for (int c = 0; c < 16; ++c) k.Y[row * 16 + c] = v[c] + k.w.b4[c];
        }
    }
    if (!ok && tid == 0) atomicExch(k.err, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 128);
}

}  // namespace fpic

using namespace fpic;

struct fpic_mlp {
    int device = 0, sm_count = 0;
    void* buf = nullptr;     // device: bf16 weights + biases + error word
    MlpDev d{};
    int* err = nullptr;
};

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

static int mlp_forward_impl(fpic_mlp* m, const float* X, float* Y, uint16_t* H, long long B, cudaStream_t s)
{
    if (!g_fwd_attr_set) {
        FPIC_CUDA(cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
        g_fwd_attr_set = true;
    }
    if (B == 0) return FPIC_OK;
    FwdK k{m->d, X, Y, H, B, m->err};
    const long long ntiles = (B + 127) / 128;
    const unsigned grid = (unsigned)(ntiles < (long long)m->sm_count ? ntiles : m->sm_count);
    k_mlp_fwd<<<grid, 128, FW_SMEM, s>>>(k);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_mlp_forward(fpic_mlp* m, const float* X, float* Y, long long B, void* stream)
{
    if (!m || (B > 0 && (!X || !Y))) return set_error(FPIC_EINVAL, "fpic_mlp_forward: NULL argument");
    if (B < 0) return set_error(FPIC_EINVAL, "fpic_mlp_forward: B < 0");
    FPIC_CUDA(cudaSetDevice(m->device));
    return mlp_forward_impl(m, X, Y, nullptr, B, (cudaStream_t)stream);
}

extern "C" int fpic_mlp_status(fpic_mlp* m, int* status)
{
    if (!m || !status) return set_error(FPIC_EINVAL, "fpic_mlp_status: NULL argument");
    FPIC_CUDA(cudaMemcpy(status, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    return *status ? set_error(FPIC_ETIMEOUT, "a tensor-core wait timed out") : FPIC_OK;
}
