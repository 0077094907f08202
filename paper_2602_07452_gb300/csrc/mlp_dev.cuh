// Building blocks of the fused tcgen05 forward of the learned-guess MLP
// (14 -> 128 -> 128 -> 128 -> 9, ReLU): the bf16 weight layouts, the
// shared-memory map of a CTA that keeps all four weight matrices resident,
// and the per-tile chain of four MMAs with their epilogues.  Shared by the
// plain forward (mlp.cu) and the fused corrector of the push (push.cu).
#pragma once
#include "tc.cuh"

namespace fpic {

struct MlpDev {
    // bf16 weights, row-major [out][in] padded: W1 [128][16], W2, W3 [128][128], W4 [16][128]
    uint16_t *W1, *W2, *W3, *W4;
    // transposes for the backward: W2t, W3t [128][128] (= [in][out]), W4t [128][16]
    uint16_t *W2t, *W3t, *W4t;
    float *b1, *b2, *b3, *b4;    // b4 padded to 16
};

// shared memory map (bytes)
constexpr int FW_W1 = 0, FW_W2 = FW_W1 + 128 * 16 * 2, FW_W3 = FW_W2 + 128 * 128 * 2, FW_W4 = FW_W3 + 128 * 128 * 2,
              FW_X = FW_W4 + 16 * 128 * 2, FW_H = FW_X + 128 * 16 * 2, FW_B = FW_H + 128 * 128 * 2,
              FW_BAR = FW_B + (3 * 128 + 16) * 4, FW_SMEM = FW_BAR + 64;
constexpr int FW_THREADS = 256;

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

// Epilogue of a hidden layer: z = acc + b; a = bf16(relu(z)) into sH.  Row
// r = thread % 128 (its TMEM lane); the two halves of the block take
// columns [0, 64) and [64, 128).  Optionally to global H (bf16 [B][128]).
__device__ __forceinline__ void hidden_epilogue(uint32_t tbase, const float* b, uint8_t* sH, uint16_t* Hg,
                                                long long row, long long B)
{
    const int r = threadIdx.x & 127, warp = (threadIdx.x >> 5) & 3, half = threadIdx.x >> 7;
    for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 32) {
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


// CTA set-up: weights and biases into shared memory, 128 TMEM columns,
// the MMA mbarrier.  Returns the TMEM base; *mbar points at the barrier.
__device__ __forceinline__ uint32_t mlp_cta_setup(const MlpDev& w, uint8_t* smem, uint64_t** mbar)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    float* sb = (float*)(smem + FW_B);
    *mbar = (uint64_t*)(smem + FW_BAR);
    uint32_t* tslot = (uint32_t*)(smem + FW_BAR + 16);
    load_tile_kmajor(smem + FW_W1, w.W1, 128, 16);
    load_tile_kmajor(smem + FW_W2, w.W2, 128, 128);
    load_tile_kmajor(smem + FW_W3, w.W3, 128, 128);
    load_tile_kmajor(smem + FW_W4, w.W4, 16, 128);
    for (int i = tid; i < 3 * 128 + 16; i += FW_THREADS)
        sb[i] = i < 128 ? w.b1[i] : i < 256 ? w.b2[i - 128] : i < 384 ? w.b3[i - 256] : w.b4[i - 384];
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    if (tid == 0) tc::mbar_init(*mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return *tslot;
}

// The four layers of one 128-row tile whose bf16 inputs are in FW_X; the
// output layer's accumulators stay in TMEM columns 0-15.  Hg (nullable):
// bf16 hidden activations for training, 3 x B x 128.  Returns 0 if a
// bounded tensor-core wait ran out.
__device__ __forceinline__ int mlp_tile_layers(uint32_t tbase, uint8_t* smem, uint64_t* mbar, uint32_t& phase,
                                               uint16_t* Hg, long long row, long long B)
{
    const float* sb = (const float*)(smem + FW_B);
    if (!layer_mma(tbase, smem + FW_X, smem + FW_W1, 128, 16, mbar, phase)) return 0;
    hidden_epilogue(tbase, sb, smem + FW_H, Hg, row, B);
    if (!layer_mma(tbase, smem + FW_H, smem + FW_W2, 128, 128, mbar, phase)) return 0;
    hidden_epilogue(tbase, sb + 128, smem + FW_H, Hg ? Hg + (size_t)B * 128 : nullptr, row, B);
    if (!layer_mma(tbase, smem + FW_H, smem + FW_W3, 128, 128, mbar, phase)) return 0;
    hidden_epilogue(tbase, sb + 256, smem + FW_H, Hg ? Hg + (size_t)2 * B * 128 : nullptr, row, B);
    return layer_mma(tbase, smem + FW_H, smem + FW_W4, 16, 128, mbar, phase);
}

// CTA tear-down: error word on a timed-out wait, TMEM freed.
__device__ __forceinline__ void mlp_cta_teardown(uint32_t tbase, int ok, int* err)
{
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    tc::fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tbase, 128);
}

}  // namespace fpic

namespace fpic {

// ---------------------------------------------------------------------------
// Four independent 128-row tile pipelines in one CTA of 512 threads (one
// CTA per SM): the weights are resident once, each group of four warps
// (g = warp / 4) owns 128 TMEM columns, its own input / hidden tiles and
// its own mbarrier, and synchronises on named barrier 1 + g, so one group's
// epilogue overlaps another's MMAs.
// ---------------------------------------------------------------------------
constexpr int G4_GROUPS = 4, G4_THREADS = 128 * G4_GROUPS;
constexpr int G4_B = FW_X;                                   // biases after the weights
constexpr int G4_TILE0 = ((G4_B + (3 * 128 + 16) * 4 + 1023) / 1024) * 1024;
constexpr int G4_TILE_BYTES = 128 * 16 * 2 + 128 * 128 * 2;  // X + H of one group
constexpr int G4_BAR = G4_TILE0 + G4_GROUPS * G4_TILE_BYTES;
constexpr int G4_SMEM = G4_BAR + 128;

__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g));
}

// AND of pred over the 128 threads of group g (named barrier 1 + g).
__device__ __forceinline__ int group_sync_and(int g, int pred)
{
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.and.pred q, %2, 128, p;\n"
        " selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(pred), "r"(1 + g));
    return r;
}

__device__ __forceinline__ int layer_mma_g(int g, uint32_t tbase, const uint8_t* sA, const uint8_t* sB, int N, int K,
                                           uint64_t* mbar, uint32_t& phase)
{
    tc::fence_async_smem();
    tc::fence_before();
    group_sync(g);
    if ((threadIdx.x & 127) == 0) {
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
    const int ok = group_sync_and(g, done);
    tc::fence_after();
    return ok;
}

// Hidden-layer epilogue of one group: thread t % 128 owns row t % 128 (its
// TMEM lane) and all 128 columns.
__device__ __forceinline__ void hidden_epilogue_g(uint32_t tbase, const float* b, uint8_t* sH)
{
    const int r = threadIdx.x & 127, wq = (threadIdx.x >> 5) & 3;
    for (int c0 = 0; c0 < 128; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int gq = 0; gq < 4; ++gq) {
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + gq * 8 + 2 * q;
                const float z0 = v[gq * 8 + 2 * q] + b[c], z1 = v[gq * 8 + 2 * q + 1] + b[c + 1];
                pk[q] = tc::pack_bf2(z0 > 0.f ? z0 : 0.f, z1 > 0.f ? z1 : 0.f);
            }
            *(uint4*)(sH + tc::kmajor_off(r, c0 + gq * 8, 128)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

// The four layers of group g's tile (inputs already in its X tile); the
// output layer's accumulators stay in its TMEM columns 0-15.
__device__ __forceinline__ int mlp_tile_layers_g(int g, uint32_t tbase, uint8_t* smem, uint64_t* mbar,
                                                 uint32_t& phase)
{
    const float* sb = (const float*)(smem + G4_B);
    uint8_t* sX = smem + G4_TILE0 + g * G4_TILE_BYTES;
    uint8_t* sH = sX + 128 * 16 * 2;
    if (!layer_mma_g(g, tbase, sX, smem + FW_W1, 128, 16, mbar, phase)) return 0;
    hidden_epilogue_g(tbase, sb, sH);
    if (!layer_mma_g(g, tbase, sH, smem + FW_W2, 128, 128, mbar, phase)) return 0;
    hidden_epilogue_g(tbase, sb + 128, sH);
    if (!layer_mma_g(g, tbase, sH, smem + FW_W3, 128, 128, mbar, phase)) return 0;
    hidden_epilogue_g(tbase, sb + 256, sH);
    return layer_mma_g(g, tbase, sH, smem + FW_W4, 16, 128, mbar, phase);
}

// CTA set-up of the four-group layout: weights and biases into shared
// memory, 512 TMEM columns, one mbarrier per group.  Returns the TMEM base.
__device__ __forceinline__ uint32_t mlp_cta_setup4(const MlpDev& w, uint8_t* smem)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    float* sb = (float*)(smem + G4_B);
    uint64_t* mbar = (uint64_t*)(smem + G4_BAR);
    uint32_t* tslot = (uint32_t*)(smem + G4_BAR + 64);
    load_tile_kmajor(smem + FW_W1, w.W1, 128, 16);
    load_tile_kmajor(smem + FW_W2, w.W2, 128, 128);
    load_tile_kmajor(smem + FW_W3, w.W3, 128, 128);
    load_tile_kmajor(smem + FW_W4, w.W4, 16, 128);
    for (int i = tid; i < 3 * 128 + 16; i += blockDim.x)
        sb[i] = i < 128 ? w.b1[i] : i < 256 ? w.b2[i - 128] : i < 384 ? w.b3[i - 256] : w.b4[i - 384];
    if (warp == 0) tc::tmem_alloc(tslot, 128 * G4_GROUPS);
    if (tid < G4_GROUPS) tc::mbar_init(mbar + tid, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return *tslot;
}

__device__ __forceinline__ void mlp_cta_teardown4(uint32_t tbase, int ok, int* err)
{
    if (!ok) atomicExch(err, 1);
    tc::fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tbase, 128 * G4_GROUPS);
}

}  // namespace fpic
