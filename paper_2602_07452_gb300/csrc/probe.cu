// Measurement helper: sustained FP64 FMA throughput of the device.  Eight
// independent FMA chains per thread keep the FP64 pipe fed; the result is
// stored so the chains cannot be removed.
#include "ff.cuh"
#include "fpic_internal.h"

namespace fpic {

__global__ void __launch_bounds__(256) k_fma64(double* out, int reps, double x)
{
    double a0 = x + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const double m = 0.999999999, c = 1e-9;
    for (int i = 0; i < reps; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
            a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void k_math(int fn, const double* __restrict__ x, double* __restrict__ y, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    if (fn == 0) {
        y[i] = rcp_nr(v);
    } else if (fn == 1) {
        y[i] = sqrt_dep(v);
    } else if (fn == 3) {
        y[i] = ff_to(ff_sqrt(ff_from(v)));
    } else if (fn == 5) {
        y[i] = rsqrt_nr(v);
    } else if (fn == 6) {
        y[i] = ff_to(ff_rcp(ff_from(v)));
    } else if (fn == 7) {
        // pair (a, b) = (x[2i], x[2i + 1]) of element i < n / 2: the integer
        // compares of non-negative doubles beside the FP64 ones
        if (2 * i + 1 >= n) return;
        const double a = x[2 * i], b = x[2 * i + 1];
        double* o = y + 6 * i;
        o[0] = le_nonneg(a, b) ? 1.0 : 0.0;
        o[1] = (a <= b) ? 1.0 : 0.0;
        o[2] = lt_nonneg(a, b) ? 1.0 : 0.0;
        o[3] = (a < b) ? 1.0 : 0.0;
        o[4] = fmax_nonneg(a, b);
        o[5] = fmax(a, b);
    } else if (fn == 4) {
        ff sh, cm;
        sincos_step_ff(v, sh, cm);
        y[2 * i] = ff_to(sh);
        y[2 * i + 1] = ff_to(cm);
    } else {
        double sh, cm;
        sincos_step(v, sh, cm);
        y[2 * i] = sh;
        y[2 * i + 1] = cm;
    }
}

}  // namespace fpic

extern "C" int fpic_probe_math(int fn, const double* x, double* y, long long n, void* stream)
{
    using namespace fpic;
    if (fn < 0 || fn > 7 || n < 0 || (n > 0 && (!x || !y))) return set_error(FPIC_EINVAL, "fpic_probe_math: bad argument");
    if (n == 0) return FPIC_OK;
    k_math<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(fn, x, y, n);
    FPIC_CUDA(cudaGetLastError());
    return FPIC_OK;
}

extern "C" int fpic_probe_fp64(double* gflops_out, int reps)
{
    using namespace fpic;
    if (!gflops_out || reps < 1) return set_error(FPIC_EINVAL, "fpic_probe_fp64: bad argument");
    int dev, sms;
    FPIC_CUDA(cudaGetDevice(&dev));
    FPIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    double* out = nullptr;
    FPIC_CUDA(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma64<<<blocks, threads>>>(out, 4, 1.0);   // warm-up
    cudaEventRecord(e0);
    k_fma64<<<blocks, threads>>>(out, reps, 1.0);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    FPIC_CUDA(err);
    const double flops = 2.0 * 8 * 16 * (double)reps * blocks * threads;
    *gflops_out = flops / (ms * 1e-3) / 1e9;
    return FPIC_OK;
}
