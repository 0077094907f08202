// Library-internal context and helpers shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fpic.h"
#include "fpic_device.cuh"

// fpic_push_host: particle chunks whose host-to-device copies overlap the
// explicit pass of the earlier chunks.
#define FPIC_HOST_CHUNKS 4

struct fpic_ctx {
    int device = 0;
    int sm_count = 0;
    double M = 1.0, a = 0.0;
    fpic::BH bh{};
    double r_h = 0.0;
    // grid
    bool has_grid = false;
    int Nr = 0, Nth = 0, ld = 0;
    double* d_nodes = nullptr;       // rn rh tn th irn irh itn ith (library-owned)
    fpic::GridDev G{};
    // host copies of the node tables
    std::string h_nodes;             // raw bytes of rn, rh, tn, th
    // metric tables at the Yee points (library-owned), see pic.cu
    double* d_metric = nullptr;
    size_t metric_stride = 0;        // elements per table
    // device counters (library-owned) and their pinned host mirror
    long long* d_cnt = nullptr;
    long long* h_cnt = nullptr;
    // scratch grown on demand
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // batched push: run descriptors (pinned host staging + device copy)
    void* h_runs = nullptr;
    void* d_runs = nullptr;
    int runs_cap = 0;
    // second scratch (sort / deposit)
    void* d_scratch2 = nullptr;
    size_t scratch2_bytes = 0;
    // launch-shape tuning (fpic_set_tuning)
    int imr_blocks_per_sm = 4;
    int dep_threads = 128;           // threads per block of the deposit's particle kernel
    int dep_lattice = 1;             // FPIC_TUNE_DEP_LATTICE: 1 paired-FP32 trapezoid lattices, 0 FP64
    int async = 0;                   // FPIC_TUNE_ASYNC: stats copied asynchronously, no host-side synchronisation
    int host_staging = 0;            // FPIC_TUNE_HOST_STAGING: fpic_push_host copies even mapped arrays
    // per-cell field interpolation coefficients (rebuilt by every push with fields)
    void* d_fcoef = nullptr;
    size_t fcoef_bytes = 0;
    int static_fields = 0;           // FPIC_TUNE_STATIC_FIELDS: reuse the coefficients of unchanged pointers
    // FPIC_TUNE_REUSE_SLOPE: the right-hand side at the end of each particle's
    // step, kept for the first RK4 stage of the next (see push.cu); the
    // cache is cold whenever its key (particle arrays, n, fields, grid) changes
    int reuse_slope = 0;
    void* d_slope = nullptr;
    size_t slope_bytes = 0;
    const void* slope_key_r = nullptr;
    long long slope_key_n = -1;
    const double* slope_key_f[6] = {};
    double slope_key_B0field = 0.0;
    unsigned long long slope_key_grid = 0;
    unsigned long long grid_gen = 0;    // incremented by every fpic_set_grid
    // FPIC_TUNE_STAGE_FIELDS: TMA staging of the coefficient tiles a block of
    // cell-sorted particles touches (tensor maps of d_fcoef, see push.cu)
    int stage_fields = 0;
    void* d_stage_maps = nullptr;
    const void* stage_key = nullptr;
    int stage_key_Nr = 0, stage_key_ld = 0;
    const double* fcoef_src[6] = {};  // the field arrays the coefficients were built from
    // fpic_push_host: copy stream and per-chunk events (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[FPIC_HOST_CHUNKS + 1] = {};
    // fpic_div_clean: the chain of Jacobi sweeps as an instantiated graph,
    // rebuilt when its key (scratch base, grid shape, sweep count) changes
    cudaGraphExec_t clean_exec = nullptr;
    const void* clean_key_base = nullptr;
    int clean_key_Nr = 0, clean_key_Nth = 0, clean_key_iter = -1;
    // buffers superseded by a larger one (scratch, coefficients, run table,
    // node and metric tables): a CUDA graph captured earlier may still
    // address them, so they are freed only by fpic_destroy
    std::vector<void*> retired_dev;
    std::vector<void*> retired_host;
};

namespace fpic {

enum { CNT_QUEUE = 0, CNT_HEAD = 1, CNT_ITERS = 2, CNT_NOTCONV = 3, CNT_REMOVED = 4,
       CNT_ALIVE = 5, CNT_EVALS = 6, CNT_ERR = 7, CNT_WORK = 8, CNT_SKIP = 9, CNT_PRIO = 10,
       CNT_NORM = 11, CNT_SLOPE = 12, CNT_STAGED = 13, CNT_STRAG = 14, CNT_N = 15 };

int set_error(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);
int ensure_scratch(fpic_ctx* c, size_t bytes);
int ensure_scratch2(fpic_ctx* c, size_t bytes);
int ensure_copy_stream(fpic_ctx* c);
// Moves a superseded buffer to the context's retired list (nothing is freed
// before fpic_destroy) and clears the pointer.
void retire(fpic_ctx* c, void** p, bool host = false);
bool particles_ok(const fpic_particles* p, bool need_state);
int mlp_forward_dev(fpic_mlp* m, const float* X, float* Y, long long B, cudaStream_t s);
struct MlpDev;
const MlpDev& mlp_weights(const fpic_mlp* m);
int* mlp_err(const fpic_mlp* m);
int mlp_sm_count(const fpic_mlp* m);
// Forward pass of min(B, *count) rows, count read on the device (B bounds the launch).
int mlp_forward_dev_count(fpic_mlp* m, const float* X, float* Y, long long B, const long long* count,
                          cudaStream_t s);

}  // namespace fpic

#define FPIC_CUDA(call)                                                   \
    do {                                                                  \
        int _rc = fpic::check_cuda((call), #call);                        \
        if (_rc) return _rc;                                              \
    } while (0)
