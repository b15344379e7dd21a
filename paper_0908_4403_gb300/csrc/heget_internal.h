// heget_internal.h -- host-side state and helpers shared by the C-ABI
// translation units (the context, argument checks, launch constants).
// Include after heget_kernels.cuh.
#pragma once

#include <cstdarg>

#include <cuda_runtime.h>

#include "heget.h"
#include "heget_common.cuh"
#include "heget_graphcache.h"

namespace heget {

constexpr int kBlockThreads = 256;   // amplitude kernels: threads per block
constexpr int kMaxGrid = 65536;      // block partials held by a context

// Records a message for heget_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// Makes `dev` current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace heget

// The library context (opaque in the C ABI).
struct heget_ctx {
    int device = 0;
    int num_sms = 0;
    heget_params params{};
    heget::Partial* partials = nullptr;      // kMaxGrid block partials
    int* flag = nullptr;              // device input-check flag
    heget_xsec_result* res_dev = nullptr;
    heget_xsec_result* res_host = nullptr;  // pinned
    int last_parts = 0;               // block partials of the last heget_xsec_launch
    int last_kind = 0;                // its sampler kind
    bool last_ws = false;             // it used the warp-specialised kernel
    bool last_esc = false;            // it launched the FP64 escalation kernel after it
    int tiles[2][2][heget::kMaxN + 1] = {};  // [amp2|xsec][fp32|fp64][n] tile overrides (0 = default)
    int shapes[2][heget::kMaxN + 1] = {};    // [fp32|fp64][n] tile-kernel shape of the fused cross section
    int alg = 0;                      // ordering sum: HEGET_ALG_TREE or HEGET_ALG_SUBSET
    double esc_tau = 0.0;             // FP32 -> FP64 escalation threshold (0 = off)
    int hel_sample = 0;               // one sampled helicity per point (heget_set_helicity_sampling)
    // escalation lists of the fused FP32 launch (grown on demand): entries
    // [grid][cap] of (point index, FP32 weight) and per-block counts
    long long* esc_idx = nullptr;
    double* esc_w = nullptr;
    int* esc_cnt = nullptr;
    size_t esc_idx_cap = 0, esc_w_cap = 0, esc_cnt_cap = 0;
    // escalation list of FP32 heget_amp2 (row indices) and its device counter
    int* amp_esc_list = nullptr;
    size_t amp_esc_cap = 0;
    int* amp_esc_count = nullptr;
    // mixed-n batch workspace (grown on demand)
    unsigned char* batch_host = nullptr;   // pinned staging of work items + request table
    unsigned char* batch_dev = nullptr;
    size_t batch_cap = 0, batch_dev_cap = 0;
    heget::Partial* batch_partials = nullptr;
    size_t batch_partials_cap = 0;
    cudaEvent_t batch_copied = nullptr;    // staging may be rewritten once this has fired
    int graphs = 0;                        // batch launches replay CUDA graphs per launch-shape bucket
    heget::BatchGraphCache batch_graphs;
    // heget_hist: per-block partial histograms (grown on demand)
    double* hist_parts = nullptr;
    size_t hist_parts_cap = 0;
};

namespace heget {
struct AmpLaunch;
// Grows the escalation lists of a fused FP32 launch of shape L over N points.
int reserve_escalation(heget_ctx* ctx, const AmpLaunch& L, long long N);
Physics physics_of(const heget_params& p, int n);
Physics physics_of(const heget_ctx* c, int n);
int check_sampler(const heget_sampler* s);
SamplerArgs sampler_args(const heget_sampler* s);
int check_common(const heget_ctx* ctx, int n, long long N);
int check_precision(int p);
// i0 >= 0 and the last point index i0 + N - 1 representable as int64.
int check_range(long long i0, long long N);
// Finite alpha > 0, finite nonzero charge, finite pt_min >= 0 and eta_max > 0,
// dr_min not NaN.
int check_params(const heget_params* p);
// Grows a workspace buffer to at least `need` bytes (device, or pinned host).
int grow(void** p, size_t* cap, size_t need, bool pinned);
}  // namespace heget
