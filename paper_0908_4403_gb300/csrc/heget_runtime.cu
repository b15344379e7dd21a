// heget_runtime.cu -- launch machinery around the kernels: CUDA-graph capture
// of the cross-section step and the launch-shape autotuner.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "heget_kernels.cuh"
#include "heget_internal.h"

using namespace heget;

// A captured heget_xsec_launch + heget_xsec_finalize: a chain of kernel
// nodes -- the event kernel, the FP64 escalation kernel when the context
// escalates FP32 points, then the finalisation.  Replays update the first
// two arguments (uint64_t seed, long long i0) of the event and escalation
// kernels, which every variant of them takes first.
struct GraphKernel {
    cudaGraphNode_t node = nullptr;
    cudaKernelNodeParams kp{};   // captured parameters
    int nargs = 0;
};

struct heget_graph {
    heget_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKernel k[2];   // event kernel, escalation kernel
    int nk = 0;
    long long N = 0;    // points per replay
};

namespace {
int graph_fail(heget_graph* g, int code) {
    if (g) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
    }
    return code;
}
}  // namespace

extern "C" {

int heget_graph_xsec(heget_ctx* ctx, int n, int64_t N, const heget_sampler* smp, int precision,
                     heget_xsec_result* result_dev, heget_graph** out) {
    if (!out) return fail(HEGET_EINVAL, "out is NULL");
    *out = nullptr;
    int r = check_common(ctx, n, N);
    if (r) return r;
    if ((r = check_precision(precision))) return r;
    if ((r = check_sampler(smp))) return r;
    if (N < 1 || !result_dev) return fail(HEGET_EINVAL, "a graph needs N >= 1 and result_dev");
    DeviceGuard dg(ctx->device);
    // allocations cannot be captured: grow the escalation lists first
    if (precision == HEGET_FP32 && ctx->esc_tau > 0) {
        AmpLaunch L;
        if ((r = default_amp_launch(n, precision, N, ctx->num_sms, &L, true, ctx->tiles[1][0][n], ctx->alg,
                                    ctx->shapes[0][n])))
            return cuda_fail((cudaError_t)r, "occupancy");
        if ((r = reserve_escalation(ctx, L, N))) return r;
    }
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    heget_graph* g = new heget_graph();
    g->ctx = ctx;
    g->N = N;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(st);
        return graph_fail(g, cuda_fail(e, "cudaStreamBeginCapture"));
    }
    r = heget_xsec_launch(ctx, n, 0, 0, N, smp, precision, nullptr, st);
    if (!r) r = heget_xsec_finalize(ctx, result_dev, st);
    e = cudaStreamEndCapture(st, &g->graph);
    cudaStreamDestroy(st);
    if (r) return graph_fail(g, r);
    if (e != cudaSuccess) return graph_fail(g, cuda_fail(e, "cudaStreamEndCapture"));
    // walk the chain from its root: event kernel, [escalation kernel], finalisation
    g->nk = ctx->last_esc ? 2 : 1;
    g->k[0].nargs = ctx->last_ws ? 8 : 9;
    g->k[1].nargs = 8;
    size_t cnt = 1;
    e = cudaGraphGetRootNodes(g->graph, &g->k[0].node, &cnt);
    if (e != cudaSuccess || cnt != 1) return graph_fail(g, fail(HEGET_ECUDA, "unexpected captured graph shape"));
    for (int j = 0; j < g->nk && e == cudaSuccess; ++j) {
        e = cudaGraphKernelNodeGetParams(g->k[j].node, &g->k[j].kp);
        if (e == cudaSuccess && j + 1 < g->nk) {
            cnt = 1;
            e = cudaGraphNodeGetDependentNodes(g->k[j].node, &g->k[j + 1].node, nullptr, &cnt);
            if (e == cudaSuccess && cnt != 1) return graph_fail(g, fail(HEGET_ECUDA, "unexpected captured graph shape"));
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return graph_fail(g, cuda_fail(e, "graph instantiate"));
    *out = g;
    return HEGET_OK;
}

int heget_graph_launch(heget_graph* g, uint64_t seed, int64_t i0, void* stream) {
    if (!g) return fail(HEGET_EINVAL, "graph is NULL");
    int r = check_range(i0, g->N);
    if (r) return r;
    DeviceGuard dg(g->ctx->device);
    long long i0v = i0;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < g->nk && e == cudaSuccess; ++j) {
        void* args[9];
        for (int a = 0; a < g->k[j].nargs; ++a) args[a] = g->k[j].kp.kernelParams[a];
        args[0] = &seed;
        args[1] = &i0v;
        cudaKernelNodeParams p = g->k[j].kp;
        p.kernelParams = args;
        p.extra = nullptr;
        e = cudaGraphExecKernelNodeSetParams(g->exec, g->k[j].node, &p);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "heget_graph_launch");
    return HEGET_OK;
}

void heget_graph_destroy(heget_graph* g) {
    if (!g) return;
    DeviceGuard dg(g->ctx->device);
    graph_fail(g, 0);
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

namespace {
// Times every candidate launch (shape, tile) of heget_amp2 (kind 0: tiles of
// the context's shape) or heget_xsec (kind 1: every shape, each with its
// default tile and the tiles 256/2^n x 2^k up to 1024) on probe_points
// synthetic points; the context keeps the fastest.
int autotune_impl(heget_ctx* ctx, int n, int precision, int kind, int64_t probe_points, bool shapes, int* best_shape,
                  int* best_tile, double* best_ms) {
    int r = check_common(ctx, n, probe_points);
    if (r) return r;
    if ((r = check_precision(precision))) return r;
    if (kind != 0 && kind != 1) return fail(HEGET_EINVAL, "kind must be 0 (amp2) or 1 (xsec)");
    if (probe_points < 1) return fail(HEGET_EINVAL, "probe_points must be >= 1");
    DeviceGuard dg(ctx->device);
    const int pi = precision == HEGET_FP64;
    const int unit = kBlockThreads >> n;
    const int nshapes = kind == 1 && shapes ? xsec_shape_count(n, precision, ctx->alg) : 1;
    std::vector<std::pair<int, int>> cands;   // (shape, tile)
    for (int sh = 0; sh < nshapes; ++sh) {
        const int shape = kind == 1 && shapes ? sh : ctx->shapes[pi][n];
        if (kind == 1) cands.emplace_back(shape, 0);   // the shape's default tile (warp-specialised where it applies)
        for (int t = unit; t <= 1024; t *= 2) cands.emplace_back(shape, t);
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* mom = nullptr;
    double* amp = nullptr;
    heget_xsec_result* res = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && kind == 0) e = cudaMalloc(&mom, sizeof(double) * 4 * (n + 2) * probe_points);
    if (e == cudaSuccess && kind == 0) e = cudaMalloc(&amp, sizeof(double) * probe_points);
    if (e == cudaSuccess && kind == 1) e = cudaMalloc(&res, sizeof(heget_xsec_result));
    heget_sampler toy{HEGET_SAMPLER_TOY_PDF, 0, 0, 0, 7000.0, 100.0, 64};
    if (e == cudaSuccess && kind == 0)
        r = heget_phase_space_ex(ctx, 0x0908440300000777ull, 0, probe_points, n, &toy, mom, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, st);
    const int saved_tile = ctx->tiles[kind][pi][n], saved_shape = ctx->shapes[pi][n];
    int best = -1;
    float best_t = 1e30f;
    for (int c = 0; c < (int)cands.size(); ++c) {
        if (e != cudaSuccess || r) break;
        ctx->shapes[pi][n] = cands[c].first;
        ctx->tiles[kind][pi][n] = cands[c].second;
        auto run = [&]() {
            return kind == 0 ? heget_amp2(ctx, n, probe_points, mom, nullptr, precision, amp, st)
                             : heget_xsec_async(ctx, n, 0x0908440300000778ull, 0, probe_points, &toy, precision, res,
                                                nullptr, st);
        };
        if (run() != HEGET_OK) continue;   // e.g. shared memory of this tile exceeds the device limit
        float tmin = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaEventRecord(e0, st);
            ok = run() == HEGET_OK;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) tmin = std::min(tmin, ms);
        }
        if (ok && tmin < best_t) {
            best_t = tmin;
            best = c;
        }
    }
    if (mom) cudaFree(mom);
    if (amp) cudaFree(amp);
    if (res) cudaFree(res);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess || r || best < 0) {
        ctx->tiles[kind][pi][n] = saved_tile;
        ctx->shapes[pi][n] = saved_shape;
        if (e != cudaSuccess) return cuda_fail(e, "heget_autotune");
        return r ? r : fail(HEGET_ECUDA, "no launch shape ran");
    }
    ctx->shapes[pi][n] = cands[best].first;
    ctx->tiles[kind][pi][n] = cands[best].second;
    if (best_shape) *best_shape = cands[best].first;
    if (best_tile) *best_tile = cands[best].second;
    if (best_ms) *best_ms = best_t;
    return HEGET_OK;
}
}  // namespace

int heget_autotune(heget_ctx* ctx, int n, int precision, int kind, int64_t probe_points, int* best_tile,
                   double* best_ms) {
    return autotune_impl(ctx, n, precision, kind, probe_points, true, nullptr, best_tile, best_ms);
}

int heget_autotune_shape(heget_ctx* ctx, int n, int precision, int64_t probe_points, int* best_shape, int* best_tile,
                         double* best_ms) {
    return autotune_impl(ctx, n, precision, 1, probe_points, true, best_shape, best_tile, best_ms);
}

int heget_autotune_save(const heget_ctx* ctx, const char* path) {
    if (!ctx || !path) return fail(HEGET_EINVAL, "NULL argument");
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    std::string gpu(prop.name);
    std::replace(gpu.begin(), gpu.end(), ' ', '_');
    // keep other GPUs' lines, replace this GPU's
    std::vector<std::string> keep;
    if (FILE* f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof line, f))
            if (std::strncmp(line, gpu.c_str(), gpu.size()) != 0 || line[gpu.size()] != ' ') keep.emplace_back(line);
        std::fclose(f);
    }
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(HEGET_EINVAL, "cannot write %s", path);
    for (const auto& l : keep) std::fputs(l.c_str(), f);
    for (int kind = 0; kind < 2; ++kind)
        for (int p = 0; p < 2; ++p)
            for (int n = kMinN; n <= kMaxN; ++n) {
                const int shape = kind == 1 ? ctx->shapes[p][n] : 0;
                if (ctx->tiles[kind][p][n] > 0 || shape > 0)
                    std::fprintf(f, "%s %d %d %d %d %d\n", gpu.c_str(), n, p ? HEGET_FP64 : HEGET_FP32, kind,
                                 ctx->tiles[kind][p][n], shape);
            }
    std::fclose(f);
    return HEGET_OK;
}

int heget_autotune_load(heget_ctx* ctx, const char* path) {
    if (!ctx || !path) return fail(HEGET_EINVAL, "NULL argument");
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    std::string gpu(prop.name);
    std::replace(gpu.begin(), gpu.end(), ' ', '_');
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(HEGET_EINVAL, "cannot read %s", path);
    char name[256];
    int n, prec, kind, tile, shape;
    while (std::fscanf(f, "%255s %d %d %d %d %d", name, &n, &prec, &kind, &tile, &shape) == 6) {
        if (gpu != name) continue;
        heget_set_tile(ctx, n, prec, kind, tile);
        if (kind == 1) heget_set_shape(ctx, n, prec, shape);
    }
    std::fclose(f);
    return HEGET_OK;
}

}  // extern "C"
