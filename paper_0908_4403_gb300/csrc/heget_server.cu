// heget_server.cu -- continuous-batching request server over the mixed-n
// batch kernel.
//
// A worker thread owns one CUDA stream.  Requests wait in a FIFO until a slot
// is free and the device arena has room for their tile partials and result
// (admission); admitted requests are cut into the tiles heget_xsec would use,
// and every launch takes tiles round-robin from all admitted requests until
// its work budget is filled, so requests that arrive while others run join
// the next launch and share the GPU with them.  A request is finalised in the
// launch that carries its last tile; its result is copied to pinned host
// memory and reported when that launch's completion event has fired.  Up to
// two launches are in flight, so the host builds launch k+1 while the GPU runs
// launch k.  Every wait is bounded (condition-variable timeouts, event polls).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "heget_arena.h"
#include "heget_kernels.cuh"
#include "heget_internal.h"

using namespace heget;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// FP32-flop equivalents per point: the amplitudes of the server's
// ordering-sum algorithm -- the tree (2^n lanes, 28 flop per step, 16 per
// closure) or the subset recursion met in the middle (12 multiply-adds per
// current term and Q product, 8 per contraction term over the sets of n/2
// photons, for every helicity assignment of each set) -- plus the
// phase-space generation (~1e3 FP64 operations at ~1/64 of the FP32 rate).
// FP64 amplitude flops count as FP32 ones: weighting them by the pipes'
// rate ratio made FP64 launches too small to keep the GPU busy (a sweep of
// weights 1, 4, 16 on the serving traces: 1 gave the highest throughput and
// the lowest latencies with both algorithms).
double binom(int n, int k) {
    double c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}
double point_cost(int n, int alg) {
    double amp = 0;
    if (alg == kAlgSubset) {
        const int m = n / 2, mk = n - m;
        double fma = 0;
        for (int k = 1; k <= m; ++k) fma += binom(n, k) * (1 << k) * (k >= 2 ? 12.0 * k + 12.0 : 12.0);
        for (int k = 1; k < mk; ++k) fma += binom(n, k) * (1 << k) * (k >= 2 ? 12.0 * k + 12.0 : 12.0);
        if (mk >= 2) fma += binom(n, mk) * (1 << mk) * 12.0 * mk;
        fma += binom(n, m) * (1 << n) * 8.0;
        amp = 2.0 * fma;
    } else {
        double f = 1;
        for (int i = 2; i <= n; ++i) f *= i;
        double steps = 0, term = 1;
        for (int l = 1; l <= n - 1; ++l) {
            term *= (n - l + 1);
            if (l >= 2) steps += term;
        }
        amp = (double)(1 << n) * (28.0 * steps + 16.0 * f);
    }
    return amp + 6.4e4;
}

struct Req {
    uint64_t ticket;
    heget_request q;
    int tile, ntiles, next_tile;
    size_t arena_off, arena_bytes;
    double t_submit, t_admit;
};

struct Launch {
    cudaEvent_t done = nullptr;
    std::vector<Req*> finished;          // requests finalised in this launch
    std::vector<int> result_slot;        // their slots in the pinned result array
    unsigned char* host = nullptr;       // pinned staging (items + request tables)
    unsigned char* dev = nullptr;
    size_t cap = 0;
    bool busy = false;
};

}  // namespace

struct heget_server {
    heget_ctx* ctx = nullptr;
    heget_server_cfg cfg{};
    cudaStream_t stream = nullptr;
    unsigned char* arena_dev = nullptr;
    heget::Arena arena;
    heget_xsec_result* results_host = nullptr;   // pinned, one slot per admitted request
    std::vector<int> free_slots;
    Launch launches[2];
    int next_launch = 0;
    bool graphs = false;                         // the context's graph setting when the server started
    int alg = 0;                                 // the context's ordering-sum algorithm when the server started
    heget::BatchGraphCache graph_cache;          // per-round launches by launch-shape bucket (worker thread)

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::vector<Req*> active;                    // admitted, tiles still to launch
    std::map<uint64_t, heget_result> done;
    std::map<uint64_t, int> state;               // 0 pending, 1 admitted, 2 done
    uint64_t next_ticket = 1;
    bool stopping = false;
    int admitted = 0;
    std::thread worker;
    std::atomic<int> fatal{0};

    void run();
    bool admit_locked(Req* r);
    int build_and_launch(Launch& L);
    void complete(Launch& L, int status);
    void fail_all(Launch& L);
};

bool heget_server::admit_locked(Req* r) {
    if (admitted >= cfg.max_inflight || free_slots.empty()) return false;
    const size_t bytes = (size_t)r->ntiles * sizeof(Partial) + sizeof(heget_xsec_result) + 256;
    size_t off = 0;
    if (!arena.alloc(bytes, &off)) return false;
    r->arena_off = off;
    r->arena_bytes = bytes;
    r->t_admit = now_s();
    ++admitted;
    state[r->ticket] = 1;
    return true;
}

void heget_server::complete(Launch& L, int status) {
    std::lock_guard<std::mutex> lock(mu);
    const double t = now_s();
    for (size_t k = 0; k < L.finished.size(); ++k) {
        Req* r = L.finished[k];
        heget_result res{};
        res.status = status;
        if (status == HEGET_OK) res.result = results_host[L.result_slot[k]];
        res.t_submit = r->t_submit;
        res.t_admit = r->t_admit;
        res.t_done = t;
        done[r->ticket] = res;
        state[r->ticket] = 2;
        if (L.result_slot[k] >= 0) free_slots.push_back(L.result_slot[k]);
        arena.release(r->arena_off, r->arena_bytes);
        --admitted;
        delete r;
    }
    L.finished.clear();
    L.result_slot.clear();
    L.busy = false;
    cv_done.notify_all();
    cv_work.notify_all();
}

// Builds one launch from the admitted requests and enqueues it: both
// precisions' work lists share one staging area and one upload.  Returns the
// number of tiles launched (0: nothing to do) or -1 on a CUDA error.
int heget_server::build_and_launch(Launch& L) {
    std::vector<Req*> take;
    {
        std::lock_guard<std::mutex> lock(mu);
        while (!pending.empty() && admit_locked(pending.front())) {
            active.push_back(pending.front());
            pending.pop_front();
        }
        take = active;
    }
    if (take.empty()) return 0;
    // round-robin tiles under the work budget, and at least two tiles per SM
    // when the admitted requests have them (a launch of fewer tiles leaves SMs
    // idle however long its tiles run: large-n FP64 tiles take up to seconds)
    std::vector<int> ntake(take.size(), 0);
    double budget = cfg.max_launch_work;
    const long long min_tiles = 2ll * ctx->num_sms;
    long long taken = 0;
    auto more = [&] { return budget > 0 || taken < min_tiles; };
    for (bool any = true; more() && any;) {
        any = false;
        for (size_t i = 0; i < take.size() && more(); ++i) {
            Req* r = take[i];
            if (r->next_tile + ntake[i] >= r->ntiles) continue;
            ++ntake[i];
            ++taken;
            budget -= point_cost(r->q.n, alg) * r->tile;
            any = true;
        }
    }
    struct Part {
        std::vector<WorkItem> items;
        std::vector<BatchReq> br, fin;
        size_t smem = 0, off_items = 0, off_br = 0, off_fin = 0;
    } part[2];
    std::vector<Req*> finishing;
    for (size_t i = 0; i < take.size(); ++i) {
        Req* r = take[i];
        if (ntake[i] == 0) continue;
        Part& P = part[r->q.precision == HEGET_FP64];
        BatchReq b{};
        b.seed = r->q.seed;
        b.i0 = r->q.i0;
        b.S = sampler_args(&r->q.sampler);
        b.ph = physics_of(ctx, r->q.n);
        b.w_out = nullptr;
        b.parts = reinterpret_cast<Partial*>(arena_dev + r->arena_off);
        b.result = reinterpret_cast<heget_xsec_result*>(arena_dev + r->arena_off + (size_t)r->ntiles * sizeof(Partial));
        b.n = r->q.n;
        b.tile = r->tile;
        b.ntiles = r->ntiles;
        for (int k = 0; k < ntake[i]; ++k) {
            const long long start = (long long)(r->next_tile + k) * r->tile;
            P.items.push_back(
                WorkItem{(int)P.br.size(), r->q.n, (int)std::min<long long>(r->tile, r->q.N - start), 0, start});
        }
        P.br.push_back(b);
        if (r->next_tile + ntake[i] >= r->ntiles) {
            P.fin.push_back(b);
            finishing.push_back(r);
        }
        const size_t sm = batch_tile_smem(r->q.n, r->q.precision, alg, r->tile);
        P.smem = std::max(P.smem, sm);
    }
    size_t bytes = 0;
    for (Part& P : part) {
        P.off_items = bytes;
        bytes += align16(P.items.size() * sizeof(WorkItem));
        P.off_br = bytes;
        bytes += align16(P.br.size() * sizeof(BatchReq));
        P.off_fin = bytes;
        bytes += align16(P.fin.size() * sizeof(BatchReq));
    }
    if (bytes > L.cap) {
        graph_cache.clear();   // graph arguments point into the launch buffers
        if (L.host) cudaFreeHost(L.host);
        if (L.dev) cudaFree(L.dev);
        L.host = nullptr;
        L.dev = nullptr;
        L.cap = 0;
        size_t c = 1 << 16;
        while (c < bytes) c *= 2;
        if (cudaMallocHost(&L.host, c) != cudaSuccess || cudaMalloc(&L.dev, c) != cudaSuccess) return -1;
        L.cap = c;
    }
    for (Part& P : part) {
        std::memcpy(L.host + P.off_items, P.items.data(), P.items.size() * sizeof(WorkItem));
        std::memcpy(L.host + P.off_br, P.br.data(), P.br.size() * sizeof(BatchReq));
        std::memcpy(L.host + P.off_fin, P.fin.data(), P.fin.size() * sizeof(BatchReq));
    }
    if (cudaMemcpyAsync(L.dev, L.host, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) return -1;
    int launched = 0;
    for (int pi = 0; pi < 2; ++pi) {
        Part& P = part[pi];
        if (P.items.empty()) continue;
        const int nitems = (int)P.items.size();
        const int grid = std::max(1, std::min(nitems, 8 * ctx->num_sms));
        const WorkItem* items_d = reinterpret_cast<const WorkItem*>(L.dev + P.off_items);
        const BatchReq* br_d = reinterpret_cast<const BatchReq*>(L.dev + P.off_br);
        const BatchReq* fin_d = reinterpret_cast<const BatchReq*>(L.dev + P.off_fin);
        const int nfin = (int)P.fin.size();
        auto launch = [&](cudaStream_t s2, bool set_attr) {
            int rr = pi == 0 ? launch_batch_f32(items_d, nitems, br_d, P.smem, grid, alg, s2, set_attr)
                             : launch_batch_f64(items_d, nitems, br_d, P.smem, grid, alg, s2, set_attr);
            if (!rr && nfin > 0) rr = launch_batch_finalize(fin_d, nfin, s2);
            return rr;
        };
        int r;
        if (graphs) {
            r = pi == 0 ? prepare_batch_f32(P.smem, alg) : prepare_batch_f64(P.smem, alg);
            if (!r)
                r = graph_cache.run(BatchGraphKey{pi == 0 ? HEGET_FP32 : HEGET_FP64, alg, nitems, nfin, grid, P.smem,
                                                  items_d, br_d, fin_d},
                                    stream, [&](cudaStream_t s2) { return launch(s2, false); });
        } else {
            r = launch(stream, true);
        }
        if (r) return -1;
        launched += nitems;
    }
    for (size_t i = 0; i < take.size(); ++i) take[i]->next_tile += ntake[i];
    {
        std::lock_guard<std::mutex> lock(mu);
        for (Req* r : finishing) {
            const int slot = free_slots.back();
            free_slots.pop_back();
            L.finished.push_back(r);
            L.result_slot.push_back(slot);
            active.erase(std::find(active.begin(), active.end(), r));
        }
    }
    for (size_t k = 0; k < L.finished.size(); ++k) {
        Req* r = L.finished[k];
        if (cudaMemcpyAsync(results_host + L.result_slot[k],
                            arena_dev + r->arena_off + (size_t)r->ntiles * sizeof(Partial),
                            sizeof(heget_xsec_result), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
            return -1;
    }
    if (cudaEventRecord(L.done, stream) != cudaSuccess) return -1;
    L.busy = true;
    return launched;
}

// A CUDA error ends the server's work: every admitted request completes with
// HEGET_ECUDA and nothing more is launched.
void heget_server::fail_all(Launch& L) {
    fatal = 1;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (Req* r : active) {
            if (std::find(L.finished.begin(), L.finished.end(), r) != L.finished.end()) continue;
            L.finished.push_back(r);
            L.result_slot.push_back(-1);
        }
        active.clear();
        stopping = true;
    }
    complete(L, HEGET_ECUDA);
    for (Launch& O : launches)
        if (O.busy) complete(O, HEGET_ECUDA);
}

void heget_server::run() {
    DeviceGuard dg(ctx->device);
    bool stalled = false;
    for (;;) {
        // retire finished launches (oldest first)
        for (int k = 0; k < 2; ++k) {
            Launch& L = launches[(next_launch + k) % 2];
            if (L.busy) {
                const cudaError_t q = cudaEventQuery(L.done);
                if (q == cudaSuccess) complete(L, HEGET_OK);
                else if (q != cudaErrorNotReady) {
                    cudaStreamSynchronize(stream);   // nothing of this server runs on after the error
                    fail_all(L);
                }
            }
        }
        {
            std::unique_lock<std::mutex> lock(mu);
            const bool idle = active.empty() && pending.empty();
            if (stopping && idle && !launches[0].busy && !launches[1].busy) break;
            const bool need_slot = launches[next_launch].busy;
            if (need_slot || (idle && !stopping) || stalled)
                cv_work.wait_for(lock, std::chrono::microseconds(need_slot || stalled ? 50 : 2000));
            stalled = false;
            if (stopping && !pending.empty()) {   // cancel what never started
                for (Req* r : pending) {
                    heget_result res{};
                    res.status = HEGET_EBUSY;
                    res.t_submit = r->t_submit;
                    res.t_done = now_s();
                    done[r->ticket] = res;
                    state[r->ticket] = 2;
                    delete r;
                }
                pending.clear();
                cv_done.notify_all();
            }
        }
        Launch& L = launches[next_launch];
        if (L.busy) continue;
        const int got = build_and_launch(L);
        if (got < 0) {
            cudaStreamSynchronize(stream);
            fail_all(L);
        } else if (got > 0) {
            next_launch ^= 1;
        } else {
            stalled = true;   // requests wait for admission: let a launch retire first
        }
    }
}

extern "C" {

int heget_server_start(heget_ctx* ctx, const heget_server_cfg* cfg_in, heget_server** out) {
    if (!ctx || !out) return fail(HEGET_EINVAL, "NULL argument");
    *out = nullptr;
    heget_server_cfg cfg = cfg_in ? *cfg_in : heget_server_cfg{0, 0, 0, 0};
    if (cfg.max_inflight <= 0) cfg.max_inflight = 256;
    if (cfg.max_launch_work <= 0) cfg.max_launch_work = 2e11;
    if (cfg.hbm_reserve_frac <= 0 || cfg.hbm_reserve_frac >= 1) cfg.hbm_reserve_frac = 0.1;
    DeviceGuard dg(ctx->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    const size_t usable = (size_t)((double)free_b * (1.0 - cfg.hbm_reserve_frac));
    size_t arena = cfg.arena_bytes ? cfg.arena_bytes : std::min<size_t>(usable, (size_t)256 << 20);
    if (arena > usable) return fail(HEGET_ENOMEM, "arena of %zu bytes exceeds usable free HBM (%zu)", arena, usable);
    heget_server* s = new heget_server();
    s->ctx = ctx;
    s->graphs = ctx->graphs != 0;
    s->alg = ctx->alg;
    s->cfg = cfg;
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_dev, arena);
    if (e == cudaSuccess) e = cudaMallocHost(&s->results_host, sizeof(heget_xsec_result) * cfg.max_inflight);
    for (auto& L : s->launches)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        heget_server_stop(s);
        return cuda_fail(e, "heget_server_start");
    }
    s->arena.init(arena);
    for (int k = cfg.max_inflight - 1; k >= 0; --k) s->free_slots.push_back(k);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return HEGET_OK;
}

int heget_submit(heget_server* s, const heget_request* q, uint64_t* ticket) {
    if (!s || !q || !ticket) return fail(HEGET_EINVAL, "NULL argument");
    int r = check_common(s->ctx, q->n, q->N);
    if (!r) r = check_precision(q->precision);
    if (!r) r = check_sampler(&q->sampler);
    if (!r) r = check_range(q->i0, q->N);
    if (r) return r;
    if (q->N < 1) return fail(HEGET_EINVAL, "a request needs N >= 1");
    const int t = s->ctx->tiles[1][q->precision == HEGET_FP64][q->n];
    const int tile = t > 0 ? t : batch_default_tile(q->n, q->precision, s->alg);
    const long long ntiles = (q->N + tile - 1) / tile;
    if (ntiles > (long long)(s->arena.size / sizeof(Partial)))
        return fail(HEGET_ENOMEM, "request of %lld tiles cannot fit the arena of %zu bytes", ntiles, s->arena.size);
    Req* rq = new Req();
    rq->q = *q;
    rq->tile = tile;
    rq->ntiles = (int)ntiles;
    rq->next_tile = 0;
    rq->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) {
            delete rq;
            return fail(HEGET_EBUSY, "server is stopping");
        }
        const size_t need = (size_t)rq->ntiles * sizeof(Partial) + sizeof(heget_xsec_result) + 256;
        if (need > s->arena.size) {
            delete rq;
            return fail(HEGET_ENOMEM, "request needs %zu bytes of device state, arena holds %zu", need, s->arena.size);
        }
        rq->ticket = s->next_ticket++;
        s->state[rq->ticket] = 0;
        s->pending.push_back(rq);
        *ticket = rq->ticket;
    }
    s->cv_work.notify_all();
    return HEGET_OK;
}

int heget_poll(heget_server* s, uint64_t ticket, heget_result* out) {
    if (!s || !out) return fail(HEGET_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto st = s->state.find(ticket);
    if (st == s->state.end()) return fail(HEGET_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (st->second != 2) return HEGET_EBUSY;
    auto it = s->done.find(ticket);
    *out = it->second;
    s->done.erase(it);
    s->state.erase(st);
    return HEGET_OK;
}

int heget_wait(heget_server* s, uint64_t ticket, double timeout_s, heget_result* out) {
    if (!s || !out) return fail(HEGET_EINVAL, "NULL argument");
    if (!(timeout_s >= 0)) return fail(HEGET_EINVAL, "timeout_s must be >= 0");
    timeout_s = std::min(timeout_s, 1e7);   // keeps the deadline inside the clock's range
    std::unique_lock<std::mutex> lock(s->mu);
    auto st = s->state.find(ticket);
    if (st == s->state.end()) return fail(HEGET_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s));
    const bool fin = s->cv_done.wait_until(lock, deadline, [&] {
        auto f = s->state.find(ticket);
        return f == s->state.end() || f->second == 2;
    });
    if (s->state.find(ticket) == s->state.end())   // claimed by a concurrent poll
        return fail(HEGET_ENOTFOUND, "ticket %llu released while waiting", (unsigned long long)ticket);
    if (!fin) return fail(HEGET_ETIMEOUT, "ticket %llu not done within %.3f s", (unsigned long long)ticket, timeout_s);
    auto it = s->done.find(ticket);
    *out = it->second;
    s->done.erase(it);
    s->state.erase(ticket);
    return HEGET_OK;
}

int heget_server_stop(heget_server* s) {
    if (!s) return fail(HEGET_EINVAL, "NULL argument");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    DeviceGuard dg(s->ctx->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->graph_cache.release();
    for (auto& L : s->launches) {
        if (L.done) cudaEventDestroy(L.done);
        if (L.host) cudaFreeHost(L.host);
        if (L.dev) cudaFree(L.dev);
    }
    for (Req* r : s->active) delete r;
    for (Req* r : s->pending) delete r;
    if (s->results_host) cudaFreeHost(s->results_host);
    if (s->arena_dev) cudaFree(s->arena_dev);
    if (s->stream) cudaStreamDestroy(s->stream);
    const int bad = s->fatal.load();
    delete s;
    return bad ? fail(HEGET_ECUDA, "a server launch failed") : HEGET_OK;
}

}  // extern "C"

