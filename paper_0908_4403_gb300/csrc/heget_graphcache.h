// heget_graphcache.h -- CUDA graphs of the mixed-n batch launch, one per
// launch-shape bucket.
//
// A batch launch of one precision is two kernels on a stream: the work-list
// kernel over (items, nitems, reqs) with `grid` blocks and `smem` bytes, and
// the per-request finalisation over (fin, nfin).  Requests of recurring sizes
// (a serving loop, a Monte Carlo loop over seeds) repeat the same bucket --
// the same argument values and launch shape, with new request contents
// uploaded into the same device buffers -- and replay its captured graph
// instead of launching the kernels one by one.  Capture happens on a private
// stream (the caller's may be the legacy default stream, which cannot be
// captured); the replay runs on the caller's stream, after the upload.  The
// cache is bounded; the oldest bucket is dropped first.  Host code, one owner
// thread per cache.
#pragma once

#include <cstring>
#include <vector>

#include <cuda_runtime.h>

namespace heget {

struct BatchGraphKey {
    int prec, alg, nitems, nfin, grid;   // alg: the work-list kernel's ordering-sum algorithm
    size_t smem;
    const void* items;
    const void* reqs;
    const void* fin;
    bool operator==(const BatchGraphKey& o) const {
        return prec == o.prec && alg == o.alg && nitems == o.nitems && nfin == o.nfin && grid == o.grid &&
               smem == o.smem && items == o.items && reqs == o.reqs && fin == o.fin;
    }
};

struct BatchGraphCache {
    static constexpr size_t kMax = 32;
    struct Entry {
        BatchGraphKey key;
        cudaGraphExec_t exec;
    };
    std::vector<Entry> entries;   // oldest first
    cudaStream_t capture = nullptr;
    long long replays = 0, captures = 0;

    void clear() {
        for (auto& e : entries) cudaGraphExecDestroy(e.exec);
        entries.clear();
    }
    void release() {
        clear();
        if (capture) cudaStreamDestroy(capture);
        capture = nullptr;
    }
    // The graph of this bucket, captured by `launch(stream)` on first use.
    // Returns a cudaError_t as int (0 on success).
    template <class Launch>
    int run(const BatchGraphKey& key, cudaStream_t st, Launch&& launch) {
        for (auto& e : entries)
            if (e.key == key) {
                ++replays;
                return (int)cudaGraphLaunch(e.exec, st);
            }
        cudaError_t err = cudaSuccess;
        if (!capture) err = cudaStreamCreateWithFlags(&capture, cudaStreamNonBlocking);
        if (err != cudaSuccess) return (int)err;
        err = cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) return (int)err;
        const int r = launch(capture);
        cudaGraph_t g = nullptr;
        err = cudaStreamEndCapture(capture, &g);
        if (r) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (err != cudaSuccess) return (int)err;
        cudaGraphExec_t exec = nullptr;
        err = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (err != cudaSuccess) return (int)err;
        if (entries.size() == kMax) {
            cudaGraphExecDestroy(entries.front().exec);
            entries.erase(entries.begin());
        }
        entries.push_back(Entry{key, exec});
        ++captures;
        return (int)cudaGraphLaunch(exec, st);
    }
};

}  // namespace heget
