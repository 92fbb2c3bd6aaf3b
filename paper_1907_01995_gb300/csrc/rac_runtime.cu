// rac_runtime.cu - per-device resources that outlive a solver handle.
//
// A handle needs a few dozen device buffers, four streams, a set of events
// and two pinned host words.  Created and destroyed per handle, these cost
// more host time (cudaMalloc / cudaFree / cudaMallocHost are synchronous and
// slow) than a whole small solve.  This file keeps them per device instead:
//   * one stream-ordered memory pool whose release threshold is unbounded, so
//     the memory a closed handle frees serves the next handle's allocations
//     without a trip to the driver (rac_trim_pool() hands it back);
//   * a free list of stream sets (streams, events, pinned status words) that
//     handles borrow at setup and return, idle, when they are destroyed.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rac_internal.h"

namespace rac {

namespace {
struct DeviceRuntime {
    cudaMemPool_t pool = nullptr;
    std::vector<StreamSet *> idle;
};
std::mutex g_mu;
std::map<int, DeviceRuntime> g_dev;   // never torn down: the driver reclaims at exit

cudaError_t grow_events(std::vector<cudaEvent_t> &v, size_t want, unsigned flags) {
    while (v.size() < want) {
        cudaEvent_t e = nullptr;
        cudaError_t r = cudaEventCreateWithFlags(&e, flags);
        if (r != cudaSuccess) return r;
        v.push_back(e);
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t runtime_pool(cudaMemPool_t *pool) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceRuntime &d = g_dev[dev];
    if (!d.pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&d.pool, &props);
        if (e != cudaSuccess) {
            d.pool = nullptr;
            return e;
        }
        uint64_t keep = ~(uint64_t)0;
        e = cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    *pool = d.pool;
    return cudaSuccess;
}

cudaError_t runtime_take_streams(StreamSet **out, size_t nfev, size_t npev) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    StreamSet *ss = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto &idle = g_dev[dev].idle;
        if (!idle.empty()) {
            ss = idle.back();
            idle.pop_back();
        }
    }
    if (!ss) {
        ss = new StreamSet();
        ss->dev = dev;
        e = cudaStreamCreateWithFlags(&ss->st, cudaStreamNonBlocking);
        for (auto &q : ss->sfs)
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&ss->h_stats, sizeof(DevStats));
        if (e == cudaSuccess) e = cudaMallocHost(&ss->h_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&ss->h_aux, 4 * sizeof(double));
        if (e != cudaSuccess) {
            runtime_give_streams(ss);   // keeps what was made for a later handle
            return e;
        }
    }
    e = grow_events(ss->fev, nfev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = grow_events(ss->pev, npev, cudaEventDefault);
    if (e != cudaSuccess) {
        runtime_give_streams(ss);
        return e;
    }
    *out = ss;
    return cudaSuccess;
}

void runtime_give_streams(StreamSet *ss) {
    if (!ss) return;
    if (!ss->st || !ss->ev || !ss->h_stats || !ss->h_err || !ss->h_aux) {
        // incomplete set (creation failed part-way): release what it holds
        for (auto q : ss->sfs)
            if (q) cudaStreamDestroy(q);
        if (ss->st) cudaStreamDestroy(ss->st);
        if (ss->ev) cudaEventDestroy(ss->ev);
        for (auto e : ss->fev) cudaEventDestroy(e);
        for (auto e : ss->pev) cudaEventDestroy(e);
        if (ss->h_stats) cudaFreeHost(ss->h_stats);
        if (ss->h_err) cudaFreeHost(ss->h_err);
        if (ss->h_aux) cudaFreeHost(ss->h_aux);
        delete ss;
        return;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    g_dev[ss->dev].idle.push_back(ss);
}

// Memo of device capability queries (occupancy, cluster co-residency):
// their answers depend only on the current device and the arguments, and the
// driver calls behind them cost tens of microseconds per handle setup.
static std::mutex g_memo_mu;
static std::map<std::tuple<int, int, long long, long long, long long>, long long> g_memo;

bool memo_get(int fid, long long a, long long b, long long c, long long *v) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_memo_mu);
    auto it = g_memo.find(std::make_tuple(dev, fid, a, b, c));
    if (it == g_memo.end()) return false;
    *v = it->second;
    return true;
}
void memo_put(int fid, long long a, long long b, long long c, long long v) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_memo_mu);
    g_memo[std::make_tuple(dev, fid, a, b, c)] = v;
}

}  // namespace rac

using namespace rac;

extern "C" rac_status rac_trim_pool(void) {
    (void)cudaGetLastError();
    cudaMemPool_t pool = nullptr;
    if (runtime_pool(&pool) != cudaSuccess) return RAC_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return RAC_ERR_CUDA;
    if (cudaMemPoolTrimTo(pool, 0) != cudaSuccess) return RAC_ERR_CUDA;
    return RAC_OK;
}
