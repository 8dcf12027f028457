// Process-wide launch counters and event timing of the stencil apply.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "pc_internal.h"

namespace pc {

struct TimedLaunch {
    cudaEvent_t a, b;
    int kind;  // 0 = complex64, 1 = complex128
    double nodes;     // nodes counted on the host (items without a skip flag)
    double launched;  // nodes of all items
};

static std::atomic<long long> g_launches{0}, g_apply_launches{0};
static std::atomic<int> g_timing{0};
static std::mutex g_mu;
static std::vector<TimedLaunch> g_pending;
static std::vector<cudaEvent_t> g_pool;
static long long g_timed[2] = {0, 0};
static double g_ms[2] = {0, 0}, g_nodes[2] = {0, 0}, g_launched[2] = {0, 0};

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void note_apply_launch(int n) { g_apply_launches.fetch_add(n, std::memory_order_relaxed); }
bool timing_enabled() { return g_timing.load(std::memory_order_relaxed) != 0; }

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Inside a stream capture a plain event record only orders the captured work; an external
// record becomes a node that records the event every time the graph runs.
static void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (s != nullptr && cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

void* timing_begin(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    TimedLaunch* t = new TimedLaunch();
    t->a = take_event();
    t->b = take_event();
    record(t->a, s);
    return t;
}

// Nodes of timed apply items whose skip flag is read on the device: an item of a converged system
// returns at once inside the apply kernels, so only the items that ran are added here, by a small
// kernel on the apply's stream right after its end event (inside a captured graph it is a node of
// the graph and counts on every replay).
__device__ unsigned long long g_dev_nodes[2];
static std::atomic<int> g_dev_used{0};

constexpr int kCountMax = 64;
struct SkipList {
    const int* f[kCountMax];
    int n;
};

__global__ void count_active_kernel(const __grid_constant__ SkipList L, unsigned long long per_item, int kind) {
    const int i = threadIdx.x;
    unsigned long long v = (i < L.n && !(L.f[i] != nullptr && *L.f[i])) ? per_item : 0ULL;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((i & 31) == 0 && v != 0ULL) atomicAdd(&g_dev_nodes[kind], v);
}

void timing_end(void* h, cudaStream_t s, int kind, const ApplyItem* items, int nitems, double nodes_per_item) {
    TimedLaunch* t = static_cast<TimedLaunch*>(h);
    record(t->b, s);
    t->kind = kind;
    bool flagged = false;
    for (int i = 0; i < nitems && !flagged; ++i) flagged = items[i].skip != nullptr;
    t->nodes = flagged ? 0.0 : nitems * nodes_per_item;
    t->launched = nitems * nodes_per_item;
    if (flagged) {
        g_dev_used.store(1);
        for (int i0 = 0; i0 < nitems; i0 += kCountMax) {
            SkipList L{};
            L.n = std::min(kCountMax, nitems - i0);
            for (int i = 0; i < L.n; ++i) L.f[i] = items[i0 + i].skip;
            count_active_kernel<<<1, kCountMax, 0, s>>>(L, (unsigned long long)nodes_per_item, kind);
            note_launch();
        }
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(*t);
    delete t;
}

// Timing inside captured graphs: the event pairs recorded during a capture are kept with the
// graph and read after every replay (the replayed graph records the same events again).
struct TimedSet {
    size_t mark = 0;
    std::vector<TimedLaunch> recs;
};

TimedSet* timing_capture_begin() {
    std::lock_guard<std::mutex> lk(g_mu);
    TimedSet* t = new TimedSet();
    t->mark = g_pending.size();
    return t;
}

void timing_capture_end(TimedSet* t) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (t->mark < g_pending.size()) {
        t->recs.assign(g_pending.begin() + (long)t->mark, g_pending.end());
        g_pending.resize(t->mark);
    }
}

void timing_replayed(TimedSet* t) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : t->recs) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_ms[r.kind] += ms;
            g_timed[r.kind] += 1;
            g_nodes[r.kind] += r.nodes;
            g_launched[r.kind] += r.launched;
        } else {
            cudaGetLastError();  // an unreadable timing is dropped, not reported to later calls
        }
    }
}

void timing_free(TimedSet* t) {
    if (!t) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : t->recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    delete t;
}

long long launch_count() { return g_launches.load(); }
long long apply_launch_count() { return g_apply_launches.load(); }

static void drain() {
    for (auto& t : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(t.b);
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            g_ms[t.kind] += ms;
            g_timed[t.kind] += 1;
            g_nodes[t.kind] += t.nodes;
            g_launched[t.kind] += t.launched;
        } else {
            cudaGetLastError();
        }
        g_pool.push_back(t.a);
        g_pool.push_back(t.b);
    }
    g_pending.clear();
}

// FP64 FMA throughput: every thread runs 8 independent chains a = fma(a, m, c) (m just below 1, so
// the values stay bounded); the 8-way ILP and 32 warps per SM keep the FP64 pipe saturated.  The
// sum is stored only under a condition that never holds, which keeps every chain live.
__global__ void fp64_fma_rate_kernel(int iters, double seed, double* sink) {
    double a[8];
    const double m = 1.0 - 1e-9 * (double)(1 + (threadIdx.x & 7));
    const double c = 1e-12 * seed;
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + (double)j + 1e-3 * (double)threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += a[j];
    if (t == -1.0) *sink = t;
}

}  // namespace pc

using namespace pc;

extern "C" {

int pc_fp64_peak(double seconds, double* tflops, double* fma_per_s) {
    if (!tflops || !(seconds > 0) || seconds > 60) return fail(PC_EINVAL, "pc_fp64_peak: bad argument");
    const int sms = device_sm_count();
    const int threads = 512, blocks = 2 * sms;
    double* sink = nullptr;
    PC_CUDA_TRY(cudaMalloc(&sink, sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 256;
    double best = 0.0;
    int rc = PC_OK;
    for (int round = 0; round < 12 && rc == PC_OK; ++round) {
        cudaEventRecord(e0, 0);
        fp64_fma_rate_kernel<<<blocks, threads, 0, 0>>>(iters, 1.0 + round, sink);
        note_launch();
        cudaEventRecord(e1, 0);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fp64_fma_rate_kernel");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fmas = (double)blocks * threads * 8.0 * iters;
        if (ms > 0.f && round >= 2) best = std::fmax(best, fmas / (ms * 1e-3));
        // grow the launch until it runs for about `seconds` / 4 (the last passes are the measurement)
        if (ms > 0.f && ms * 1e-3 < seconds / 4) {
            const double f = std::fmin(16.0, (seconds / 4) / (ms * 1e-3));
            iters = (int)std::fmin(1e9, iters * f);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != PC_OK) return rc;
    *tflops = 2.0 * best / 1e12;
    if (fma_per_s) *fma_per_s = best;
    return PC_OK;
}

int pc_stats_timing(int enable) {
    g_timing.store(enable ? 1 : 0);
    return PC_OK;
}

int pc_stats_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    g_launches = 0;
    g_apply_launches = 0;
    g_timed[0] = g_timed[1] = 0;
    g_ms[0] = g_ms[1] = 0;
    g_nodes[0] = g_nodes[1] = 0;
    g_launched[0] = g_launched[1] = 0;
    if (g_dev_used.load()) {
        const unsigned long long zero[2] = {0ULL, 0ULL};
        cudaDeviceSynchronize();
        PC_CUDA_TRY(cudaMemcpyToSymbol(g_dev_nodes, zero, sizeof(zero)));
    }
    return PC_OK;
}

int pc_stats_get(pc_stats* out) {
    if (!out) return fail(PC_EINVAL, "pc_stats_get: null");
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    unsigned long long dev[2] = {0ULL, 0ULL};
    if (g_dev_used.load()) {
        PC_CUDA_TRY(cudaDeviceSynchronize());
        PC_CUDA_TRY(cudaMemcpyFromSymbol(dev, g_dev_nodes, sizeof(dev)));
    }
    out->launches = g_launches.load();
    out->apply_launches = g_apply_launches.load();
    for (int k = 0; k < 2; ++k) {
        out->apply_timed[k] = g_timed[k];
        out->apply_ms[k] = g_ms[k];
        out->apply_nodes[k] = g_nodes[k] + (double)dev[k];
        out->apply_nodes_launched[k] = g_launched[k];
    }
    return PC_OK;
}

}  // extern "C"
