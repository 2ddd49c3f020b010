// Kernel-level profiler of a context: launch counts per kernel (always on)
// and, when timing is enabled, the device time of every launch from a pair of
// CUDA events recorded on the launch stream around it.  Used by the benchmark
// to time the dominant kernel inside the timed region.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace bt {

struct Profiler {
    bool timing = false;
    long long launches[K_COUNT] = {};
    double ms[K_COUNT] = {};
    struct Pending {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<cudaEvent_t> open;  // start events of launches in flight (per begin/end pair)
};

static thread_local Profiler *g_prof = nullptr;

static const char *const kNames[K_COUNT] = {
    "push_maps", "minmax", "box_rule", "igf_corner", "igf_sum", "deposit", "acc_to_rho",
    "fft_x", "fft_yz", "fft_zsolve", "fft_xinv", "green_x", "green_yz", "field",
    "gather_kick_push", "moments", "twiddle", "efix", "sort", "adjoint_particles",
    "adjoint_grid", "zero_acc", "redeposit"};

const char *kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? kNames[id] : ""; }

ProfScope::ProfScope(Profiler *p) : prev(g_prof) { g_prof = p; }
ProfScope::~ProfScope() { g_prof = prev; }

static cudaEvent_t take_event(Profiler *p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void prof_begin(int id, cudaStream_t s) {
    Profiler *p = g_prof;
    if (!p) return;
    p->launches[id] += 1;
    if (!p->timing) return;
    cudaEvent_t a = take_event(p);
    if (a) cudaEventRecord(a, s);
    p->open.push_back(a);
}

void prof_end(int id, cudaStream_t s) {
    Profiler *p = g_prof;
    if (!p || !p->timing || p->open.empty()) return;
    cudaEvent_t a = p->open.back();
    p->open.pop_back();
    cudaEvent_t b = take_event(p);
    if (b) cudaEventRecord(b, s);
    if (a && b) p->pending.push_back({id, a, b});
}

Profiler *profiler_new() { return new Profiler(); }

bool profiler_timing(const Profiler *p) { return p && p->timing; }

void profiler_free(Profiler *p) {
    if (!p) return;
    for (auto &q : p->pending) {
        cudaEventDestroy(q.a);
        cudaEventDestroy(q.b);
    }
    for (auto e : p->pool) cudaEventDestroy(e);
    delete p;
}

void profiler_enable(Profiler *p, bool on) {
    for (auto &q : p->pending) {
        p->pool.push_back(q.a);
        p->pool.push_back(q.b);
    }
    p->pending.clear();
    p->open.clear();
    for (int k = 0; k < K_COUNT; ++k) {
        p->launches[k] = 0;
        p->ms[k] = 0.0;
    }
    p->timing = on;
}

cudaError_t profiler_read(Profiler *p, double *ms, long long *launches, int cap) {
    for (auto &q : p->pending) {
        cudaError_t e = cudaEventSynchronize(q.b);
        if (e != cudaSuccess) return e;
        float t = 0.f;
        e = cudaEventElapsedTime(&t, q.a, q.b);
        if (e != cudaSuccess) return e;
        p->ms[q.id] += t;
        p->pool.push_back(q.a);
        p->pool.push_back(q.b);
    }
    p->pending.clear();
    for (int k = 0; k < K_COUNT && k < cap; ++k) {
        if (ms) ms[k] = p->ms[k];
        if (launches) launches[k] = p->launches[k];
    }
    return cudaSuccess;
}

}  // namespace bt
