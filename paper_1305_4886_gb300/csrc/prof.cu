// prof.cu -- optional per-kernel timing with CUDA events (a measurement aid
// for roofline reporting).  Off by default; when enabled, selected launches
// are bracketed by an event pair recorded on the launch's own stream, and
// the algorithmic flops / bytes of the launch are tallied per kernel class.
// Reading the counters synchronises on the recorded events.
#include <mutex>
#include <vector>

#include "internal.h"

namespace gp {

namespace {
struct Rec {
    cudaEvent_t a = nullptr, b = nullptr;
    int cls = 0;
    double flops = 0.0, bytes = 0.0;
};
std::mutex g_mu;
std::vector<Rec> g_pool;
size_t g_used = 0;
bool g_on = false;
int64_t g_dropped = 0;
constexpr size_t POOL = 16384;
}  // namespace

int prof_start(cudaStream_t s) {
    if (!g_on) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_used >= g_pool.size()) {
        ++g_dropped;
        return -1;
    }
    Rec &r = g_pool[g_used];
    if (cudaEventRecord(r.a, s) != cudaSuccess) return -1;
    return static_cast<int>(g_used++);
}

void prof_stop(int idx, cudaStream_t s, int cls, double flops, double bytes) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec &r = g_pool[idx];
    r.cls = cls;
    r.flops = flops;
    r.bytes = bytes;
    cudaEventRecord(r.b, s);
}

}  // namespace gp

using namespace gp;

extern "C" {

int gp_prof_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (on && g_pool.empty()) {
        g_pool.resize(POOL);
        for (auto &r : g_pool) {
            if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
                g_pool.clear();
                return GP_ERR_CUDA;
            }
        }
    }
    g_used = 0;
    g_dropped = 0;
    g_on = on != 0;
    return GP_OK;
}

int gp_prof_read(int cls, double *ms_total, int64_t *launches, double *flops, double *bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    double ms = 0.0, fl = 0.0, by = 0.0;
    int64_t cnt = 0;
    for (size_t i = 0; i < g_used; ++i) {
        Rec &r = g_pool[i];
        if (r.cls != cls) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return GP_ERR_CUDA;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return GP_ERR_CUDA;
        ms += t;
        fl += r.flops;
        by += r.bytes;
        ++cnt;
    }
    if (ms_total) *ms_total = ms;
    if (launches) *launches = cnt;
    if (flops) *flops = fl;
    if (bytes) *bytes = by;
    return g_dropped ? GP_ERR_WORKSPACE : GP_OK;
}

}  // extern "C"
