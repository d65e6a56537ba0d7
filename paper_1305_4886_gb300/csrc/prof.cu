// prof.cu -- optional per-kernel timing with CUDA events (a measurement aid
// for roofline reporting).  Off by default; when enabled, selected launches
// are bracketed by an event pair recorded on the launch's own stream, and
// the algorithmic flops / bytes of the launch are tallied per kernel class.
// The event pool grows on demand in blocks of 4096 pairs, up to
// PROF_MAX_LAUNCHES; launches beyond that are counted as dropped.  Reading
// the counters synchronises on the recorded events.
#include <deque>
#include <mutex>

#include "internal.h"

namespace gp {

namespace {
struct Rec {
    cudaEvent_t a = nullptr, b = nullptr;
    int cls = 0;
    double flops = 0.0, bytes = 0.0;
};
std::mutex g_mu;
std::deque<Rec> g_pool;  // a deque keeps references stable while it grows
size_t g_used = 0;
bool g_on = false;
int64_t g_dropped = 0;
constexpr size_t GROW = 4096;
constexpr size_t PROF_MAX_LAUNCHES = size_t(1) << 20;

// Adds GROW event pairs; false if the cap is reached or CUDA refuses.
bool grow_locked() {
    if (g_pool.size() + GROW > PROF_MAX_LAUNCHES) return false;
    for (size_t i = 0; i < GROW; ++i) {
        Rec r;
        if (cudaEventCreate(&r.a) != cudaSuccess) return false;
        if (cudaEventCreate(&r.b) != cudaSuccess) {
            cudaEventDestroy(r.a);
            return false;
        }
        g_pool.push_back(r);
    }
    return true;
}
}  // namespace

int prof_start(cudaStream_t s) {
    if (!g_on) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_used >= g_pool.size() && !grow_locked()) {
        ++g_dropped;
        return -1;
    }
    Rec &r = g_pool[g_used];
    r.cls = -1;  // counted once prof_stop has recorded its end
    if (cudaEventRecord(r.a, s) != cudaSuccess) {
        ++g_dropped;
        return -1;
    }
    return static_cast<int>(g_used++);
}

void prof_stop(int idx, cudaStream_t s, int cls, double flops, double bytes) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec &r = g_pool[idx];
    r.cls = cls;
    r.flops = flops;
    r.bytes = bytes;
    if (cudaEventRecord(r.b, s) != cudaSuccess) {
        r.cls = -1;  // unusable: left out of the sums
        ++g_dropped;
    }
}

thread_local int t_contract_cls = GP_PROF_CONTRACT;
int prof_contract_class() { return t_contract_cls; }
ProfContractRole::ProfContractRole(int cls) : prev(t_contract_cls) { t_contract_cls = cls; }
ProfContractRole::~ProfContractRole() { t_contract_cls = prev; }

static bool class_matches(int want, int have) {
    if (want == have) return true;
    return want == GP_PROF_CONTRACT &&
           (have == GP_PROF_CONTRACT_CHOL || have == GP_PROF_CONTRACT_TRTRI ||
            have == GP_PROF_CONTRACT_LAUUM);
}

}  // namespace gp

using namespace gp;

extern "C" {

int gp_prof_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (on && g_pool.empty() && !grow_locked()) return GP_ERR_CUDA;
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
        if (r.cls < 0 || !class_matches(cls, r.cls)) continue;
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

int64_t gp_prof_dropped(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_dropped;
}

}  // extern "C"
