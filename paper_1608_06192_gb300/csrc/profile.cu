// Optional per-kernel timing with CUDA events on the launching stream.
//
// When enabled, every instrumented launch is bracketed by two events recorded
// on its own stream; dcrf_profile_read synchronises on them and reports, per
// kernel name, the number of launches and the summed device time.  Solvers
// launch eagerly (no internal graph) while profiling is on, so that every
// launch has its own pair of events.
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

struct Rec {
    int id;
    cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

const char *kNames[] = {"embed_insert", "lattice_finalize", "neighbours", "splat_dense", "blur_pass", "slice",
                        "fw_pixel", "fw_latdot", "fw_alpha", "fw_latupd", "fw_lin", "lp_sort",
                        "lp_runs", "lp_splat", "lp_neighbours", "lp_blur", "lp_slice", "lp_combine",
                        "lp_project", "lp_local", "fw_blur", "dcneg_pixel"};
constexpr int kNumNames = sizeof(kNames) / sizeof(kNames[0]);

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

bool dcrf_profiling() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

ProfScope::ProfScope(int id, cudaStream_t s) : id_(id), s_(s), a_(nullptr) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on || id < 0 || id >= kNumNames) return;
    a_ = get_event();
    cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    cudaEventRecord(b, s_);
    g_recs.push_back(Rec{id_, (cudaEvent_t)a_, b});
}

extern "C" dcrf_status dcrf_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return DCRF_OK;
}

extern "C" int dcrf_profile_read(const char **names, int64_t *launches, double *ms, int capacity) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<int64_t> cnt(kNumNames, 0);
    std::vector<double> tot(kNumNames, 0.0);
    for (auto &r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            cnt[r.id] += 1;
            tot[r.id] += t;
        }
    }
    int k = 0;
    for (int i = 0; i < kNumNames && k < capacity; ++i) {
        if (cnt[i] == 0) continue;
        if (names) names[k] = kNames[i];
        if (launches) launches[k] = cnt[i];
        if (ms) ms[k] = tot[i];
        ++k;
    }
    return k;
}
