// prof.cu -- per-launch CUDA-event tracing (include/fcirc_prof.h), and an
// NVTX range named after the kernel around every launch (visible to
// profilers that collect NVTX; a no-op otherwise).
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fcirc_prof.h"
#include "common.hpp"
#include "prof.hpp"

namespace fcirc {

namespace {
struct Rec {
    const char *name;
    int dev;
    cudaEvent_t e0, e1;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<std::pair<int, cudaEvent_t>> g_pool;

cudaEvent_t get_event(int dev)
{
    for (size_t i = 0; i < g_pool.size(); ++i)
        if (g_pool[i].first == dev) {
            cudaEvent_t e = g_pool[i].second;
            g_pool.erase(g_pool.begin() + i);
            return e;
        }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

bool prof_on() { return g_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(const char *name, cudaStream_t s) : name_(name), s_(s)
{
    nvtxRangePushA(name);
    if (!prof_on()) return;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    dev_ = dev;
    e0_ = get_event(dev);
    e1_ = get_event(dev);
    if (e0_) cudaEventRecord(e0_, s_);
}

ProfScope::~ProfScope()
{
    if (e0_ && e1_) {
        cudaEventRecord(e1_, s_);
        std::lock_guard<std::mutex> lk(g_mu);
        g_recs.push_back(Rec{name_, dev_, e0_, e1_});
    }
    nvtxRangePop();
}

}  // namespace fcirc

using namespace fcirc;

extern "C" {

int fcirc_prof_start(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        g_pool.push_back({r.dev, r.e0});
        g_pool.push_back({r.dev, r.e1});
    }
    g_recs.clear();
    g_on.store(true);
    return FCIRC_OK;
}

int fcirc_prof_stop(void)
{
    g_on.store(false);
    return FCIRC_OK;
}

uint64_t fcirc_prof_launches(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_recs.size();
}

int fcirc_prof_report(char *buf, uint64_t len)
{
    if (!buf || len == 0) return fail(FCIRC_EINVAL, "fcirc_prof_report: empty buffer");
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, std::pair<uint64_t, double>> agg;
    for (auto &r : g_recs) {
        cudaSetDevice(r.dev);
        FCIRC_CUDA_TRY(cudaEventSynchronize(r.e1));
        float ms = 0.f;
        FCIRC_CUDA_TRY(cudaEventElapsedTime(&ms, r.e0, r.e1));
        auto &a = agg[r.name];
        a.first += 1;
        a.second += ms;
    }
    std::string out;
    char line[256];
    for (auto &kv : agg) {
        snprintf(line, sizeof line, "%s %llu %.6f\n", kv.first.c_str(),
                 (unsigned long long)kv.second.first, kv.second.second);
        out += line;
    }
    strncpy(buf, out.c_str(), len - 1);
    buf[len - 1] = 0;
    return FCIRC_OK;
}

}  // extern "C"
