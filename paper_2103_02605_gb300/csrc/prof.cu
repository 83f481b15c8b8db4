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

// Integer-multiply throughput probe: every thread runs CH independent chains
// of one multiply kind, so the SM's multiply pipe, not latency, sets the
// rate.  KIND 0: v = v * a + b (a low-half IMAD); KIND 1: v = hi(v * a) + b
// (a high-half IMAD).  The chains' XOR is stored only if it equals a value
// the caller picks, which keeps the work from being optimised away.
template <int KIND>
__global__ void __launch_bounds__(256) k_mulprobe(uint32_t *sink, uint32_t a, uint32_t b, uint32_t iters,
                                                  uint32_t key)
{
    constexpr int CH = 16;
    uint32_t v[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) v[k] = threadIdx.x * (2 * k + 1) + blockIdx.x + k;
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if constexpr (KIND == 0)
                v[k] = v[k] * a + b;
            else
                v[k] = __umulhi(v[k], a) + b;
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < CH; ++k) x ^= v[k];
    if (x == key) sink[blockIdx.x & 255] = x;
}

}  // namespace fcirc

using namespace fcirc;

extern "C" {

int fcirc_prof_mul_probe(int kind, uint32_t ctas_per_sm, uint32_t iters, double *ms, double *mul_per_s)
{
    if ((kind != 0 && kind != 1) || ctas_per_sm == 0 || ctas_per_sm > 8 || iters == 0 || !ms || !mul_per_s)
        return fail(FCIRC_EINVAL, "fcirc_prof_mul_probe: bad arguments");
    int dev = 0, nsm = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    FCIRC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    void *sink = nullptr;
    if (dev_alloc(&sink, 1024) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(FCIRC_ENOMEM, "fcirc_prof_mul_probe: sink allocation failed");
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FCIRC_OK;
    const unsigned blocks = (unsigned)nsm * ctas_per_sm;
    auto launch = [&]() {
        if (kind == 0)
            k_mulprobe<0><<<blocks, 256, 0, s>>>(static_cast<uint32_t *>(sink), 0x9E3779B1u, 0x7F4A7C15u, iters, 1u);
        else
            k_mulprobe<1><<<blocks, 256, 0, s>>>(static_cast<uint32_t *>(sink), 0x9E3779B1u, 0x7F4A7C15u, iters, 1u);
        return cudaGetLastError();
    };
    float best = 0.f;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || launch() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        rc = fail(FCIRC_ECUDA, "fcirc_prof_mul_probe: %s", cudaGetErrorString(cudaGetLastError()));
    } else {
        for (int r = 0; r < 5 && rc == FCIRC_OK; ++r) {
            float t = 0.f;
            if (cudaEventRecord(e0, s) != cudaSuccess || launch() != cudaSuccess ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                rc = fail(FCIRC_ECUDA, "fcirc_prof_mul_probe: %s", cudaGetErrorString(cudaGetLastError()));
            else if (best == 0.f || t < best)
                best = t;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    if (rc != FCIRC_OK) return rc;
    *ms = best;
    // 16 chains of one multiply per thread and iteration
    *mul_per_s = (double)blocks * 256.0 * 16.0 * (double)iters / (best * 1e-3);
    return FCIRC_OK;
}

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
