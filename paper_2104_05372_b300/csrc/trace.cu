// Per-launch CUDA-event timing (see trace.cuh) and its C-ABI accessors.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "trace.cuh"

namespace gpa {
namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

void trace_begin(const char* name, cudaStream_t s) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{name, take(), take()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
}

void trace_end(cudaStream_t s) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_recs.empty()) cudaEventRecord(g_recs.back().b, s);
}
}  // namespace gpa

using namespace gpa;

extern "C" void gpa_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
}

extern "C" int gpa_trace_summary(char* buf, size_t len) {
    std::lock_guard<std::mutex> lk(g_mu);
    struct Agg {
        std::string name;
        long count;
        double ms;
    };
    std::vector<Agg> agg;
    for (const Rec& r : g_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        bool found = false;
        for (Agg& a : agg)
            if (a.name == r.name) {
                a.count++;
                a.ms += ms;
                found = true;
                break;
            }
        if (!found) agg.push_back({r.name, 1, (double)ms});
    }
    std::string out;
    char line[256];
    for (const Agg& a : agg) {
        snprintf(line, sizeof line, "%s %ld %.6f\n", a.name.c_str(), a.count, a.ms);
        out += line;
    }
    if (!buf || len <= out.size()) return (int)out.size();  // size query: keep the records
    memcpy(buf, out.data(), out.size());
    buf[out.size()] = '\0';
    for (const Rec& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return (int)out.size();
}
