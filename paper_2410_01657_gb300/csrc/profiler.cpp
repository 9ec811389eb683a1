// Per-kernel timing for benchmarks: while enabled, every libgnnmp kernel launch
// is bracketed by a pair of CUDA events recorded on the launch stream; the
// report sums the elapsed times per kernel name.

#include "profiler.h"

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"

namespace gnn {
namespace {

struct Record {
    const char* name;
    cudaEvent_t start, stop;
};

std::atomic<bool> g_on(false);
std::mutex g_mu;
std::vector<Record> g_pool;
size_t g_used = 0;
bool g_overflow = false;

}  // namespace

ProfScope::ProfScope(cudaStream_t stream, const char* name) : slot(-1), s(stream) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_used >= g_pool.size()) {
        g_overflow = true;
        return;
    }
    slot = (int)g_used++;
    g_pool[slot].name = name;
    cudaEventRecord(g_pool[slot].start, s);
}

ProfScope::~ProfScope() {
    if (slot >= 0) cudaEventRecord(g_pool[slot].stop, s);
}

}  // namespace gnn

extern "C" {

int gnn_profile_start(int32_t capacity) {
    GNN_REQUIRE(capacity > 0 && capacity <= (1 << 22), GNN_EINVAL, "gnn_profile_start: bad capacity");
    std::lock_guard<std::mutex> lk(gnn::g_mu);
    if (gnn::g_pool.size() < (size_t)capacity) {
        size_t old = gnn::g_pool.size();
        gnn::g_pool.resize(capacity);
        for (size_t i = old; i < gnn::g_pool.size(); ++i) {
            if (cudaEventCreate(&gnn::g_pool[i].start) != cudaSuccess ||
                cudaEventCreate(&gnn::g_pool[i].stop) != cudaSuccess) {
                gnn::g_pool.resize(i);
                return gnn::set_error(GNN_ECUDA, "gnn_profile_start: cudaEventCreate failed");
            }
        }
    }
    gnn::g_used = 0;
    gnn::g_overflow = false;
    gnn::g_on.store(true);
    return GNN_OK;
}

int gnn_profile_stop(void) {
    gnn::g_on.store(false);
    return GNN_OK;
}

int gnn_profile_report(char* out, size_t bytes) {
    GNN_REQUIRE(out && bytes > 0, GNN_EINVAL, "gnn_profile_report: NULL buffer");
    std::lock_guard<std::mutex> lk(gnn::g_mu);
    std::map<std::string, std::pair<long, double>> agg;
    for (size_t i = 0; i < gnn::g_used; ++i) {
        if (cudaEventSynchronize(gnn::g_pool[i].stop) != cudaSuccess)
            return gnn::set_error(GNN_ECUDA, "gnn_profile_report: event synchronize failed");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, gnn::g_pool[i].start, gnn::g_pool[i].stop) != cudaSuccess)
            return gnn::set_error(GNN_ECUDA, "gnn_profile_report: elapsed time failed");
        auto& a = agg[gnn::g_pool[i].name];
        a.first += 1;
        a.second += ms;
    }
    std::string s;
    char line[256];
    for (auto& kv : agg) {
        snprintf(line, sizeof(line), "%s %ld %.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
        s += line;
    }
    if (gnn::g_overflow) s += "# overflow: capacity too small\n";
    GNN_REQUIRE(s.size() + 1 <= bytes, GNN_ENOMEM, "gnn_profile_report: buffer too small");
    std::memcpy(out, s.c_str(), s.size() + 1);
    return GNN_OK;
}

}  // extern "C"
