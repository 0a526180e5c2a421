// Diagnostics of libcpd: a process-wide kernel launch counter and optional
// per-stage device timing with CUDA events recorded on the launching stream.
#include <atomic>
#include <string.h>
#include <string>
#include <vector>

#include "kernels.h"

namespace cpdk {

static std::atomic<long long> g_launches{0};
static bool g_prof = false;

struct Rec { const char* name; cudaEvent_t a, b; };
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;

void count_launch(int n) { g_launches += n; }
bool profile_enabled() { return g_prof; }

static cudaEvent_t take_event() {
  if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(cudaStream_t st, const char* name) : st_(st), name_(name), a_(nullptr) {
  if (!g_prof) return;
  a_ = take_event();
  cudaEventRecord(a_, st_);
}

ProfScope::~ProfScope() {
  if (a_ == nullptr) return;
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st_);
  g_recs.push_back(Rec{name_, a_, b});
}

}  // namespace cpdk

using namespace cpdk;

extern "C" {

long long cpd_launch_count(void) { return g_launches.load(); }

int cpd_profile_enable(int on) { g_prof = on != 0; return CPD_OK; }

int cpd_profile_read(int max_entries, char* names, double* ms, long long* launches) {
  if (max_entries < 0 || (max_entries > 0 && (!names || !ms || !launches))) return CPD_ERR_INVALID_ARG;
  std::vector<std::string> nm;
  std::vector<double> tot;
  std::vector<long long> cnt;
  for (Rec& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return CPD_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return CPD_ERR_CUDA;
    size_t k = 0;
    while (k < nm.size() && nm[k] != r.name) ++k;
    if (k == nm.size()) { nm.emplace_back(r.name); tot.push_back(0.0); cnt.push_back(0); }
    tot[k] += t;
    cnt[k] += 1;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  int n = (int)nm.size() < max_entries ? (int)nm.size() : max_entries;
  for (int i = 0; i < n; ++i) {
    strncpy(names + 32 * i, nm[i].c_str(), 31);
    names[32 * i + 31] = '\0';
    ms[i] = tot[i];
    launches[i] = cnt[i];
  }
  return n;
}

}  // extern "C"
