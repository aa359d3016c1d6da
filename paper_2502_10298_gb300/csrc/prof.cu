// Per-kernel-family event timing (see prof.h).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"
#include "prof.h"

namespace sctm {

namespace {
struct Rec {
  cudaEvent_t a, b;
  int fam;
  double flops, bytes;
  int launches;
  std::string tag;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_used = 0;
bool g_on = false;
std::mutex g_mu;
thread_local std::string g_tag;

cudaEvent_t take() {
  if (g_used < g_pool.size()) return g_pool[g_used++];
  cudaEvent_t e;
  SCTM_CUDA(cudaEventCreate(&e));
  g_pool.push_back(e);
  ++g_used;
  return e;
}
}  // namespace

void prof_enable(bool on) {
  std::lock_guard<std::mutex> l(g_mu);
  g_on = on;
  g_recs.clear();
  g_used = 0;
}

bool prof_enabled() { return g_on; }

void prof_set_tag(const char* tag) {
  if (g_on) g_tag = tag ? tag : "";
}

ProfScope::ProfScope(int family, cudaStream_t s, double flops, double bytes, int launches, const char* name)
    : fam(family), st(s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> l(g_mu);
  Rec r;
  r.a = take();
  r.b = take();
  r.fam = family;
  r.flops = flops;
  r.bytes = bytes;
  r.launches = launches;
  r.tag = name ? (g_tag.empty() ? std::string(name) : g_tag + " | " + name) : g_tag;
  SCTM_CUDA(cudaEventRecord(r.a, s));
  slot = (int)g_recs.size();
  g_recs.push_back(r);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> l(g_mu);
  cudaEventRecord(g_recs[slot].b, st);
}

void prof_collect(double* out) {
  std::lock_guard<std::mutex> l(g_mu);
  for (int i = 0; i < PF_N * 4; ++i) out[i] = 0;
  // SCTM_PROFILE_TAGS=<rows> prints the costliest (family, tag) pairs to stderr
  const char* tag_env = std::getenv("SCTM_PROFILE_TAGS");
  const int tag_rows = tag_env ? std::max(1, std::atoi(tag_env) > 0 ? std::atoi(tag_env) : 40) : 0;
  struct Sum {
    double ms = 0, flops = 0, bytes = 0;
    int n = 0;
  };
  std::map<std::string, Sum> by_tag;
  for (auto& r : g_recs) {
    SCTM_CUDA(cudaEventSynchronize(r.b));
    float ms = 0;
    SCTM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    out[r.fam * 4 + 0] += ms;
    out[r.fam * 4 + 1] += r.launches;
    out[r.fam * 4 + 2] += r.flops;
    out[r.fam * 4 + 3] += r.bytes;
    if (tag_rows) {
      Sum& t = by_tag[std::to_string(r.fam) + " " + r.tag];
      t.ms += ms;
      t.flops += r.flops;
      t.bytes += r.bytes;
      t.n += r.launches;
    }
  }
  if (tag_rows) {
    std::vector<std::pair<double, std::string>> v;
    for (auto& kv : by_tag) v.push_back({kv.second.ms, kv.first});
    std::sort(v.rbegin(), v.rend());
    for (size_t i = 0; i < v.size() && (int)i < tag_rows; ++i) {
      const Sum& t = by_tag[v[i].second];
      const double sec = t.ms * 1e-3 + 1e-30;
      std::fprintf(stderr, "[prof] %9.2f ms %6d launches %8.2f TF/s %8.1f GB/s  %s\n", t.ms, t.n,
                   t.flops / sec / 1e12, t.bytes / sec / 1e9, v[i].second.c_str());
    }
  }
  g_recs.clear();
  g_used = 0;
}

}  // namespace sctm
