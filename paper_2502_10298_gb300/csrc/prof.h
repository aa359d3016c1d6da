// Optional per-kernel-family timing with CUDA events on the launching stream.
// Disabled by default; when enabled every kernel launch of a family is
// bracketed by two events, and the caller reads summed device times, launch
// counts and algorithmic flop / byte counts per family.
#pragma once
#include <cuda_runtime.h>

namespace sctm {

enum ProfFamily { PF_CONTRACT = 0, PF_SVD = 1, PF_MISC = 2, PF_TENSOR = 3, PF_N = 4 };

void prof_enable(bool on);
// label attached to the scopes opened until the next call (e.g. an einsum
// spec with its dimensions); with SCTM_PROFILE_TAGS=<rows> in the environment,
// prof_collect also prints the labels with the most device time to stderr
void prof_set_tag(const char* tag);
bool prof_enabled();
// out: PF_N rows of {milliseconds, launches, flops, bytes}
void prof_collect(double* out);

// sets a label for the scopes of the current block and clears it on exit
struct ProfTag {
  explicit ProfTag(const char* tag) {
    if (tag) prof_set_tag(tag);
  }
  ~ProfTag() { prof_set_tag(""); }
};

struct ProfScope {
  // launches: kernel launches inside the scope; name: the kernel, appended to
  // the current label in the tagged summary
  ProfScope(int family, cudaStream_t s, double flops, double bytes, int launches = 1, const char* name = nullptr);
  ~ProfScope();
  int fam;
  cudaStream_t st;
  int slot = -1;
};

}  // namespace sctm
