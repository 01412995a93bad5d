// Per-kernel accounting: launch counts, CUDA-event times on the launching
// stream, and the algorithmic work (flops, bytes) the host attributes to each
// kernel class from the sizes it knows after each level.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

namespace fmmlu {

struct ProfEntry {
  int64_t launches = 0;
  double ms = 0;      // summed CUDA-event durations
  double flops = 0;   // real flops the launches execute on their pipe (for the
                      // exact-split tensor-core products: the bf16 digit-pair
                      // flops)
  double bytes = 0;   // algorithmic DRAM bytes attributed to these launches
  double mflops = 0;  // the method's own real flops (8 per complex multiply-add
                      // of the fp64 product it computes, whatever the pipe)
};

struct Profiler {
  struct Pending {
    const char* name;
    cudaEvent_t a, b;
  };
  std::map<std::string, ProfEntry> tot;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> spare;
  cudaEvent_t get();
  void resolve();     // call after the stream has been synchronised
  // mflops < 0: the method's flops equal the executed ones
  void add_work(const char* name, double flops, double bytes, double mflops = -1.0);
  void reset();
  std::string json() const;
  ~Profiler();
};

extern thread_local Profiler* g_prof;
int64_t launches_total();
// adjusts the count: kernels recorded into a CUDA graph count when the graph
// is launched, not when it is captured
void launches_add(int64_t d);

// sets g_prof for a scope
struct ProfScope {
  Profiler* saved;
  explicit ProfScope(Profiler* p) : saved(g_prof) { g_prof = p; }
  ~ProfScope() { g_prof = saved; }
};

}  // namespace fmmlu
