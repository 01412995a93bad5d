// Launch accounting and per-kernel CUDA-event timing (see prof.h).
#include <atomic>
#include <cstdio>
#include <sstream>

#include "fmmlu_internal.h"
#include "prof.h"

namespace fmmlu {

thread_local Profiler* g_prof = nullptr;
static std::atomic<int64_t> g_launches{0};

int64_t launches_total() { return g_launches.load(); }
void launches_add(int64_t d) { g_launches.fetch_add(d); }

void launch_begin(const char* name, cudaStream_t st) {
  g_launches.fetch_add(1);
  if (!g_prof) return;
  cudaEvent_t e = g_prof->get();
  cudaEventRecord(e, st);
  g_prof->pending.push_back({name, e, nullptr});
}

void launch_end(const char*, cudaStream_t st) {
  if (!g_prof || g_prof->pending.empty()) return;
  cudaEvent_t e = g_prof->get();
  cudaEventRecord(e, st);
  g_prof->pending.back().b = e;
}

cudaEvent_t Profiler::get() {
  if (!spare.empty()) {
    cudaEvent_t e = spare.back();
    spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Profiler::resolve() {
  for (auto& p : pending) {
    float ms = 0.f;
    if (p.a && p.b && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ProfEntry& t = tot[p.name];
      t.launches += 1;
      t.ms += ms;
    }
    if (p.a) spare.push_back(p.a);
    if (p.b) spare.push_back(p.b);
  }
  pending.clear();
}

void Profiler::add_work(const char* name, double flops, double bytes, double mflops) {
  ProfEntry& t = tot[name];
  t.flops += flops;
  t.bytes += bytes;
  t.mflops += mflops < 0.0 ? flops : mflops;
}

void Profiler::reset() {
  resolve();
  tot.clear();
}

std::string Profiler::json() const {
  std::ostringstream o;
  o.precision(10);
  o << "{";
  bool first = true;
  for (const auto& kv : tot) {
    o << (first ? "" : ", ") << "\"" << kv.first << "\": {\"launches\": " << kv.second.launches
      << ", \"ms\": " << kv.second.ms << ", \"flops\": " << kv.second.flops
      << ", \"bytes\": " << kv.second.bytes << ", \"method_flops\": " << kv.second.mflops
      << "}";
    first = false;
  }
  o << "}";
  return o.str();
}

Profiler::~Profiler() {
  for (auto& p : pending) {
    if (p.a) cudaEventDestroy(p.a);
    if (p.b) cudaEventDestroy(p.b);
  }
  for (auto e : spare) cudaEventDestroy(e);
}

}  // namespace fmmlu
