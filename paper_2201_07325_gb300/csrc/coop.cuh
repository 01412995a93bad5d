// Bounded per-box barriers for kernels whose CTAs cooperate on one box.
//
// A launch using these must be cooperative (all CTAs co-resident). Each box
// owns a counter (zeroed before the launch) and an abort flag. A CTA arrives
// by incrementing the counter and waits until it reaches nbar * P. Every wait
// is bounded: after kSpinLimit polls the abort flag is raised, the status word
// gets kStatusTimeout, and every CTA of the box returns at its next barrier.
#pragma once

#include "device_common.cuh"

namespace fmmlu {

constexpr long long kSpinLimit = 20000000;   // ~2 s at 100 ns per poll

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// returns false when the box was aborted (timeout here or in another CTA)
static __device__ bool box_barrier(unsigned* ctr, unsigned target, int* abort_flag, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(ctr, 1u);
    long long spins = 0;
    while (ld_acquire_u32(ctr) < target) {
      if (ld_acquire_u32(reinterpret_cast<unsigned*>(abort_flag))) { ok = 0; break; }
      if (++spins > kSpinLimit) {
        atomicExch(abort_flag, 1);
        set_status(status, kStatusTimeout);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }


}  // namespace fmmlu
