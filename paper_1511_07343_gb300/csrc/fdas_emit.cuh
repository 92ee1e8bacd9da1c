// Warp-aggregated append of candidates to a device list.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fdas.h"

namespace fdas {

// Every lane of the warp must call this (the ballot is warp-wide); lanes with
// pred set append (r, j, h, H). The counter is exact even past maxc, where
// entries are dropped.
__device__ __forceinline__ void emit(bool pred, int r, int j, int h, float H, fdas_cand* out,
                                     unsigned long long* count, int64_t maxc) {
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) {
    const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
    if (slot < (unsigned long long)maxc) {
      fdas_cand c;
      c.r_top = r;
      c.z_idx = j;
      c.h = h;
      c.power = H;
      out[slot] = c;
    }
  }
}

}  // namespace fdas
