// Harmonic summing, thresholding and candidate compaction (the stages the
// search adds after step 7 of Section 4).
//
// For a top-harmonic cell (r, j) and h in {1, 2, 4, 8, 16},
//     H_h(r, j) = sum_{k=1..h} P[jz(k, j, h)][rr(k, r, h)],
//     rr = round(k r / h)          (ties up:   floor((2 k r + h) / (2 h))),
//     jz = zc + round(k (j-zc) / h) (ties away from zero; zc = (Z-1)/2),
// and (r, j, h, H_h) is a candidate when H_h >= T_h, with T_h the Gamma(h, 1)
// tail point equal to the Gaussian tail at sigma. All indices are integer
// arithmetic; the fraction k/h is evaluated as q/16 with q = 16 k / h, so the
// 16 distinct terms q = 1..16 serve every level:
//     H_1 = t16, H_2 = H_1 + t8, H_4 = H_2 + (t4 + t12),
//     H_8 = H_4 + ((t2 + t6) + (t10 + t14)), H_16 = H_8 + (odd q terms).
#include "fdas_common.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

struct Thr {
  float t[5];
};

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

// Direct form: one thread per top cell, the 16 fraction terms gathered from
// the plane (sub-harmonic rows and columns are re-read through L1/L2).
__global__ void __launch_bounds__(256) k_harmsum_direct(const float* __restrict__ P, int64_t nb,
                                                        int Z, int n_levels, Thr thr,
                                                        fdas_cand* __restrict__ out,
                                                        unsigned long long* count, int64_t maxc) {
  const int j = blockIdx.y;
  const int64_t r64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r64 >= 1 && r64 < nb;
  const int r = valid ? (int)r64 : 1;
  const int zc = (Z - 1) / 2;
  const int jc = j - zc;
  const int sg = jc < 0 ? -1 : 1;
  auto term = [&](int q) -> float {
    const int rr = (2 * q * r + 16) >> 5;
    const int a = q * (jc < 0 ? -jc : jc);
    const int jz = zc + sg * ((2 * a + 16) >> 5);
    return __ldg(P + (size_t)jz * nb + rr);
  };
  float H = term(16);
  emit(valid && H >= thr.t[0], r, j, 1, H, out, count, maxc);
  if (n_levels < 2) return;
  H = H + term(8);
  emit(valid && H >= thr.t[1], r, j, 2, H, out, count, maxc);
  if (n_levels < 3) return;
  H = H + (term(4) + term(12));
  emit(valid && H >= thr.t[2], r, j, 4, H, out, count, maxc);
  if (n_levels < 4) return;
  H = H + ((term(2) + term(6)) + (term(10) + term(14)));
  emit(valid && H >= thr.t[3], r, j, 8, H, out, count, maxc);
  if (n_levels < 5) return;
  H = H + (((term(1) + term(3)) + (term(5) + term(7))) +
           ((term(9) + term(11)) + (term(13) + term(15))));
  emit(valid && H >= thr.t[4], r, j, 16, H, out, count, maxc);
}

}  // namespace

int launch_harmsum(fdas_plan* p, const float* d_plane, fdas_cand* d_out,
                   unsigned long long* d_count) {
  Thr thr;
  for (int i = 0; i < 5; ++i) thr.t[i] = p->thr[i];
  dim3 grid((unsigned)((p->nb + 255) / 256), p->Z);
  k_harmsum_direct<<<grid, 256, 0, p->stream>>>(d_plane, p->nb, p->Z, p->n_levels, thr, d_out,
                                                d_count, p->max_cands);
  return cuda_check(cudaGetLastError(), "k_harmsum_direct");
}

}  // namespace fdas
