// Block-median whitening: the cheaper variant of the whitening stage (the
// paper does not specify whitening; the search adds it before step 3).
//
//   mu_b  = median of |X_k|^2 over block b = [1 + 64 b, min(1 + 64 (b+1), nb))
//   c_b   = (first + last) / 2, the block centre
//   mu_k  = mu_b + (k - c_b) (mu_{b+1} - mu_b) / (c_{b+1} - c_b)  for c_b <= k < c_{b+1},
//           mu_0 below the first centre, mu_last from the last centre on
//   Xw_k  = X_k sqrt(ln 2 / mu_k),  Xw_0 = 0.
//
// One warp per block finds the median (two powers per lane, a bitonic
// network across the warp, +inf filling a short last block); one thread per
// bin interpolates. Centres are handled as the integers 2 c_b.
#include <math.h>

#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr int kBlk = 64;

__global__ void __launch_bounds__(256) k_block_median(const float2* __restrict__ X,
                                                      float* __restrict__ med, int64_t nb,
                                                      int64_t nblk) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nblk) return;  // b is the same for the whole warp
  const int64_t s = 1 + (int64_t)kBlk * b;
  const int64_t e = s + kBlk < nb ? s + kBlk : nb;
  const int c = (int)(e - s);
  float v[2];
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int64_t i = s + 32 * slot + lane;
    if (i < e) {
      const float2 x = __ldg(X + i);
      v[slot] = x.x * x.x + x.y * x.y;
    } else {
      v[slot] = INFINITY;
    }
  }
  // element e = 32 slot + lane; ascending bitonic sort of the 64 elements
#pragma unroll
  for (int k = 2; k <= kBlk; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // partner is the other slot of the same lane (k = 64)
        const float lo = fminf(v[0], v[1]), hi = fmaxf(v[0], v[1]);
        v[0] = lo;
        v[1] = hi;
      } else {
#pragma unroll
        for (int slot = 0; slot < 2; ++slot) {
          const int el = 32 * slot + lane;
          const float o = __shfl_xor_sync(0xffffffffu, v[slot], j);
          const bool up = (el & k) == 0, lower = (el & j) == 0;
          v[slot] = (lower == up) ? fminf(v[slot], o) : fmaxf(v[slot], o);
        }
      }
    }
  }
  const int i0 = (c - 1) >> 1, i1 = c >> 1;
  const float a0 = __shfl_sync(0xffffffffu, i0 < 32 ? v[0] : v[1], i0 & 31);
  const float a1 = __shfl_sync(0xffffffffu, i1 < 32 ? v[0] : v[1], i1 & 31);
  if (lane == 0) med[b] = 0.5f * (a0 + a1);
}

__global__ void __launch_bounds__(256) k_block_whiten(const float2* __restrict__ X,
                                                      const float* __restrict__ med,
                                                      float2* __restrict__ Xw, int64_t nb,
                                                      int64_t nblk) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nb) return;
  if (k == 0) {
    Xw[0] = make_float2(0.f, 0.f);
    return;
  }
  const int64_t last = nblk - 1;
  const int64_t two_k = 2 * k;
  const int64_t two_c_last = (int64_t)kBlk * last + nb;  // first + last bin of the last block
  float mu;
  if (two_k <= 2 + kBlk - 1) {  // at or below the first centre, 2 c_0 = 65
    mu = __ldg(med);
  } else if (two_k >= two_c_last) {
    mu = __ldg(med + last);
  } else {
    int64_t b = (two_k - (kBlk + 1)) / (2 * kBlk);
    if (b > last - 1) b = last - 1;
    const int64_t c0 = (kBlk + 1) + 2 * kBlk * b;
    const int64_t c1 = b + 1 == last ? two_c_last : c0 + 2 * kBlk;
    const float t = (float)(two_k - c0) / (float)(c1 - c0);
    const float m0 = __ldg(med + b), m1 = __ldg(med + b + 1);
    mu = m0 + t * (m1 - m0);
  }
  const float2 x = X[k];
  const float g = mu > 0.f ? sqrtf(0.69314718055994531f / mu) : 0.f;
  Xw[k] = make_float2(x.x * g, x.y * g);
}

}  // namespace

int launch_whiten_block(fdas_plan* p, const float2* d_spec, float2* d_white) {
  const int64_t nblk = (p->nb - 1 + kBlk - 1) / kBlk;
  float* med = reinterpret_cast<float*>(p->zbuf);  // free once the spectrum exists
  k_block_median<<<(unsigned)((nblk * 32 + 255) / 256), 256, 0, p->stream>>>(d_spec, med, p->nb,
                                                                            nblk);
  int rc = cuda_check(cudaGetLastError(), "k_block_median");
  if (rc) return rc;
  k_block_whiten<<<(unsigned)((p->nb + 255) / 256), 256, 0, p->stream>>>(d_spec, med, d_white,
                                                                          p->nb, nblk);
  return cuda_check(cudaGetLastError(), "k_block_whiten");
}

}  // namespace fdas
