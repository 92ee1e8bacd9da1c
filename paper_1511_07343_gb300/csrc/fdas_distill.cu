// Candidate distillation: the local maxima of a thresholded candidate list,
// with their Gaussian-equivalent significance (after the threshold; the
// paper stops at the power plane).
//
// A candidate (r, j, h, H) is kept when
//   * no candidate of the same level at (r + dr, j + dj), |dr|, |dj| <= 1,
//     has a larger H (equal H: the smaller (j, r) wins), and
//   * no candidate of an adjacent level that is the same signal - levels h
//     and 2h with |r' - 2 r| <= 2 and |jc' - 2 jc| <= 2, jc = j - zc - has a
//     larger sigma (equal sigma: the lower level wins),
// where sigma solves Phi_bar(sigma) = Q(h, H), Q the Gamma(h, 1) upper tail
// (the sum of h whitened noise powers), evaluated in its Poisson form
// Q = exp(-H) sum_{k<h} H^k / k! and kept as a logarithm.
//
// sigma is a decreasing function of ln Q, so the cross-level comparisons use
// ln Q itself (a larger sigma is a smaller ln Q, equal for equal); sigma is
// solved only for the survivors.
//
// The list goes into an open-addressing hash table (key = level, j, r; value
// = H) sized 2x the plan's candidate capacity; one thread per candidate then
// looks up its 8 same-level neighbours and the cross-level windows.
#include <math.h>

#include <algorithm>

#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long dkey(int lvl, int j, int r) {
  return ((unsigned long long)lvl << 56) | ((unsigned long long)(unsigned)j << 28) |
         (unsigned long long)(unsigned)r;
}

__device__ __forceinline__ uint32_t dslot(unsigned long long key, int bits) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

__device__ __forceinline__ int level_of(int h) { return __ffs(h) - 1; }

// ln Q(h, x) for integer h (Poisson form)
__device__ double log_gamma_tail(int h, double x) {
  double s = 0.0, term = 1.0;
  for (int k = 0; k < h; ++k) {
    if (k > 0) term *= x / k;
    s += term;
  }
  return -x + log(s);
}

// s with ln Phi_bar(s) = lp. ln Phi_bar(s) = ln(erfcx(s/sqrt2)/2) - s^2/2 is
// concave and decreasing, so Newton's method from a point above the root
// (sqrt(-2 lp) is one: ln Phi_bar(s) < -s^2/2 there) descends to it
// monotonically.
__device__ double gaussian_sigma(double lp) {
  const double rs2 = 0.70710678118654752440, k2pi = 0.79788456080286535588;  // 1/sqrt2, sqrt(2/pi)
  double s = lp < -1.2 ? sqrt(-2.0 * lp) : 1.5;
  for (int it = 0; it < 60; ++it) {
    const double e = erfcx(s * rs2);
    const double f = log(0.5 * e) - 0.5 * s * s - lp;
    const double step = f / (-k2pi / e);
    s -= step;
    if (fabs(step) <= 1e-14 * fmax(1.0, fabs(s))) break;
  }
  return s;
}

__device__ bool find(const unsigned long long* __restrict__ keys, const float* __restrict__ vals,
                     int bits, unsigned long long key, float* v) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t s = dslot(key, bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long k = keys[s];
    if (k == key) {
      *v = vals[s];
      return true;
    }
    if (k == kEmpty) return false;
    s = (s + 1) & mask;
  }
  return false;
}

__global__ void k_dist_clear(unsigned long long* __restrict__ keys, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = kEmpty;
}

__global__ void k_dist_insert(const fdas_cand* __restrict__ c, const long long* __restrict__ count,
                              int64_t maxc, unsigned long long* __restrict__ keys,
                              float* __restrict__ vals, int bits) {
  const int64_t n = min((int64_t)*count, maxc);
  const uint32_t mask = (1u << bits) - 1u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const fdas_cand a = c[i];
    const unsigned long long key = dkey(level_of(a.h), a.z_idx, a.r_top);
    uint32_t s = dslot(key, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const unsigned long long prev = atomicCAS(keys + s, kEmpty, key);
      if (prev == kEmpty || prev == key) {
        vals[s] = a.power;
        break;
      }
      s = (s + 1) & mask;
    }
  }
}

__device__ __forceinline__ int floor_div2(int x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }
__device__ __forceinline__ int ceil_div2(int x) { return -floor_div2(-x); }

__global__ void k_dist_peaks(const fdas_cand* __restrict__ c, const long long* __restrict__ count,
                             int64_t maxc, const unsigned long long* __restrict__ keys,
                             const float* __restrict__ vals, int bits, int Z, int n_levels,
                             fdas_peak* __restrict__ out, unsigned long long* __restrict__ nout,
                             int64_t cap) {
  const int64_t n = min((int64_t)*count, maxc);
  const int zc = (Z - 1) / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // whole warps iterate together so the aggregated append sees all lanes
  const int64_t n_pad = (n + 31) & ~(int64_t)31;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad; i += stride) {
    bool keep = i < n;
    fdas_cand a{};
    double lp = 0.0, sg = 0.0;
    if (keep) {
      a = c[i];
      const int lvl = level_of(a.h);
      const float v = a.power;
      float w;
      for (int dj = -1; dj <= 1 && keep; ++dj)
        for (int dr = -1; dr <= 1 && keep; ++dr) {
          if (!(dr | dj)) continue;
          const int j2 = a.z_idx + dj, r2 = a.r_top + dr;
          if (j2 < 0 || j2 >= Z || r2 < 0) continue;
          if (find(keys, vals, bits, dkey(lvl, j2, r2), &w) &&
              (w > v || (w == v && (j2 < a.z_idx || (j2 == a.z_idx && r2 < a.r_top)))))
            keep = false;
        }
      if (keep) {
        lp = log_gamma_tail(a.h, (double)v);
        const int jc = a.z_idx - zc;
        // level 2h: r' in [2r-2, 2r+2], jc' in [2jc-2, 2jc+2]
        if (lvl + 1 < n_levels)
          for (int dj = -2; dj <= 2 && keep; ++dj)
            for (int dr = -2; dr <= 2 && keep; ++dr) {
              const int j2 = zc + 2 * jc + dj, r2 = 2 * a.r_top + dr;
              if (j2 < 0 || j2 >= Z || r2 < 0) continue;
              if (find(keys, vals, bits, dkey(lvl + 1, j2, r2), &w) &&
                  log_gamma_tail(2 * a.h, (double)w) < lp)
                keep = false;
            }
        // level h/2: 2 r' in [r-2, r+2], 2 jc' in [jc-2, jc+2]
        if (lvl > 0)
          for (int jc2 = ceil_div2(jc - 2); jc2 <= floor_div2(jc + 2) && keep; ++jc2)
            for (int r2 = ceil_div2(a.r_top - 2); r2 <= floor_div2(a.r_top + 2) && keep; ++r2) {
              const int j2 = zc + jc2;
              if (j2 < 0 || j2 >= Z || r2 < 0) continue;
              if (find(keys, vals, bits, dkey(lvl - 1, j2, r2), &w) &&
                  log_gamma_tail(a.h / 2, (double)w) <= lp)
                keep = false;
            }
        if (keep) sg = gaussian_sigma(lp);
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (!mask) continue;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(nout, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (keep) {
      const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
      if (slot < (unsigned long long)cap) {
        fdas_peak pk;
        pk.r_top = a.r_top;
        pk.z_idx = a.z_idx;
        pk.h = a.h;
        pk.power = a.power;
        pk.sigma = (float)sg;
        pk.log10_p = (float)(lp * 0.43429448190325182765);
        out[slot] = pk;
      }
    }
  }
}

}  // namespace

int launch_distill(fdas_plan* p, const fdas_cand* d_cands, const int64_t* d_count,
                   fdas_peak* d_peaks, int64_t* d_npeaks) {
  int rc;
  if (!p->dkeys) {
    int bits = 10;
    while (((int64_t)1 << bits) < 2 * p->max_cands) ++bits;
    const size_t n = (size_t)1 << bits;
    if (cudaMalloc((void**)&p->dkeys, n * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&p->dvals, n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();  // a refused allocation must not surface at a later launch check
      if (p->dkeys) cudaFree(p->dkeys);
      p->dkeys = nullptr;
      p->dvals = nullptr;
      return set_error(FDAS_ERR_NOMEM, "distillation table allocation failed");
    }
    p->dbits = bits;
    p->device_bytes += (int64_t)(n * (sizeof(unsigned long long) + sizeof(float)));
  }
  const int64_t tsize = (int64_t)1 << p->dbits;
  if ((rc = cuda_check(cudaMemsetAsync(d_npeaks, 0, sizeof(int64_t), p->stream), "memset peaks")))
    return rc;
  k_dist_clear<<<(unsigned)std::min<int64_t>((tsize + 255) / 256, 4096), 256, 0, p->stream>>>(
      p->dkeys, tsize);
  if ((rc = cuda_check(cudaGetLastError(), "k_dist_clear"))) return rc;
  const unsigned grid = (unsigned)std::min<int64_t>((p->max_cands + 255) / 256, 2048);
  const auto* cnt = reinterpret_cast<const long long*>(d_count);
  k_dist_insert<<<grid, 256, 0, p->stream>>>(d_cands, cnt, p->max_cands, p->dkeys, p->dvals,
                                              p->dbits);
  if ((rc = cuda_check(cudaGetLastError(), "k_dist_insert"))) return rc;
  k_dist_peaks<<<grid, 256, 0, p->stream>>>(d_cands, cnt, p->max_cands, p->dkeys, p->dvals,
                                             p->dbits, p->Z, p->n_levels, d_peaks,
                                             reinterpret_cast<unsigned long long*>(d_npeaks),
                                             p->max_cands);
  return cuda_check(cudaGetLastError(), "k_dist_peaks");
}

}  // namespace fdas
