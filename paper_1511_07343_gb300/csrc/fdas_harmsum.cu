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
#include "fdas_emit.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

struct Thr {
  float t[5];
};

// Q4[j][g] = max(P[j][4g .. 4g+3]) and the h = 1 candidates of a given plane
// (the correlation kernel produces both itself; this serves planes supplied
// from outside).
__global__ void __launch_bounds__(256) k_pool4(const float* __restrict__ P, float* __restrict__ Q4,
                                               int64_t nb, float thr1, fdas_cand* __restrict__ out,
                                               unsigned long long* count, int64_t maxc) {
  const int j = blockIdx.y;
  const int64_t nq = nb >> 2;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool gv = g < nq;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (gv) {
    v = __ldg(reinterpret_cast<const float4*>(P + (size_t)j * nb) + g);
    Q4[(size_t)j * nq + g] = fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w));
  }
  const int r0 = (int)(4 * g);
  emit(gv && r0 >= 1 && v.x >= thr1, r0, j, 1, v.x, out, count, maxc);
  emit(gv && v.y >= thr1, r0 + 1, j, 1, v.y, out, count, maxc);
  emit(gv && v.z >= thr1, r0 + 2, j, 1, v.z, out, count, maxc);
  emit(gv && v.w >= thr1, r0 + 3, j, 1, v.w, out, count, maxc);
}

// Harmonic sums h >= 2, screened, in a fixed summation order: the fractions
// q/16 are added one after the other as q = 16, 8 | 4, 12 | 2, 6, 10, 14 |
// 1, 3, .., 15, so H_2, H_4, H_8 and H_16 are the running sums after 2, 4, 8
// and 16 terms. A block takes top row j and 16384 consecutive top bins;
// warp w takes the 2048 bins from R0w = R0 + 2048 w and lane l the 64 bins
// R0w + 64 l + i. For fraction q the sub-harmonic bin is
//     rr = round(q r / 16) = q R0w/16 + 4 q l + K(q, i),  K(q, i) = (2 q i + 16) >> 5,
// so its 4-bin group, relative to the warp's first, is q l + (K(q, i) >> 2):
// a compile-time offset from q l. Each warp stages its own slice of row
// jz(q) of Q4 (32 q + 1 groups) in shared memory, split into 2^a classes by
// index mod 2^a (q = 2^a b, b odd): lanes then read at stride b, which is
// odd, so reads are free of bank conflicts; copies are coalesced cp.async
// (16-byte for odd q, whose slice is contiguous), two fractions ahead, and
// warps never wait for one another. Each term is bounded by its group
// maximum, each pair of adjacent bins shares one bound (the larger of its
// groups); float addition is monotone, so a pair whose running bound stays
// below T_h cannot hold a candidate at level h. The rare flagged pairs are
// summed exactly from P in the same order and compared with T_h.
__host__ __device__ constexpr int frac_order(int i) {
  return i == 0 ? 16 : i == 1 ? 8 : i == 2 ? 4 : i == 3 ? 12 : i < 8 ? 2 + 4 * (i - 4)
                                                                     : 1 + 2 * (i - 8);
}
__host__ __device__ constexpr int kq(int q, int i) { return (2 * q * i + 16) >> 5; }
__host__ __device__ constexpr int ctz5(int q) {
  return (q & 1) ? 0 : (q & 2) ? 1 : (q & 4) ? 2 : (q & 8) ? 3 : 4;
}
// words between classes (a >= 1): >= 32 b + 1 entries and = 32 >> a mod 32,
// so the 2^a classes of one copy round start on distinct banks
__host__ __device__ constexpr int class_stride(int q) {
  return 32 * (q >> ctz5(q)) + (32 >> ctz5(q));
}

// a block is NT threads (128 or 256: the harmonic-sum tiling the batch
// autotuner chooses), each warp independent of the others
constexpr int kHsCells = 64;
constexpr int kWarpSpan = 32 * kHsCells;
constexpr int kStageW = 16 * 34;  // largest staged slice per warp (q = 16), floats
template <int NT>
constexpr size_t hs_smem() { return (size_t)3 * kStageW * (NT / 32) * sizeof(float); }

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
               "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

struct HsCtx {
  float* stage;  // this warp's 3 rotating buffers
  const float* Q4;
  int64_t nq, R0w;
  int lane, zc, sg, ajc;
};

// copy of the warp's slice of row jz(q) of Q4 (fraction number OI in
// summation order) into rotating buffer OI % 3
template <int OI, int NQ>
FDAS_DEV void hs_issue(const HsCtx& x) {
  if constexpr (OI < NQ) {
    constexpr int q = frac_order(OI);
    constexpr int a = ctz5(q), m = (1 << a) - 1;
    float* buf = x.stage + (OI % 3) * kStageW;
    const int row = x.zc + x.sg * ((2 * q * x.ajc + 16) >> 5);
    const int64_t e_lo = (int64_t)q * (x.R0w >> 6);
    const float* src = x.Q4 + (size_t)row * x.nq + e_lo;
    const int64_t lim = x.nq - e_lo;  // entries e < lim exist
    if constexpr (a == 0) {
      // contiguous slice of 32 q + 1 entries: 16-byte chunks (nq is a
      // multiple of 4, so a chunk is entirely inside or outside the row)
      constexpr int nchunk = (32 * q + 1 + 3) / 4;
#pragma unroll
      for (int c0 = 0; c0 < nchunk; c0 += 32) {
        const int c = c0 + x.lane;
        if (c0 + 32 <= nchunk || c < nchunk) cp_async16(buf + 4 * c, src + 4 * c, 4 * c < lim);
      }
    } else {
      constexpr int CS = class_stride(q);
      float* sb = buf + (x.lane & m) * CS + (x.lane >> a);
      const float* sl = src + x.lane;
      const int64_t llim = lim - x.lane;
#pragma unroll
      for (int k = 0; k < q; ++k) cp_async4(sb + k * (32 >> a), sl + 32 * k, 32 * k < llim);
      if (x.lane == 0) cp_async4(sb + q * (32 >> a), sl + 32 * q, 32 * q < llim);
    }
  }
  cp_async_commit();
}

template <int OI, int NQ>
FDAS_DEV void hs_steps(const HsCtx& x, float2 (&acc)[kHsCells / 4], unsigned& pmask,
                       const Thr& thr) {
  if constexpr (OI < NQ) {
    constexpr int q = frac_order(OI);
    constexpr int a = ctz5(q), m = (1 << a) - 1, b = q >> a;
    constexpr int CS = a == 0 ? 0 : class_stride(q);
    cp_async_wait1();
    __syncwarp();
    hs_issue<OI + 2, NQ>(x);
    const float* sb = x.stage + (OI % 3) * kStageW + b * x.lane;
#pragma unroll
    for (int pp = 0; pp < kHsCells / 4; ++pp) {
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int pr = 2 * pp + h;
        const int o1 = kq(q, 2 * pr) >> 2;
        const int o2 = kq(q, 2 * pr + 1) >> 2;
        v[h] = sb[(o1 & m) * CS + (o1 >> a)];
        if (o2 != o1) v[h] = fmaxf(v[h], sb[(o2 & m) * CS + (o2 >> a)]);
      }
      const float2 v2 = make_float2(v[0], v[1]);
      acc[pp] = (OI == 0) ? v2 : __fadd2_rn(acc[pp], v2);
    }
    if constexpr (OI == 1 || OI == 3 || OI == 7 || OI == 15) {
      constexpr int lvl = OI == 1 ? 1 : (OI == 3 ? 2 : (OI == 7 ? 3 : 4));
      const float t = thr.t[lvl];
      float mx = fmaxf(acc[0].x, acc[0].y);
#pragma unroll
      for (int pp = 1; pp < kHsCells / 4; ++pp) mx = fmaxf(mx, fmaxf(acc[pp].x, acc[pp].y));
      if (mx >= t) {
#pragma unroll
        for (int pp = 0; pp < kHsCells / 4; ++pp) {
          if (acc[pp].x >= t) pmask |= 1u << (2 * pp);
          if (acc[pp].y >= t) pmask |= 1u << (2 * pp + 1);
        }
      }
    }
    // the next step overwrites buffer (OI + 3) % 3 = OI % 3 only after its
    // own wait and warp barrier, which every lane reaches after these reads
    hs_steps<OI + 1, NQ>(x, acc, pmask, thr);
  }
}

template <int NLEV, int NT>
__global__ void __launch_bounds__(NT) k_harmsum_staged(
    const float* __restrict__ P, const float* __restrict__ Q4, int64_t nb, int Z, Thr thr,
    fdas_cand* __restrict__ out, unsigned long long* count, int64_t maxc) {
  constexpr int NQ = 1 << (NLEV - 1);
  extern __shared__ __align__(16) float stage[];  // per warp: 3 rotating buffers
  const int j = blockIdx.y;
  const int warp = threadIdx.x >> 5;
  HsCtx x;
  x.stage = stage + warp * 3 * kStageW;
  x.Q4 = Q4;
  x.nq = nb >> 2;
  x.R0w = (int64_t)blockIdx.x * (NT * kHsCells) + (int64_t)kWarpSpan * warp;
  x.lane = threadIdx.x & 31;
  x.zc = (Z - 1) / 2;
  const int jc = j - x.zc;
  x.ajc = jc < 0 ? -jc : jc;
  x.sg = jc < 0 ? -1 : 1;
  const int zc = x.zc, sg = x.sg, ajc = x.ajc;
  float2 acc[kHsCells / 4];
  unsigned pmask = 0;
  hs_issue<0, NQ>(x);
  hs_issue<1, NQ>(x);
  hs_steps<0, NQ>(x, acc, pmask, thr);
  // pairs past the end of the spectrum
  const int64_t first = x.R0w + (int64_t)kHsCells * x.lane;
  if (first >= nb) pmask = 0;
  else if (first + kHsCells > nb) pmask &= (1u << ((nb - first) >> 1)) - 1u;
  // exact sums of the flagged pairs, same order as the bound
  while (pmask) {
    const int pr = __ffs(pmask) - 1;
    pmask &= pmask - 1;
    for (int c = 0; c < 2; ++c) {
      const int64_t r64 = first + 2 * pr + c;
      if (r64 < 1 || r64 >= nb) continue;
      const int r = (int)r64;
      float H = 0.f;
#pragma unroll
      for (int oi = 0; oi < NQ; ++oi) {
        const int q = frac_order(oi);
        const int jzq = zc + sg * ((2 * q * ajc + 16) >> 5);
        const float v = __ldg(P + (size_t)jzq * nb + ((2 * q * r + 16) >> 5));
        H = (oi == 0) ? v : H + v;
        if (oi == 1 || oi == 3 || oi == 7 || oi == 15) {
          const int lvl = oi == 1 ? 1 : (oi == 3 ? 2 : (oi == 7 ? 3 : 4));
          if (H >= thr.t[lvl]) {
            const unsigned long long slot = atomicAdd(count, 1ull);
            if (slot < (unsigned long long)maxc) {
              fdas_cand cd;
              cd.r_top = r;
              cd.z_idx = j;
              cd.h = 1 << lvl;
              cd.power = H;
              out[slot] = cd;
            }
          }
        }
      }
    }
  }
}

Thr thresholds_of(const fdas_plan* p) {
  Thr thr;
  for (int i = 0; i < 5; ++i) thr.t[i] = p->thr[i];
  return thr;
}

}  // namespace

int launch_pool4(fdas_plan* p, const float* d_plane, float* d_q4, fdas_cand* d_out,
                 unsigned long long* d_count) {
  const int64_t w = plane_width(p);
  const int64_t nq = w >> 2;
  dim3 grid((unsigned)((nq + 255) / 256), p->Z);
  k_pool4<<<grid, 256, 0, p->stream>>>(d_plane, d_q4, w, p->thr[0], d_out, d_count,
                                       p->max_cands);
  return cuda_check(cudaGetLastError(), "k_pool4");
}

namespace {

template <int NLEV, int NT>
int hs_launch(fdas_plan* p, const float* d_plane, const float* d_q4, fdas_cand* d_out,
              unsigned long long* d_count) {
  static int attr_dev = -1;  // the shared-memory attribute, set once per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(k_harmsum_staged<NLEV, NT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs_smem<NT>());
    if (e != cudaSuccess) return cuda_check(e, "k_harmsum_staged attr");
    attr_dev = dev;
  }
  const int64_t w = plane_width(p);
  dim3 grid((unsigned)((w + NT * kHsCells - 1) / (NT * kHsCells)), p->Z);
  k_harmsum_staged<NLEV, NT><<<grid, NT, hs_smem<NT>(), p->stream>>>(
      d_plane, d_q4, w, p->Z, thresholds_of(p), d_out, d_count, p->max_cands);
  return cuda_check(cudaGetLastError(), "k_harmsum_staged");
}

template <int NT>
int hs_dispatch(fdas_plan* p, const float* d_plane, const float* d_q4, fdas_cand* d_out,
                unsigned long long* d_count) {
  switch (p->n_levels) {
    case 2: return hs_launch<2, NT>(p, d_plane, d_q4, d_out, d_count);
    case 3: return hs_launch<3, NT>(p, d_plane, d_q4, d_out, d_count);
    case 4: return hs_launch<4, NT>(p, d_plane, d_q4, d_out, d_count);
    default: return hs_launch<5, NT>(p, d_plane, d_q4, d_out, d_count);
  }
}

}  // namespace

int launch_harmsum(fdas_plan* p, const float* d_plane, const float* d_q4, fdas_cand* d_out,
                   unsigned long long* d_count) {
  if (p->n_levels < 2) return FDAS_OK;
  return p->hs_threads == 128 ? hs_dispatch<128>(p, d_plane, d_q4, d_out, d_count)
                              : hs_dispatch<256>(p, d_plane, d_q4, d_out, d_count);
}

}  // namespace fdas
