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
// 16 distinct terms q = 1..16 serve every level: with t_q the term of
// fraction q/16, H_1 = t16, H_2 = t16 + t8, H_4 adds t4 and t12, H_8 adds
// t2, t6, t10, t14 and H_16 the odd q, one term at a time in that order.
#include <algorithm>
#include <numeric>
#include <vector>

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
// and 16 terms. A block takes top row j and NT * 64 consecutive top bins;
// warp w takes the 2048 bins from R0w = R0 + 2048 w and lane l the 64 bins
// R0w + 64 l + i, as 32 pairs of 2 bins. For fraction q the sub-harmonic bin
// is
//     rr = round(q r / 16) = q R0w/16 + 4 q l + K(q, i),  K(q, i) = (2 q i + 16) >> 5,
// so its 4-bin group, relative to the warp's first, is q l + (K(q, i) >> 2):
// lane l needs the groups q l .. q l + omax(q) (omax <= q), a compile-time
// offset from q l for every pair. Each warp copies its slice of row jz(q) of
// Q4 (32 q + 1 groups at most) into shared memory with 16-byte cp.async, two
// fractions ahead, and every lane reads its own groups as one vector per 4
// (q = 0 mod 4, 16-byte chunks XOR-swizzled within rows of 8 so that a
// quarter-warp hits 8 bank groups), per 2 (q = 2 mod 4, odd 8-byte stride) or
// one by one (odd q, odd stride); the group just past a lane's range is the
// next lane's first (a shuffle). Each pair's term is bounded by the maximum
// of the (one or two) groups its two sub-harmonic bins fall in; float
// addition is monotone, so a pair whose running bound stays below T_h holds
// no candidate at level h. The rare flagged pairs go to a list that a
// second kernel (k_harmsum_exact) sums exactly from P, in the same order,
// and compares with T_h.
__host__ __device__ constexpr int frac_order(int i) {
  return i == 0 ? 16 : i == 1 ? 8 : i == 2 ? 4 : i == 3 ? 12 : i < 8 ? 2 + 4 * (i - 4)
                                                                     : 1 + 2 * (i - 8);
}
__host__ __device__ constexpr int kq(int q, int i) { return (2 * q * i + 16) >> 5; }

constexpr int kHsCells = 64;                  // top bins per lane
constexpr int kHsPairs = kHsCells / 2;        // bin pairs per lane
constexpr int kWarpSpan = 32 * kHsCells;      // top bins per warp
// block sizes of the screen (threads) and their order tables: one-warp
// blocks are the default (each warp retires on its own and a block fits
// beside the correlation kernel's); 256 is the alternative the batch
// autotuner times
constexpr int kHsBlocks[2] = {256, 32};
constexpr int hs_block_index(int nt) { return nt == 256 ? 0 : 1; }
// last group offset a lane reads for fraction q, groups staged per warp
__host__ __device__ constexpr int omax(int q) { return kq(q, kHsCells - 1) >> 2; }
__host__ __device__ constexpr int nchunk(int q) {
  return (32 * q + (omax(q) == q ? 1 : 0) + 3) / 4;
}
// 16-byte slot of chunk C of fraction q's slice: for q = 8 and 16, lane l
// reads chunks (q/4) l + c, and XOR-ing the slot within its row of 8 with
// (row mod q/4) puts the 8 lanes of a quarter-warp on 8 different bank groups
__host__ __device__ constexpr int swz(int q, int C) {
  return (q == 8 || q == 16) ? (C ^ ((C >> 3) & (q / 4 - 1))) : C;
}
constexpr int kStageW = 4 * nchunk(16);  // largest staged slice per warp, floats
template <int NT>
constexpr size_t hs_smem() { return (size_t)3 * kStageW * (NT / 32) * sizeof(float); }

struct HsCtx {
  float* stage;  // this warp's 3 rotating buffers
  const float* Q4;  // + 4 lane
  int64_t R0w;
  // 32-bit row pitch and slice origin (nq <= 2^21 for N <= 2^24): the
  // per-fraction address work stays in 32-bit uniform registers
  uint32_t nq, r64;
  int lane, zc, sg, ajc2;
};

// copy of the warp's slice of row jz(q) of Q4 (fraction number OI in
// summation order) into rotating buffer OI % 3; the slice starts at group
// q R0w / 64, a multiple of 32, and rows hold a multiple of 4 groups, so
// every 16-byte chunk is aligned and lies entirely inside or outside the row
template <int OI, int NQ>
FDAS_DEV void hs_issue(const HsCtx& x) {
  if constexpr (OI < NQ) {
    constexpr int q = frac_order(OI);
    constexpr int NC = nchunk(q);
    float* buf = x.stage + (OI % 3) * kStageW;
    const int row = x.zc + x.sg * ((q * x.ajc2 + 16) >> 5);
    const uint32_t e_lo = (uint32_t)q * x.r64;
    // per lane: chunks C = lane + 32 i; the swizzle of chunk C depends on
    // lane only (32 i keeps the row's low bits), so the addresses are a
    // lane base plus compile-time offsets
    const float* src = x.Q4 + ((uint64_t)(uint32_t)row * x.nq + e_lo);
    float* dst = buf + 4 * swz(q, x.lane);
    constexpr int full = NC / 32, rest = NC % 32;
    if (e_lo + 4 * NC <= x.nq) {  // the whole slice lies inside the row
#pragma unroll
      for (int i = 0; i < full; ++i) cp_async16(dst + 128 * i, src + 128 * i, true);
      if (rest && x.lane < rest) cp_async16(dst + 128 * full, src + 128 * full, true);
    } else {
      const int lim = (int)(x.nq - e_lo) - 4 * x.lane;  // this lane's chunk i exists if 128 i < lim
#pragma unroll
      for (int i = 0; i < full; ++i) cp_async16(dst + 128 * i, src + 128 * i, 128 * i < lim);
      if (rest && x.lane < rest) cp_async16(dst + 128 * full, src + 128 * full, 128 * full < lim);
    }
  }
  cp_async_commit();
}

// the groups q l .. q l + omax(q) of this lane, from the staged slice
template <int q>
FDAS_DEV void hs_groups(const float* buf, int lane, float (&v)[omax(q) + 1]) {
  constexpr int OM = omax(q);
  if constexpr (q % 4 == 0) {
    constexpr int k = q / 4;
    const float4* b4 = reinterpret_cast<const float4*>(buf);
#pragma unroll
    for (int c = 0; c < k; ++c) {
      const float4 t = b4[swz(q, k * lane + c)];
      v[4 * c] = t.x;
      v[4 * c + 1] = t.y;
      v[4 * c + 2] = t.z;
      if (4 * c + 3 <= OM) v[4 * c + 3] = t.w;
    }
  } else if constexpr (q % 2 == 0) {
    constexpr int k = q / 2;
    const float2* b2 = reinterpret_cast<const float2*>(buf);
#pragma unroll
    for (int c = 0; c < k; ++c) {
      const float2 t = b2[k * lane + c];
      v[2 * c] = t.x;
      if (2 * c + 1 <= OM) v[2 * c + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int o = 0; o <= OM; ++o) v[o] = buf[q * lane + o];
  }
  if constexpr (q % 2 == 0 && OM == q) {
    // group q (l + 1) is the next lane's first; lane 31 reads it (chunk 8 q,
    // which no swizzle moves)
    const float nx = __shfl_down_sync(0xffffffffu, v[0], 1);
    v[q] = lane == 31 ? buf[32 * q] : nx;
  }
}

template <int OI, int NQ>
FDAS_DEV void hs_steps(const HsCtx& x, float2 (&acc)[kHsPairs / 2], unsigned& pmask,
                       const Thr& thr) {
  if constexpr (OI < NQ) {
    constexpr int q = frac_order(OI);
    cp_async_wait<1>();
    __syncwarp();
    hs_issue<OI + 2, NQ>(x);
    float v[omax(q) + 1];
    hs_groups<q>(x.stage + (OI % 3) * kStageW, x.lane, v);
#pragma unroll
    for (int pp = 0; pp < kHsPairs / 2; ++pp) {
      float b[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * pp + h;
        const int o1 = kq(q, 2 * i) >> 2;
        const int o2 = kq(q, 2 * i + 1) >> 2;  // o1 or o1 + 1
        b[h] = o2 == o1 ? v[o1] : fmaxf(v[o1], v[o2]);
      }
      const float2 b2 = make_float2(b[0], b[1]);
      acc[pp] = (OI == 0) ? b2 : __fadd2_rn(acc[pp], b2);
    }
    if constexpr (OI == 1 || OI == 3 || OI == 7 || OI == 15) {
      constexpr int lvl = OI == 1 ? 1 : (OI == 3 ? 2 : (OI == 7 ? 3 : 4));
      const float t = thr.t[lvl];
      float mx = fmaxf(acc[0].x, acc[0].y);
#pragma unroll
      for (int pp = 1; pp < kHsPairs / 2; ++pp) mx = fmaxf(mx, fmaxf(acc[pp].x, acc[pp].y));
      if (mx >= t) {
#pragma unroll
        for (int pp = 0; pp < kHsPairs / 2; ++pp) {
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

// Exact H_h of top bins r and r + 1 of row j, in the order of the screen,
// and the candidates among them (r >= 1, r + 1 < nb). The 2 x NQ loads are
// independent and issued together.
template <int NQ>
FDAS_DEV void hs_exact_pair(const float* __restrict__ P, int64_t nb, int j, int zc, int r,
                            const Thr& thr, fdas_cand* __restrict__ out,
                            unsigned long long* count, int64_t maxc) {
  const int jc = j - zc;
  const int ajc = jc < 0 ? -jc : jc, sg = jc < 0 ? -1 : 1;
  float H[2] = {0.f, 0.f};
#pragma unroll
  for (int oi = 0; oi < NQ; ++oi) {
    const int q = frac_order(oi);
    const float* row = P + (size_t)(zc + sg * ((2 * q * ajc + 16) >> 5)) * nb;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float v = __ldg(row + ((2 * q * (r + c) + 16) >> 5));
      H[c] = (oi == 0) ? v : H[c] + v;
    }
    if (oi == 1 || oi == 3 || oi == 7 || oi == 15) {
      const int lvl = oi == 1 ? 1 : (oi == 3 ? 2 : (oi == 7 ? 3 : 4));
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (r + c >= 1 && H[c] >= thr.t[lvl]) {
          const unsigned long long slot = atomicAdd(count, 1ull);
          if (slot < (unsigned long long)maxc) {
            fdas_cand cd;
            cd.r_top = r + c;
            cd.z_idx = j;
            cd.h = 1 << lvl;
            cd.power = H[c];
            out[slot] = cd;
          }
        }
      }
    }
  }
}

// The screen. Flagged pairs go to a list, (j << 32) | r, for k_harmsum_exact;
// a lane whose flags do not fit the list (capacity cap) sums them itself.
// A block takes tile order[blockIdx.x] = j * ntile + t (row j, bins from
// t * NT * 64), or tile blockIdx.x itself without an order table.
template <int NLEV, int NT>
__global__ void __launch_bounds__(NT, NT == 32 ? 32 : 0) k_harmsum_staged(
    const float* __restrict__ P, const float* __restrict__ Q4, int64_t nb, int Z, Thr thr,
    const uint32_t* __restrict__ order, int64_t ntile,
    unsigned long long* __restrict__ list, unsigned long long* nlist, int64_t cap,
    fdas_cand* __restrict__ out, unsigned long long* count, int64_t maxc) {
  constexpr int NQ = 1 << (NLEV - 1);
  extern __shared__ __align__(16) float stage[];  // per warp: 3 rotating buffers
  // tile ids are below 2^32 (the order tables exist only then)
  const uint32_t tile = order ? __ldg(order + blockIdx.x) : blockIdx.x;
  const int j = (int)(tile / (uint32_t)ntile);
  const int64_t t = (int64_t)(tile - (uint32_t)j * (uint32_t)ntile);
  const int warp = threadIdx.x >> 5;
  HsCtx x;
  x.stage = stage + warp * 3 * kStageW;
  x.lane = threadIdx.x & 31;
  x.Q4 = Q4 + 4 * x.lane;
  x.nq = (uint32_t)(nb >> 2);
  x.R0w = t * (NT * kHsCells) + (int64_t)kWarpSpan * warp;
  x.r64 = (uint32_t)(x.R0w >> 6);
  x.zc = (Z - 1) / 2;
  const int jc = j - x.zc;
  x.ajc2 = 2 * (jc < 0 ? -jc : jc);
  x.sg = jc < 0 ? -1 : 1;
  float2 acc[kHsPairs / 2];
  unsigned pmask = 0;
  hs_issue<0, NQ>(x);
  hs_issue<1, NQ>(x);
  hs_steps<0, NQ>(x, acc, pmask, thr);
  // pairs past the end of the spectrum (nb - first is even)
  const int64_t first = x.R0w + (int64_t)kHsCells * x.lane;
  if (first >= nb) pmask = 0;
  else if (first + kHsCells > nb) pmask &= (1u << ((nb - first) >> 1)) - 1u;
  if (pmask == 0) return;
  const unsigned n = (unsigned)__popc(pmask);
  const unsigned long long base = atomicAdd(nlist, (unsigned long long)n);
  const unsigned long long key = (unsigned long long)j << 32;
  for (unsigned k = 0; pmask; ++k) {
    const int r = (int)(first + 2 * (__ffs(pmask) - 1));
    pmask &= pmask - 1;
    if (base + k < (unsigned long long)cap) list[base + k] = key | (unsigned)r;
    else hs_exact_pair<NQ>(P, nb, j, x.zc, r, thr, out, count, maxc);
  }
}

// Exact sums of the listed pairs (grid-stride over the list).
template <int NLEV>
__global__ void __launch_bounds__(256) k_harmsum_exact(
    const float* __restrict__ P, const unsigned long long* __restrict__ list,
    const unsigned long long* nlist, int64_t cap, int64_t nb, int Z, Thr thr,
    fdas_cand* __restrict__ out, unsigned long long* count, int64_t maxc) {
  constexpr int NQ = 1 << (NLEV - 1);
  const int64_t n = min((int64_t)*nlist, cap);
  const int zc = (Z - 1) / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long e = list[i];
    hs_exact_pair<NQ>(P, nb, (int)(e >> 32), zc, (int)(e & 0xffffffffu), thr, out, count, maxc);
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
  e = cudaMemsetAsync(p->hs_nlist, 0, sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return cuda_check(e, "memset flagged-pair count");
  const int64_t w = plane_width(p);
  const int64_t ntile = (w + NT * kHsCells - 1) / (NT * kHsCells);
  const uint32_t* order = p->hs_order_w == w ? p->hs_order[hs_block_index(NT)] : nullptr;
  k_harmsum_staged<NLEV, NT><<<(unsigned)(ntile * p->Z), NT, hs_smem<NT>(), p->stream>>>(
      d_plane, d_q4, w, p->Z, thresholds_of(p), order, ntile, p->hs_list, p->hs_nlist,
      kHsListCap, d_out, d_count, p->max_cands);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(e, "k_harmsum_staged");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_check(e, "SM count");
  k_harmsum_exact<NLEV><<<16 * sms, 256, 0, p->stream>>>(d_plane, p->hs_list, p->hs_nlist,
                                                        kHsListCap, w, p->Z, thresholds_of(p),
                                                        d_out, d_count, p->max_cands);
  return cuda_check(cudaGetLastError(), "k_harmsum_exact");
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

// The screen's tile order: ascending angle (j - zc) / (t + 1/2) about the
// centre row. The sub-harmonic cells of top cell (j, r) lie near the ray
// from (zc, 0) through it, at (zc + q (j - zc)/16, q r/16), so tiles of one
// angle share the 4-bin maxima they read; run together they take them from
// DRAM about once (an LRU model of the 126 MB L2 at the 2^23-sample,
// 201-row size: 0.84 GB of DRAM reads, the size of the maxima, against
// 2.2 GB row by row). Made on the host for the current plane width at plan
// set-up, outside any stream capture; a launch whose width differs uses
// the row-by-row order.
void free_hs_order(fdas_plan* p) {
  for (int k = 0; k < 2; ++k) {
    if (p->hs_order[k]) cudaFree(p->hs_order[k]);
    p->hs_order[k] = nullptr;
  }
  p->hs_order_w = 0;
}

int make_hs_order(fdas_plan* p) {
  const int64_t w = plane_width(p);
  if (p->hs_order[0] && p->hs_order_w == w) return FDAS_OK;
  for (int k = 0; k < 2; ++k)
    if (p->hs_order[k]) {
      const int NT = kHsBlocks[k];
      const int64_t ntile = (p->hs_order_w + NT * kHsCells - 1) / (NT * kHsCells);
      p->device_bytes -= (int64_t)sizeof(uint32_t) * ntile * p->Z;
    }
  free_hs_order(p);
  const int zc = (p->Z - 1) / 2;
  for (int k = 0; k < 2; ++k) {
    const int NT = kHsBlocks[k];
    const int64_t ntile = (w + NT * kHsCells - 1) / (NT * kHsCells);
    const int64_t n = ntile * p->Z;
    if (n > (int64_t)UINT32_MAX) return FDAS_OK;  // row-by-row order
    std::vector<uint32_t> ord((size_t)n);
    std::iota(ord.begin(), ord.end(), 0u);
    std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
      const int64_t ja = a / ntile, ta = a - ja * ntile, jb = b / ntile, tb = b - jb * ntile;
      // compare (ja - zc) / (ta + 1/2) with (jb - zc) / (tb + 1/2) exactly
      const int64_t l = (ja - zc) * (2 * tb + 1), r = (jb - zc) * (2 * ta + 1);
      if (l != r) return l < r;
      return ta != tb ? ta < tb : ja < jb;
    });
    uint32_t* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, sizeof(uint32_t) * (size_t)n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(FDAS_ERR_NOMEM, "tile order table");
    }
    p->hs_order[k] = d;
    p->device_bytes += (int64_t)sizeof(uint32_t) * n;
    e = cudaMemcpy(d, ord.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(e, "tile order upload");
  }
  p->hs_order_w = w;
  return FDAS_OK;
}

int launch_harmsum(fdas_plan* p, const float* d_plane, const float* d_q4, fdas_cand* d_out,
                   unsigned long long* d_count) {
  if (p->n_levels < 2) return FDAS_OK;
  return p->hs_threads == 256 ? hs_dispatch<256>(p, d_plane, d_q4, d_out, d_count)
                              : hs_dispatch<32>(p, d_plane, d_q4, d_out, d_count);
}

}  // namespace fdas
