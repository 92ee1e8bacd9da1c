// Steps 3-7 of Section 4: overlapped segments, segment FFT, multiplication by
// the conjugated template spectra, inverse FFT, power and edge removal; the
// result is the f-fdot power plane of Eq. 1,
//     P[j][r] = | sum_{d=-m/2}^{m/2-1} Xw[r+d] tau_{z_j}(d) |^2,
// computed by overlap-save (Section 2): segment s holds Xw[s V - m/2 + i],
// i < L (zero outside the spectrum); the circular correlation of a segment
// with the template is exact for the V = L - m outputs i = m/2 .. m/2+V-1,
// which are kept as r = s V + (i - m/2).
#include "fdas_common.cuh"
#include "fdas_internal.h"
#include "fdas_emit.cuh"
#include "fdas_tmem.cuh"

namespace fdas {
namespace {

constexpr int kNT = 256;
// pairs per chunk of the correlation's dynamically shared tail
constexpr int kChunk = 8;

// Step 3 + step 4: gather segment s (zero-filled at the spectrum edges) and
// FFT it forward; seg[s][k] in natural order.
template <int L>
__global__ void __launch_bounds__(kNT) k_segments(const float2* __restrict__ Xw,
                                                  float2* __restrict__ seg, int64_t nb, int V,
                                                  int m, const float2* __restrict__ tw) {
  extern __shared__ float2 sbuf[];
  const int tid = threadIdx.x;
  const int s = blockIdx.x;
  const int64_t base = (int64_t)s * V - m / 2;
  for (int i = tid; i < L; i += kNT) {
    const int64_t g = base + i;
    sbuf[i] = (g >= 0 && g < nb) ? Xw[g] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  block_fft<L, kFwd, kNT, 1>(sbuf, tw, tid);
  // packed layout (see the correlation kernel)
  constexpr int RA2 = L / 512;
  float4* out = reinterpret_cast<float4*>(seg) + (size_t)s * (L / 2);
  for (int sl = tid; sl < L / 2; sl += kNT) {
    const int u = sl & 15, ab = sl >> 4;
    const int a = ab % RA2, b = ab / RA2;
    const int k0 = 2 * u + 32 * (a + RA2 * b);
    const float2 x0 = sbuf[k0], x1 = sbuf[k0 + 1];
    out[sl] = make_float4(x0.x, x1.x, x0.y, x1.y);
  }
}

// Packed layout of a length-L spectrum (segments and templates alike): with
// k = k1 + 32 k2, k1 = 2u + e (u < 16, e in {0, 1}), k2 = a + RA2 b
// (a < RA2 = L/512, b < 16), slot (b RA2 + a) 16 + u holds the float4
// (re[k1=2u], re[2u+1], im[2u], im[2u+1]): one 16-byte load gives a thread
// the packed pair it transforms.
template <int L>
__host__ __device__ constexpr int pk_ra2() { return L / 512; }

// Steps 5-7, fused: one pass per (segment, template) pair through
//   Y = F_s * T_z  ->  inverse FFT  ->  |.|^2  ->  keep the V valid outputs,
// with the complex plane never leaving the SM. Length-L inverse FFT,
// L = 32 NA, NA = 16 RA2 (= threads), n = n2 + NA n1, n2 = c + 16 d:
//   A1 radix-16 over b of Y[k1 + 32 (a + RA2 b)], times w_NA^{a c}
//        thread (u, a): the pair k1 = 2u, 2u+1, packed
//   A2 radix-RA2 over a -> Z[k1][c + 16 d], times w_L^{k1 (c + 16 d)}
//        16/RA2 packed butterflies (u, c) per thread
//   B  radix-32 over k1 -> c[n2 + NA n1]     thread n2 (two packed radix-16
//        DFTs of the even and odd k1, then a scalar radix-2 combination)
// All butterflies work on packed f32x2 pairs (two transforms per FP32
// instruction). Two shared-memory exchanges per pair and three CTA barriers
// (A1 -> A2, A2 -> B, and B's reads done before the next pair's A1 writes);
// the segment spectrum and the thread's B-stage twiddles live in tensor
// memory for the whole
// sweep over templates; template spectra stream from L2. Besides the plane
// row the kernel writes the 4-bin maxima Q4[z][r/4] (used to screen the
// harmonic sums) and emits the h = 1 candidates. One wave of CTAs; each takes
// a contiguous range of 3/4 of the (segment, template) pairs split evenly,
// then chunks of the rest from a device counter.
template <int L>
struct Corr {
  static constexpr int T = L / 32;
  static constexpr int NA = L / 32;
  static constexpr int RA2 = NA / 16;
  static constexpr int NB2 = 16 / RA2;
  static constexpr int NW = T / 32;
  static constexpr int XF4 = L / 2;  // the exchange buffer: L/2 packed pairs
  static constexpr int NGROUPS = (NW + 3) / 4;  // warps w and w + 4 share TMEM lanes
  static constexpr int NCOLS = 128 * NGROUPS;   // per thread: 64 (F) + 64 (B twiddles)
  static constexpr int MAXCTA = 512 / NCOLS;
  // registers per thread: two (L = 8192) or four CTAs per SM leave 4 K of the
  // SM's 64 K registers free, room for a warp of another trial lane's
  // harmonic-sum screen beside them (measured 0.8% faster alone, 0.5% per
  // lane-overlapped trial, against 128; 112 spills)
  static constexpr int MAXREG = 120;
  // exchange buffer, A1 twiddles, power row (L floats), 4-bin maxima row (L/4)
  static constexpr size_t SMEM = 16 * (size_t)(XF4 + RA2 * 17) + 4 * (size_t)L + (size_t)L;
};

// Exchange-buffer slot of row r, packed pair u: 16 float4 per row, the pair
// index XOR-swizzled by r % 8 so that 8 lanes reading one column of 8
// consecutive rows, or 8 consecutive columns of one row, hit distinct banks.
// Rows are r = 16 a + c (A1 -> A2, a over the A2 radix) and n2 = c + 16 d
// (A2 -> B): A2 thread (u, c) reads rows {16 a + c} and writes its outputs d
// into rows {16 d + c}, the same slots, so it needs no barrier in between.
FDAS_DEV int xsw(int r, int u) { return r * 16 + (u ^ (r & 7)); }

// Bulk copy (TMA engine, no tensor map) of `bytes` from shared to global
// memory; both addresses 16-byte aligned, bytes a multiple of 16. The lines
// are marked evict-first in L2: the plane and its maxima stream out to HBM
// and would otherwise push the template bank and segment spectra, which
// every pair re-reads, out of L2 (measured: the correlation 2.28 -> 2.07 ms).
FDAS_DEV void bulk_s2g(void* gdst, const void* ssrc, uint32_t bytes) {
  uint64_t policy;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
  asm volatile(
      "cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
      "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes), "l"(policy)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
FDAS_DEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
FDAS_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
FDAS_DEV void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

FDAS_DEV c2 c2_of(float4 v) { return c2{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
FDAS_DEV float4 f4_of(c2 v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }

template <int L, int IB>
__global__ void __maxnreg__(Corr<L>::MAXREG)
    k_correlate_fused(const float4* __restrict__ seg4, const float4* __restrict__ bank4,
                      float* __restrict__ plane, float* __restrict__ q4, int64_t nb, int Z, int V,
                      int m, int64_t n_pairs, const float2* __restrict__ twL, float thr1,
                      fdas_cand* __restrict__ cands, unsigned long long* count, int64_t maxc,
                      unsigned long long* next) {
  constexpr int ib = IB;
  using C = Corr<L>;
  constexpr int T = C::T, NA = C::NA, RA2 = C::RA2, NB2 = C::NB2;
  constexpr int L2 = L / 2;
  extern __shared__ float4 smem4[];
  float4* X = smem4;
  // (c, c, s, s) of exp(+2 pi i a c / NA), a < RA2, c < 16, at a * 17 + c: a
  // warp reads two rows a at once, which the padding puts on other banks
  float4* twA = smem4 + C::XF4;
  float* Ps = reinterpret_cast<float*>(twA + RA2 * 17);
  float* Q4s = Ps + L;  // 4-bin maxima of the row slice (bulk path)
  __shared__ uint32_t s_tmem;
  // Integer-bin planes with m % 16 == 0 leave the kernel by bulk copies: the
  // valid slice of the power row (Ps + m/2, 4 nvalid bytes) and its 4-bin
  // maxima (Q4s, nvalid bytes), both 16-byte aligned at either end. Thread 0
  // issues the copies of a pair after the first CTA barrier of the next pair
  // the CTA does (every thread has fenced its shared-memory writes of the
  // pair before it) and waits until they have read shared memory before the
  // second one, after which the next pair rewrites Ps and Q4s.
  const bool bulk = IB == 0 && (m % 16) == 0;
  auto issue_bulk = [&](int64_t pp) {  // pair pp's row slice (thread 0)
    const int ps = (int)(pp / Z);
    const int pz = (int)(pp - (int64_t)ps * Z);
    const int64_t pr0 = (int64_t)ps * V;
    const uint32_t nv = (uint32_t)min((int64_t)V, nb - pr0);
    if (plane) bulk_s2g(plane + (size_t)pz * nb + pr0, Ps + m / 2, 4 * nv);
    if (q4) bulk_s2g(q4 + (size_t)pz * (nb >> 2) + (pr0 >> 2), Q4s, nv);
  };
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < RA2 * 16; e += T) {
    const float2 w = cconj(__ldg(twL + (((e >> 4) * (e & 15) * 32) & (L - 1))));
    twA[(e >> 4) * 17 + (e & 15)] = make_float4(w.x, w.x, w.y, w.y);
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, C::NCOLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase =
      s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
  // B-stage twiddles exp(+2 pi i k1 n2 / L), k1 = 2u, 2u+1, n2 = c + 16 d, for
  // this thread's A2 butterflies -> tensor-memory columns 64..127
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float f[16];
#pragma unroll
    for (int w4 = 0; w4 < 4; ++w4) {
      const int idx = q * 4 + w4;  // = i * RA2 + d
      const int i = idx / RA2, d = idx % RA2;
      const int g = tid + T * i;
      const int u = g & 15, c = g >> 4;
      const int n2 = c + 16 * d;
      const float2 w0 = cconj(__ldg(twL + ((2 * u * n2) & (L - 1))));
      const float2 w1 = cconj(__ldg(twL + (((2 * u + 1) * n2) & (L - 1))));
      f[4 * w4] = w0.x;
      f[4 * w4 + 1] = w1.x;
      f[4 * w4 + 2] = w0.y;
      f[4 * w4 + 3] = w1.y;
    }
    tmem_st16(tbase + 64 + 16 * q, f);
  }
  tmem_wait_st();

  const int u1 = tid & 15, a1 = tid >> 4;  // A1 role
  const int half_m = m / 2;
  const int64_t nq = nb >> 2;
  // The first 3/4 of the pairs are split evenly in contiguous ranges, one
  // per CTA (the segment spectrum is reloaded only when the segment
  // changes); the rest go out in chunks of kChunk consecutive pairs from the
  // counter `next` (zeroed before the launch), so that CTAs on SMs that run
  // faster take more of the tail. Thread 0 claims the next chunk during the
  // last pair of a range, before that pair's first CTA barrier; the claim is
  // read after the range, and its slot alternates with the range parity.
  const int64_t nstat = n_pairs * 3 / 4 / kChunk * kChunk;
  const int64_t ndyn = (n_pairs - nstat + kChunk - 1) / kChunk;
  __shared__ int64_t s_next[2];
  int s_cur = -1;
  int64_t p_prev = -1;  // the last pair done, whose row slice is not yet copied out
  int64_t chunk = -1;   // -1: this CTA's static range
  for (int k = 0; chunk < ndyn; ++k) {
    const int64_t q0 = chunk < 0 ? (int64_t)blockIdx.x * nstat / gridDim.x : nstat + chunk * kChunk;
    const int64_t q1 =
        chunk < 0 ? (int64_t)(blockIdx.x + 1) * nstat / gridDim.x : min(q0 + kChunk, n_pairs);
    if (q1 <= q0) {  // an empty static range claims its first chunk here
      if (tid == 0) s_next[k & 1] = (int64_t)atomicAdd(next, 1ull);
      __syncthreads();
    }
    for (int64_t p = q0; p < q1; ++p) {
      if (tid == 0 && p == q1 - 1) s_next[k & 1] = (int64_t)atomicAdd(next, 1ull);
      const int s = (int)(p / Z);
      const int z = (int)(p - (int64_t)s * Z);
      if (s != s_cur) {  // segment spectrum -> tensor memory columns 0..63
        const float4* fs = seg4 + (size_t)s * L2 + a1 * 16 + u1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float f[16];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 v = __ldg(fs + (q * 4 + i) * RA2 * 16);
            f[4 * i] = v.x;
            f[4 * i + 1] = v.y;
            f[4 * i + 2] = v.z;
            f[4 * i + 3] = v.w;
          }
          tmem_st16(tbase + 16 * q, f);
        }
        tmem_wait_st();
        s_cur = s;
      }
      // ---- A1
      c2 v[16];
      const float4* tz = bank4 + (size_t)z * L2 + a1 * 16 + u1;
#pragma unroll
      // (L2 only: the shared-memory carve-out leaves L1 too small to keep
      // a 64 KB template row; measured 1% faster than the read-only path)
      for (int b = 0; b < 16; ++b) v[b] = c2_of(__ldcg(tz + b * RA2 * 16));
#pragma unroll
      for (int q = 0; q < 4; q += 2) {
        float f[32];
        tmem_ld16x2(tbase + 16 * q, tbase + 16 * q + 16, f);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          v[q * 4 + i] = c2_mul(v[q * 4 + i], c2{make_float2(f[4 * i], f[4 * i + 1]),
                                                make_float2(f[4 * i + 2], f[4 * i + 3])});
      }
      dft_pairs<16, kInv>(v);
#pragma unroll
      for (int c = 1; c < 16; ++c) {
        const float4 tw = twA[a1 * 17 + c];
        v[brev<16>(c)] = c2_mul_cs(v[brev<16>(c)], make_float2(tw.x, tw.y), make_float2(tw.z, tw.w));
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) X[xsw(a1 * 16 + c, u1)] = f4_of(v[brev<16>(c)]);
      __syncthreads();
      if (bulk && tid == 0 && p_prev >= 0) issue_bulk(p_prev);  // the previous pair's row slice
      // ---- A2
      c2 w[NB2][RA2];
#pragma unroll
      for (int i = 0; i < NB2; ++i) {
        const int g = tid + T * i;
        const int u = g & 15, c = g >> 4;
#pragma unroll
        for (int a = 0; a < RA2; ++a) w[i][a] = c2_of(X[xsw(a * 16 + c, u)]);
      }
      // (no barrier: each thread writes its results into the slots it read)
#pragma unroll
      for (int i = 0; i < NB2; ++i) {
        dft_pairs<RA2, kInv>(w[i]);
        const int g = tid + T * i;
        const int u = g & 15, c = g >> 4;
#pragma unroll
        for (int d0 = 0; d0 < RA2; d0 += 4) {
          float f[16];
          tmem_ld16(tbase + 64 + 4 * (i * RA2 + d0), f);
#pragma unroll
          for (int dd = 0; dd < 4; ++dd) {
            const int d = d0 + dd;
            const c2 t = c2_mul_cs(w[i][brev<RA2>(d)], make_float2(f[4 * dd], f[4 * dd + 1]),
                                   make_float2(f[4 * dd + 2], f[4 * dd + 3]));
            X[xsw(16 * d + c, u)] = f4_of(t);
          }
        }
      }
      // the copies of the previous pair's row slice have read Ps and Q4s
      if (bulk && tid == 0 && p_prev >= 0) bulk_wait_read();
      __syncthreads();
      // ---- B
      c2 y[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) y[u] = c2_of(X[xsw(tid, u)]);
      // every warp has read X: the next pair's A1 may overwrite it
      __syncthreads();
      // every output goes to Ps[n] (room for all L); the valid V start at half_m
      dft32_dit<kInv>(y, [&](int e, float2 o) { Ps[tid + NA * e] = cnorm(o); });
      // Outputs n .. n+3 (n % 4 == 0) come from threads n % NA .. +3, lanes of
      // one warp; so each warp stores the float4s its own lanes produced and a
      // warp barrier suffices (the next pair writes Ps only after its first
      // CTA barrier, which every warp reaches after this output stage).
      __syncwarp();
      // coalesced float4 stores of the plane row slice, its 4-bin maxima and
      // the h = 1 candidates; r = s V + i, i < V, r < nb
      const int64_t r0 = (int64_t)s * V;
      int64_t nvalid = nb - r0;
      if (nvalid > V) nvalid = V;
      const int nhi = half_m + (int)nvalid;  // valid outputs n in [half_m, nhi), multiples of 4 apart
      // (half-bin planes, ib = 1: template row z = 2j + e fills columns 2r + e
      // of plane row j; rows 2j and 2j+1 are consecutive pairs, so each sector
      // is completed in L2 before it is written back)
      float* prow = plane ? plane + (size_t)(z >> ib) * (nb << ib) + (r0 << ib) + (z & ib) : nullptr;
      float* qrow = q4 ? q4 + (size_t)z * nq + (r0 >> 2) : nullptr;
      const float4* P4 = reinterpret_cast<const float4*>(Ps);
      const int lane = tid & 31;
      // lane: 4 outputs starting at n = NA j + 32 warp + 4 (lane % 8), j = lane / 8 + 4 i
      const int nw = 32 * warp + 4 * (lane & 7);
      bool hit = false;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = NA * ((lane >> 3) + 4 * i) + nw;
        if (n >= half_m && n < nhi) {
          const float4 p4 = P4[n >> 2];
          const int k = (n - half_m) >> 2;  // float4 index in the row slice
          const float mx = fmaxf(fmaxf(p4.x, p4.y), fmaxf(p4.z, p4.w));
          if (bulk) {
            Q4s[k] = mx;  // the plane row itself leaves from Ps
          } else if (prow) {
            if constexpr (IB) {
              prow[8 * k] = p4.x;
              prow[8 * k + 2] = p4.y;
              prow[8 * k + 4] = p4.z;
              prow[8 * k + 6] = p4.w;
            } else {
              reinterpret_cast<float4*>(prow)[k] = p4;
            }
          }
          if (qrow && !bulk) qrow[k] = mx;
          hit |= mx >= thr1;
        }
      }
      if (cands && __any_sync(0xffffffffu, hit)) {
        // rare: some power this warp stored reached T_1; the warp scans its
        // own float4s again and appends
#pragma unroll 1
        for (int i = 0; i < 8; ++i) {
          const int n = NA * ((lane >> 3) + 4 * i) + nw;
          const bool in = n >= half_m && n < nhi;
          const float4 p4 = in ? P4[n >> 2] : make_float4(0.f, 0.f, 0.f, 0.f);
          const int rk = (int)(r0 + (n - half_m));
          emit(in && rk >= 1 && p4.x >= thr1, rk, z, 1, p4.x, cands, count, maxc);
          emit(in && p4.y >= thr1, rk + 1, z, 1, p4.y, cands, count, maxc);
          emit(in && p4.z >= thr1, rk + 2, z, 1, p4.z, cands, count, maxc);
          emit(in && p4.w >= thr1, rk + 3, z, 1, p4.w, cands, count, maxc);
        }
      }
      // this thread's Ps and Q4s writes, visible to the bulk copies
      if (bulk) fence_proxy_async_shared();
      p_prev = p;
    }
    chunk = s_next[k & 1];
  }
  if (bulk) {  // the last pair's row slice
    __syncthreads();
    if (tid == 0 && p_prev >= 0) {
      issue_bulk(p_prev);
      bulk_wait_all();
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(s_tmem, C::NCOLS);
}

// Natural-order copy of the packed template bank (for export).
template <int L>
__global__ void k_bank_natural(const float* __restrict__ bankf, float2* __restrict__ out, int Z) {
  constexpr int RA2 = pk_ra2<L>();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)Z * L) return;
  const int j = (int)(i / L), k = (int)(i % L);
  const int e = k & 1, u = (k & 31) >> 1, k2 = k >> 5;
  const int slot = ((k2 / RA2) * RA2 + (k2 % RA2)) * 16 + u;
  const float* f = bankf + ((size_t)j * (L / 2) + slot) * 4;
  out[i] = make_float2(f[e], f[2 + e]);
}

template <int L>
int seg_launch(fdas_plan* p, const float2* Xw) {
  const size_t smem = sizeof(float2) * L;
  cudaError_t e = cudaFuncSetAttribute(k_segments<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "k_segments attr");
  k_segments<L><<<p->S, kNT, smem, p->stream>>>(Xw, p->seg, p->nb, p->V, p->m, p->tw_L);
  return cuda_check(cudaGetLastError(), "k_segments");
}

template <int L, int IB>
int corr_launch(fdas_plan* p, float* plane, float* q4, fdas_cand* cands,
                unsigned long long* count) {
  using C = Corr<L>;
  int dev = 0, sms = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // Cap resident CTAs per SM so that their tensor-memory columns fit (512):
  // request enough shared memory that at most MAXCTA CTAs fit on an SM.
  size_t smem = C::SMEM;
  const size_t cap = (size_t)smem_sm / (C::MAXCTA + 1) + 1;
  if (smem + 1024 < cap) smem = cap - 1024 + 16;
  cudaError_t e = cudaFuncSetAttribute(k_correlate_fused<L, IB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "k_correlate_fused attr");
  e = cudaFuncSetAttribute(k_correlate_fused<L, IB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return cuda_check(e, "k_correlate_fused carveout");
  // Resident CTAs per SM from the kernel's own resource use (registers in
  // units of 8 per thread, shared memory incl. the 1 KB per-CTA reserve,
  // threads), capped by the tensor-memory budget.
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_correlate_fused<L, IB>);
  if (e != cudaSuccess) return cuda_check(e, "k_correlate_fused attributes");
  int regs_sm = 0, thr_sm = 0;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * C::T;
  int occ = regs_sm / regs_cta;
  const int by_smem = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
  if (by_smem < occ) occ = by_smem;
  if (thr_sm / C::T < occ) occ = thr_sm / C::T;
  if (occ > C::MAXCTA) occ = C::MAXCTA;
  if (occ < 1) return set_error(FDAS_ERR_CUDA, "k_correlate_fused cannot be resident");
  p->corr_ctas_per_sm = occ;
  // half-bin planes: 2Z template rows, the plane alone (4-bin maxima and
  // h = 1 candidates of the interleaved plane come from k_pool4)
  constexpr int ib = IB;
  const int zrows = p->Z << ib;
  const int64_t n_pairs = (int64_t)p->S * zrows;
  int64_t grid = (int64_t)occ * sms;
  if (grid > n_pairs) grid = n_pairs;
  p->corr_grid = (int)grid;
  e = cudaMemsetAsync(p->hs_nlist + 1, 0, sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return cuda_check(e, "clear the pair counter");
  k_correlate_fused<L, IB><<<(unsigned)grid, C::T, smem, p->stream>>>(
      reinterpret_cast<const float4*>(p->seg),
      reinterpret_cast<const float4*>(ib ? p->bank_ib : p->bank), plane, ib ? nullptr : q4, p->nb,
      zrows, p->V, p->m, n_pairs, p->tw_L, p->thr[0], ib ? nullptr : cands, count, p->max_cands,
      p->hs_nlist + 1);
  return cuda_check(cudaGetLastError(), "k_correlate_fused");
}

template <int L>
int bank_natural_launch(fdas_plan* p, float2* out) {
  const int64_t n = (int64_t)p->Z * L;
  k_bank_natural<L><<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(
      reinterpret_cast<const float*>(p->bank), out, p->Z);
  return cuda_check(cudaGetLastError(), "k_bank_natural");
}

}  // namespace

int launch_bank_natural(fdas_plan* p, float2* d_out) {
  switch (p->L) {
    case 2048: return bank_natural_launch<2048>(p, d_out);
    case 4096: return bank_natural_launch<4096>(p, d_out);
    case 8192: return bank_natural_launch<8192>(p, d_out);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported segment length");
}

int launch_segments(fdas_plan* p, const float2* d_white) {
  switch (p->L) {
    case 2048: return seg_launch<2048>(p, d_white);
    case 4096: return seg_launch<4096>(p, d_white);
    case 8192: return seg_launch<8192>(p, d_white);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported segment length");
}

int launch_correlate(fdas_plan* p, float* d_plane, float* d_q4, fdas_cand* d_cands,
                     unsigned long long* d_count) {
  switch (p->L) {
    case 2048:
      return p->interbin ? corr_launch<2048, 1>(p, d_plane, d_q4, d_cands, d_count)
                         : corr_launch<2048, 0>(p, d_plane, d_q4, d_cands, d_count);
    case 4096:
      return p->interbin ? corr_launch<4096, 1>(p, d_plane, d_q4, d_cands, d_count)
                         : corr_launch<4096, 0>(p, d_plane, d_q4, d_cands, d_count);
    case 8192:
      return p->interbin ? corr_launch<8192, 1>(p, d_plane, d_q4, d_cands, d_count)
                         : corr_launch<8192, 0>(p, d_plane, d_q4, d_cands, d_count);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported segment length");
}

}  // namespace fdas
