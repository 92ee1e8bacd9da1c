// Steps 5-7 of Section 4 for segments of L = 8192 bins: multiplication of a
// segment spectrum by a conjugated template spectrum, inverse FFT, power and
// edge removal (overlap-save, Section 2), i.e. the rows of the power plane of
// Eq. 1,
//     P[j][r] = | sum_{d=-m/2}^{m/2-1} Xw[r+d] tau_{z_j}(d) |^2 ,
// for r = s V + i, i < V, from segment s (bins s V - m/2 .. s V - m/2 + L - 1).
//
// One CTA of 512 threads transforms one (segment, template) pair at a time,
// 16 complex points per thread. Complex values are kept as (re, im) pairs in
// 64-bit registers, so a complex add or subtract is one packed f32x2
// instruction and a thread needs only its 16 points in registers for a
// radix-16 step: two CTAs (32 warps) fit on an SM.
//
// Index split of the inverse DFT y[n] = sum_k Y[k] exp(+2 pi i k n / L):
//   k = k1 + 32 a + 512 b      (k1 < 32, a < 16, b < 16)
//   n = c + 16 d + 256 n1      (c < 16, d < 16, n1 < 32), n2 = c + 16 d
//   A1  thread (k1, a): 16-point DFT over b -> c, times exp(2 pi i a c / 256)
//   A2  thread (k1, c): 16-point DFT over a -> d, times exp(2 pi i k1 n2 / L)
//   B   thread (n2, h): 16-point DFT over j of Z[k1 = 2 j + h] -> E (h = 0)
//       or O (h = 1); the pair of lanes h = 0, 1 swaps halves by shuffle and
//       forms y[n2 + 256 r] = E[r] + w O[r], y[n2 + 256 (r + 16)] = E[r] - w O[r],
//       w = exp(2 pi i r / 32), and only |y|^2 is kept.
// Warp w is a in A1, c in A2 and d in B; the lane is k1 in A1 and A2, and
// 2 c + h in B. The segment spectrum (this thread's 16 points) and the A2
// twiddles live in tensor memory for the whole sweep over templates.
// Template and segment spectra are stored in natural order (float2).
#include "fdas_common.cuh"
#include "fdas_emit.cuh"
#include "fdas_internal.h"
#include "fdas_tmem.cuh"

namespace fdas {
namespace {

constexpr int kL16 = 8192;
constexpr int kT16 = 512;                 // threads per CTA = L / 16
constexpr int kPs16 = kL16;               // power row (permuted, see ps_idx)
constexpr int kCols16 = 256;              // TMEM columns per CTA
constexpr size_t kSmem16 = sizeof(float2) * kL16 + sizeof(float) * kPs16 + sizeof(float2) * 256;

// Exchange-buffer slot of (x, c, k1): rows of 32 float2 indexed by k1, the
// column XOR-swizzled by 2 c so that B's reads (16 rows c at once, two
// adjacent k1 each) hit distinct banks; A1 writes (x = a) and A2 reads and
// writes (x = a, then x = d) touch one whole row per warp instruction, and A2
// writes exactly the slots it read.
FDAS_DEV int xslot(int x, int c, int k1) { return x * 512 + c * 32 + (k1 ^ ((2 * c) & 31)); }

// Power-row index of output n = n2 + 256 n1: bit 4 of n2 flipped when bit 3
// and bit 0 of n1 differ (a permutation within each row of 256 that keeps
// float4 groups whole), so the B-stage stores (lanes h = 0, 1 write n1 that
// differ in bit 3) and the float4 reads of the output stage (8 lanes cover
// two adjacent n1) are free of bank conflicts.
FDAS_DEV int ps_idx(int n) {
  const int n1 = n >> 8;
  return n ^ (16 * (((n1 >> 3) ^ n1) & 1));
}

FDAS_DEV float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
FDAS_DEV float2 f2_sub(float2 a, float2 b) { return p_sub(a, b); }
// a * (c + i s), scalar (the same FMA-pipe cost as the packed form)
FDAS_DEV float2 f2_rot(float2 a, float c, float s) {
  return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}
FDAS_DEV float2 f2_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// v * exp(+2 pi i e / 16), e a constant after unrolling: quarter turns are
// swaps, eighth turns two adds and two multiplies.
FDAS_DEV float2 f2_tw16(float2 v, int e) {
  e &= 15;
  if (e == 0) return v;
  if (e == 4) return make_float2(-v.y, v.x);
  if (e == 8) return make_float2(-v.x, -v.y);
  if (e == 12) return make_float2(v.y, -v.x);
  const int k = 2 * e;  // in 32nds of a turn
  float c = kCos32[k & 15], sn = kSin32[k & 15];
  if (k >= 16) {
    c = -c;
    sn = -sn;
  }
  if (c == sn) return make_float2((v.x - v.y) * c, (v.x + v.y) * c);
  if (c == -sn) return make_float2((v.x + v.y) * c, (v.y - v.x) * c);
  return f2_rot(v, c, sn);
}

// In-place inverse 4-point DFT, X_k = sum_n a_n exp(+2 pi i n k / 4); the
// factor i of the odd outputs is folded into scalar adds.
FDAS_DEV void dft4_inv(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = f2_add(a0, a2), t1 = f2_sub(a0, a2), t2 = f2_add(a1, a3),
               t3 = f2_sub(a1, a3);
  a0 = f2_add(t0, t2);
  a2 = f2_sub(t0, t2);
  a1 = make_float2(t1.x - t3.y, t1.y + t3.x);  // t1 + i t3
  a3 = make_float2(t1.x + t3.y, t1.y - t3.x);  // t1 - i t3
}

// Inverse 16-point DFT as 4 x 4 (4-point DFTs over n2 of x[n1 + 4 n2],
// twiddles exp(2 pi i n1 k1 / 16), 4-point DFTs over n1); output k sits in
// x[brev<16>(k)].
FDAS_DEV void dft16_inv(float2 (&x)[16]) {
  float2 y[16];  // y[n1 + 4 k1]
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 a0 = x[n1], a1 = x[n1 + 4], a2 = x[n1 + 8], a3 = x[n1 + 12];
    dft4_inv(a0, a1, a2, a3);
    y[n1] = a0;
    y[n1 + 4] = f2_tw16(a1, n1);
    y[n1 + 8] = f2_tw16(a2, 2 * n1);
    y[n1 + 12] = f2_tw16(a3, 3 * n1);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a0 = y[4 * k1], a1 = y[4 * k1 + 1], a2 = y[4 * k1 + 2], a3 = y[4 * k1 + 3];
    dft4_inv(a0, a1, a2, a3);
    x[brev<16>(k1)] = a0;
    x[brev<16>(k1 + 4)] = a1;
    x[brev<16>(k1 + 8)] = a2;
    x[brev<16>(k1 + 12)] = a3;
  }
}

// 8 consecutive columns of this thread's lane (one load, one wait).
FDAS_DEV void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <int IB>
__global__ void __launch_bounds__(kT16, 2)
    k_corr16(const float2* __restrict__ seg, const float2* __restrict__ bank,
             float* __restrict__ plane, float* __restrict__ q4, int64_t nb, int Z, int V, int m,
             int64_t n_pairs, const float2* __restrict__ twL, float thr1,
             fdas_cand* __restrict__ cands, unsigned long long* count, int64_t maxc) {
  constexpr int L = kL16;
  extern __shared__ float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);
  float* Ps = reinterpret_cast<float*>(X + L);
  float2* twA = reinterpret_cast<float2*>(Ps + kPs16);  // exp(+2 pi i a c / 256) at 16 a + c
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < 256; e += kT16)
    twA[e] = cconj(__ldg(twL + (((e >> 4) * (e & 15) * 32) & (L - 1))));
  if (warp == 0) {
    tmem_alloc(&s_tmem, kCols16);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  // this thread's lane (its warp's quarter) and its warp's 32-column groups:
  // segment points at 32 (warp / 4), A2 twiddles at 128 + 32 (warp / 4)
  const uint32_t tl = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t tF = tl + 32u * (uint32_t)(warp >> 2);
  const uint32_t tW = tl + 128u + 32u * (uint32_t)(warp >> 2);
  // A2 twiddles exp(+2 pi i k1 (c + 16 d) / L), k1 = lane, c = warp, d = 0..15
#pragma unroll
  for (int hd = 0; hd < 2; ++hd) {
    float f[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int d = 8 * hd + i;
      const float2 w = cconj(__ldg(twL + ((lane * (warp + 16 * d)) & (L - 1))));
      f[2 * i] = w.x;
      f[2 * i + 1] = w.y;
    }
    tmem_st16(tW + 16 * hd, f);
  }
  tmem_wait_st();

  const int half_m = m / 2;
  const int64_t nq = nb >> 2;
  const int64_t p0 = (int64_t)blockIdx.x * n_pairs / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * n_pairs / gridDim.x;
  const int cB = lane >> 1, hB = lane & 1;  // B role: n2 = cB + 16 warp, parity hB of k1
  int s_cur = -1;
  for (int64_t p = p0; p < p1; ++p) {
    const int s = (int)(p / Z);
    const int z = (int)(p - (int64_t)s * Z);
    if (s != s_cur) {  // this thread's points k1 + 32 a + 512 b of segment s -> TMEM
      const float2* fs = seg + (size_t)s * L + lane + 32 * warp;
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        float f[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 v = __ldg(fs + 512 * (8 * hb + i));
          f[2 * i] = v.x;
          f[2 * i + 1] = v.y;
        }
        tmem_st16(tF + 16 * hb, f);
      }
      tmem_wait_st();
      s_cur = s;
    }
    // ---- A1: Y[k] = F_s[k] T_z[k], DFT over b, twiddle, store
    float2 v[16];
    const float2* tz = bank + (size_t)z * L + lane + 32 * warp;
#pragma unroll
    for (int b = 0; b < 16; ++b) v[b] = __ldg(tz + 512 * b);
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
      float f[16];
      tmem_ld16(tF + 16 * hb, f);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[8 * hb + i] = f2_mul(v[8 * hb + i], make_float2(f[2 * i], f[2 * i + 1]));
    }
    dft16_inv(v);
#pragma unroll
    for (int c = 1; c < 16; ++c) v[brev<16>(c)] = f2_mul(v[brev<16>(c)], twA[16 * warp + c]);
#pragma unroll
    for (int c = 0; c < 16; ++c) X[xslot(warp, c, lane)] = v[brev<16>(c)];
    __syncthreads();
    // ---- A2: DFT over a, twiddle, back into the slots just read
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = X[xslot(a, warp, lane)];
    dft16_inv(v);
#pragma unroll
    for (int d0 = 0; d0 < 16; d0 += 4) {
      float f[8];
      tmem_ld8(tW + 2 * d0, f);
#pragma unroll
      for (int dd = 0; dd < 4; ++dd)
        X[xslot(d0 + dd, warp, lane)] =
            f2_mul(v[brev<16>(d0 + dd)], make_float2(f[2 * dd], f[2 * dd + 1]));
    }
    __syncthreads();
    // ---- B: DFT over j of Z[2 j + hB]
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = X[xslot(warp, cB, 2 * j + hB)];
    // every warp has read X: the next pair's A1 may overwrite it
    __syncthreads();
    dft16_inv(v);  // E[r] (hB = 0) or O[r] (hB = 1) in v[brev(r)]
    // lane hB = 0 keeps r = 0..7 and takes O[0..7]; hB = 1 keeps r = 8..15
    // and takes E[8..15]
    const int n2 = cB + 16 * warp;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 give = hB ? v[brev<16>(i)] : v[brev<16>(8 + i)];
      float2 got;
      got.x = __shfl_xor_sync(0xffffffffu, give.x, 1);
      got.y = __shfl_xor_sync(0xffffffffu, give.y, 1);
      const float2 E = hB ? got : v[brev<16>(i)];
      const float2 O = hB ? v[brev<16>(8 + i)] : got;
      // t = exp(2 pi i r / 32) O, r = i + 8 hB (the 8 adds a quarter turn)
      float2 t = O;
      if (i == 4) t = make_float2((O.x - O.y) * kCos32[4], (O.x + O.y) * kCos32[4]);
      else if (i != 0) t = f2_rot(O, kCos32[i], kSin32[i]);
      if (hB) t = make_float2(-t.y, t.x);
      const int r = i + 8 * hB;
      Ps[ps_idx(n2 + 256 * r)] = cnorm(f2_add(E, t));
      Ps[ps_idx(n2 + 256 * (r + 16))] = cnorm(f2_sub(E, t));
    }
    // the float4s of the output stage come from lanes of this warp only
    __syncwarp();
    // plane row slice, its 4-bin maxima and the h = 1 candidates: outputs
    // n in [m/2, m/2 + V) are bins r = s V + n - m/2 (r < nb); lane l stores
    // the float4s at n = 16 warp + 4 (l % 4) + 256 ((l / 4) + 8 i)
    const int64_t r0 = (int64_t)s * V;
    int64_t nvalid = nb - r0;
    if (nvalid > V) nvalid = V;
    const int nhi = half_m + (int)nvalid;
    // (half-bin planes, IB = 1: template row z = 2j + e fills columns 2r + e
    // of plane row j; rows 2j and 2j+1 are consecutive pairs, so each sector
    // is completed in L2 before it is written back)
    float* prow = plane ? plane + (size_t)(z >> IB) * (nb << IB) + (r0 << IB) + (z & IB) : nullptr;
    float* qrow = q4 ? q4 + (size_t)z * nq + (r0 >> 2) : nullptr;
    const int nw = 16 * warp + 4 * (lane & 3);
    bool hit = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = nw + 256 * ((lane >> 2) + 8 * i);
      if (n >= half_m && n < nhi) {
        const float4 p4 = *reinterpret_cast<const float4*>(Ps + ps_idx(n));
        const int k = (n - half_m) >> 2;  // float4 index in the row slice
        const float mx = fmaxf(fmaxf(p4.x, p4.y), fmaxf(p4.z, p4.w));
        if (prow) {
          if constexpr (IB) {
            prow[8 * k] = p4.x;
            prow[8 * k + 2] = p4.y;
            prow[8 * k + 4] = p4.z;
            prow[8 * k + 6] = p4.w;
          } else {
            reinterpret_cast<float4*>(prow)[k] = p4;
          }
        }
        if (qrow) qrow[k] = mx;
        hit |= mx >= thr1;
      }
    }
    if (cands && __any_sync(0xffffffffu, hit)) {
      // rare: some power this warp stored reached T_1; the warp scans its
      // own float4s again and appends
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        const int n = nw + 256 * ((lane >> 2) + 8 * i);
        const bool in = n >= half_m && n < nhi;
        const float4 p4 =
            in ? *reinterpret_cast<const float4*>(Ps + ps_idx(n)) : make_float4(0.f, 0.f, 0.f, 0.f);
        const int rk = (int)(r0 + (n - half_m));
        emit(in && rk >= 1 && p4.x >= thr1, rk, z, 1, p4.x, cands, count, maxc);
        emit(in && p4.y >= thr1, rk + 1, z, 1, p4.y, cands, count, maxc);
        emit(in && p4.z >= thr1, rk + 2, z, 1, p4.z, cands, count, maxc);
        emit(in && p4.w >= thr1, rk + 3, z, 1, p4.w, cands, count, maxc);
      }
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(s_tmem, kCols16);
}

// Steps 3 + 4: segment s (zero-filled at the spectrum edges), forward FFT in
// shared memory, stored in natural order.
__global__ void __launch_bounds__(256) k_segments16(const float2* __restrict__ Xw,
                                                    float2* __restrict__ seg, int64_t nb, int V,
                                                    int m, const float2* __restrict__ tw) {
  extern __shared__ float2 sbuf[];
  const int tid = threadIdx.x;
  const int s = blockIdx.x;
  const int64_t base = (int64_t)s * V - m / 2;
  for (int i = tid; i < kL16; i += 256) {
    const int64_t g = base + i;
    sbuf[i] = (g >= 0 && g < nb) ? Xw[g] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  block_fft<kL16, kFwd, 256, 1>(sbuf, tw, tid);
  float2* out = seg + (size_t)s * kL16;
  for (int i = tid; i < kL16; i += 256) out[i] = sbuf[i];
}

template <int IB>
int corr16_launch(fdas_plan* p, float* plane, float* q4, fdas_cand* cands,
                  unsigned long long* count) {
  int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e != cudaSuccess) return cuda_check(e, "device attributes");
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_corr16<IB>);
  if (e != cudaSuccess) return cuda_check(e, "k_corr16 attributes");
  // Half the SM's shared memory per CTA (less the 1 KB per-CTA reserve and
  // the static part): at most two CTAs, 2 x 256 tensor-memory columns, share
  // an SM, and with any other kernel here that holds tensor memory the
  // shares of columns never exceed the shares of shared memory, so
  // tcgen05.alloc never waits.
  size_t smem = kSmem16;
  const size_t half = ((size_t)smem_sm / 2 - 1024 - fa.sharedSizeBytes) & ~(size_t)15;
  if (smem < half) smem = half;
  e = cudaFuncSetAttribute(k_corr16<IB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "k_corr16 attr");
  e = cudaFuncSetAttribute(k_corr16<IB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return cuda_check(e, "k_corr16 carveout");
  int occ = regs_sm / (((fa.numRegs + 7) / 8) * 8 * kT16);
  const int by_smem = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
  if (by_smem < occ) occ = by_smem;
  if (occ > 2) occ = 2;
  if (occ < 1) return set_error(FDAS_ERR_CUDA, "k_corr16 cannot be resident");
  p->corr_ctas_per_sm = occ;
  const int zrows = p->Z << IB;
  const int64_t n_pairs = (int64_t)p->S * zrows;
  int64_t grid = (int64_t)occ * sms;
  if (grid > n_pairs) grid = n_pairs;
  p->corr_grid = (int)grid;
  k_corr16<IB><<<(unsigned)grid, kT16, smem, p->stream>>>(
      p->seg, IB ? p->bank_ib : p->bank, plane, IB ? nullptr : q4, p->nb, zrows, p->V, p->m,
      n_pairs, p->tw_L, p->thr[0], IB ? nullptr : cands, count, p->max_cands);
  return cuda_check(cudaGetLastError(), "k_corr16");
}

}  // namespace

int launch_segments16(fdas_plan* p, const float2* d_white) {
  const size_t smem = sizeof(float2) * kL16;
  cudaError_t e = cudaFuncSetAttribute(k_segments16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "k_segments16 attr");
  k_segments16<<<p->S, 256, smem, p->stream>>>(d_white, p->seg, p->nb, p->V, p->m, p->tw_L);
  return cuda_check(cudaGetLastError(), "k_segments16");
}

int launch_correlate16(fdas_plan* p, float* d_plane, float* d_q4, fdas_cand* d_cands,
                       unsigned long long* d_count) {
  return p->interbin ? corr16_launch<1>(p, d_plane, d_q4, d_cands, d_count)
                     : corr16_launch<0>(p, d_plane, d_q4, d_cands, d_count);
}

}  // namespace fdas
