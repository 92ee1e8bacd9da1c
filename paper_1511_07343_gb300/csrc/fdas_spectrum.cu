// Step 2 of Section 4 (real-to-complex DFT of the series) and the running-
// median spectral whitening that precedes the correlation.
//
// Real FFT: the N real samples are read as M = N/2 complex points
// z_n = x_{2n} + i x_{2n+1} (a free reinterpretation of the float array),
// transformed by a four-step FFT M = M1 * M2 (columns, twiddle, rows), and
// unpacked with X_k = (Z_k + conj Z_{M-k})/2 - (i/2) w^k (Z_k - conj Z_{M-k}),
// w = exp(-2 pi i / N). The whole M-point working set (32 MiB at N = 2^23)
// stays in L2 between the passes.
#include <float.h>

#include "fdas_common.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr int kNT = 256;

// Batches of NB column transforms: for n1 in [b0, b0+NB) the length-LEN DFT
// over n2 of z[n1 + M1 n2], times exp(-2 pi i n1 k2 / M), stored transposed
// as T[k2 * M1 + n1].
template <int LEN, int NB>
__global__ void __launch_bounds__(kNT) k_fft_cols(const float2* __restrict__ z,
                                                  float2* __restrict__ T, int M1,
                                                  const float2* __restrict__ tw_len,
                                                  const float2* __restrict__ tw_lo,
                                                  const float2* __restrict__ tw_hi, int h4) {
  extern __shared__ float2 buf[];  // NB * LEN
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * NB;
  for (int i = tid; i < NB * LEN; i += kNT) {
    const int b = i % NB, e = i / NB;
    buf[b * LEN + e] = z[(size_t)(b0 + b) + (size_t)M1 * e];
  }
  __syncthreads();
  block_fft<LEN, kFwd, kNT, NB>(buf, tw_len, tid);
  const int mask = (1 << h4) - 1;
  for (int i = tid; i < NB * LEN; i += kNT) {
    const int b = i % NB, k2 = i / NB;
    const int n1 = b0 + b;
    const int e = n1 * k2;
    const float2 w = cmul(__ldg(tw_lo + (e & mask)), __ldg(tw_hi + (e >> h4)));
    T[(size_t)k2 * M1 + n1] = cmul(buf[b * LEN + k2], w);
  }
}

// Batches of NB row transforms: for k2 in [b0, b0+NB) the length-LEN DFT over
// n1 of T[k2 * LEN + n1], stored as Z[k2 + M2 k1].
template <int LEN, int NB>
__global__ void __launch_bounds__(kNT) k_fft_rows(const float2* __restrict__ T,
                                                  float2* __restrict__ Zo, int M2,
                                                  const float2* __restrict__ tw_len) {
  extern __shared__ float2 buf[];  // NB * LEN
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * NB;
  for (int i = tid; i < NB * LEN; i += kNT) {
    const int b = i / LEN, e = i % LEN;
    buf[b * LEN + e] = T[(size_t)(b0 + b) * LEN + e];
  }
  __syncthreads();
  block_fft<LEN, kFwd, kNT, NB>(buf, tw_len, tid);
  for (int i = tid; i < NB * LEN; i += kNT) {
    const int b = i % NB, k1 = i / NB;
    Zo[(size_t)(b0 + b) + (size_t)M2 * k1] = buf[b * LEN + k1];
  }
}

// Unpack the packed complex FFT into the first M bins of the real FFT.
__global__ void k_unpack(const float2* __restrict__ Zf, float2* __restrict__ X, int64_t M,
                         const float2* __restrict__ tw_lo, const float2* __restrict__ tw_hi,
                         int hN) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const float2 a = Zf[k];
  const float2 b = cconj(Zf[k == 0 ? 0 : M - k]);
  const float2 ev = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
  const float2 od = make_float2(0.5f * (a.x - b.x), 0.5f * (a.y - b.y));
  const int mask = (1 << hN) - 1;
  const float2 w = cmul(__ldg(tw_lo + (k & mask)), __ldg(tw_hi + (k >> hN)));
  // -(i) * w * od
  const float2 t = cmul(w, od);
  X[k] = make_float2(ev.x + t.y, ev.y - t.x);
}

template <int LEN>
int launch_cols(fdas_plan* p, const float2* z, float2* T) {
  // NB columns per CTA: NB consecutive float2 of a row make one 32-byte
  // sector from NB = 4 on
  constexpr int NB = LEN >= 4096 ? 2 : 4;
  constexpr int smem = NB * LEN * (int)sizeof(float2);
  if (smem > 48 * 1024) {
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && attr_dev != dev) {
      e = cudaFuncSetAttribute(k_fft_cols<LEN, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem);
      if (e == cudaSuccess) attr_dev = dev;
    }
    if (e != cudaSuccess) return cuda_check(e, "k_fft_cols attr");
  }
  k_fft_cols<LEN, NB><<<p->M1 / NB, kNT, smem, p->stream>>>(z, T, p->M1, p->tw_M2, p->tw4_lo,
                                                              p->tw4_hi, p->h4);
  return cuda_check(cudaGetLastError(), "k_fft_cols");
}

template <int LEN>
int launch_rows(fdas_plan* p, const float2* T, float2* Zo) {
  // NB rows per CTA: the transposed stores write NB consecutive float2
  constexpr int NB = LEN >= 4096 ? 2 : 4;
  constexpr int smem = NB * LEN * (int)sizeof(float2);
  if (smem > 48 * 1024) {
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && attr_dev != dev) {
      e = cudaFuncSetAttribute(k_fft_rows<LEN, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem);
      if (e == cudaSuccess) attr_dev = dev;
    }
    if (e != cudaSuccess) return cuda_check(e, "k_fft_rows attr");
  }
  k_fft_rows<LEN, NB><<<p->M2 / NB, kNT, smem, p->stream>>>(T, Zo, p->M2, p->tw_M1);
  return cuda_check(cudaGetLastError(), "k_fft_rows");
}

int dispatch_cols(fdas_plan* p, const float2* z, float2* T) {
  switch (p->M2) {
    case 32: return launch_cols<32>(p, z, T);
    case 64: return launch_cols<64>(p, z, T);
    case 128: return launch_cols<128>(p, z, T);
    case 256: return launch_cols<256>(p, z, T);
    case 512: return launch_cols<512>(p, z, T);
    case 1024: return launch_cols<1024>(p, z, T);
    case 2048: return launch_cols<2048>(p, z, T);
    case 4096: return launch_cols<4096>(p, z, T);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported column FFT length");
}

int dispatch_rows(fdas_plan* p, const float2* T, float2* Zo) {
  switch (p->M1) {
    case 32: return launch_rows<32>(p, T, Zo);
    case 64: return launch_rows<64>(p, T, Zo);
    case 128: return launch_rows<128>(p, T, Zo);
    case 256: return launch_rows<256>(p, T, Zo);
    case 512: return launch_rows<512>(p, T, Zo);
    case 1024: return launch_rows<1024>(p, T, Zo);
    case 2048: return launch_rows<2048>(p, T, Zo);
    case 4096: return launch_rows<4096>(p, T, Zo);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported row FFT length");
}

// ----------------------------------------------------------------------------
// Whitening: mu_k = even-count median of |X|^2 over the 64-bin window of bin
// k ([k-32, k+31] shifted into [1, nb-1]); Xw_k = X_k sqrt(ln2 / mu_k).
// One warp takes 64 consecutive bins (a tile); no CTA barrier is used.
//  1. The union of the tile's windows (at most 127 bins from u0) is loaded
//     as 128 keys, the power's bit pattern (powers are >= 0, so the patterns
//     order like the values; entries past the spectrum get the largest key),
//     each carrying its entry index, and sorted by a bitonic network in
//     registers: slot i = 4 lane + w, compare-exchanges at distance 1 and 2
//     inside a lane, at distance >= 4 through shuffles. Ties need no order:
//     equal powers are equal order statistics, and a compare-exchange moves
//     or keeps both of its entries, so the slots stay a permutation.
//  2. pos[e] = sorted slot of entry e. The window of offset o (entries
//     o .. o+63) is the 128-bit mask M(o) of the slots its entries hold:
//     M(0) is an XOR reduction of the bits of entries 0..63 over the warp,
//     and M(o) = M(0) ^ XOR_{i<o} (bit(pos[i]) ^ bit(pos[i+64])), an
//     exclusive XOR scan over the lanes; lane l gets M(2l) and M(2l+1).
//  3. Bin k = k0 + 2l + c has offset wstart(k) - u0 (= 2l + c unless a
//     window of the tile is shifted at a spectrum edge; then its mask comes
//     from the lane holding it); its median is
//     the mean of the sorted powers at the 32nd and 33rd set bits of its mask.
// ----------------------------------------------------------------------------
constexpr int kWin = 64;
constexpr int kWTile = 64;       // bins per warp
constexpr int kSortN = 128;      // sorted entries per warp
constexpr int kWWarps = 8;       // warps (tiles) per CTA

__device__ __forceinline__ int64_t wstart(int64_t k, int64_t nb) {
  int64_t s = k - kWin / 2;
  s = s < 1 ? 1 : s;
  return s > nb - kWin ? nb - kWin : s;
}

struct Bits128 {
  unsigned long long lo, hi;
};
FDAS_DEV Bits128 bit128(unsigned p) {
  const unsigned long long b = 1ull << (p & 63u);
  return Bits128{p < 64 ? b : 0ull, p < 64 ? 0ull : b};
}
FDAS_DEV Bits128 operator^(Bits128 a, Bits128 b) { return Bits128{a.lo ^ b.lo, a.hi ^ b.hi}; }
FDAS_DEV Bits128 shfl128(Bits128 a, int src) {
  return Bits128{__shfl_sync(0xffffffffu, a.lo, src), __shfl_sync(0xffffffffu, a.hi, src)};
}

// position of the set bit of rank r (0-based) of m (m has more than r set bits)
FDAS_DEV int select128(Bits128 m, int r) {
  const int c = __popcll(m.lo);
  const unsigned long long x = r < c ? m.lo : m.hi;
  int base = r < c ? 0 : 64;
  r = r < c ? r : r - c;
  unsigned w = (unsigned)x;
  const int c32 = __popc(w);
  if (r >= c32) {
    w = (unsigned)(x >> 32);
    base += 32;
    r -= c32;
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) {
    const int cs = __popc(w & ((1u << sh) - 1u));
    if (r >= cs) {
      r -= cs;
      w >>= sh;
      base += sh;
    }
  }
  return base;
}

__global__ void __launch_bounds__(32 * kWWarps) k_whiten(const float2* __restrict__ X,
                                                         float2* __restrict__ Xw, int64_t nb) {
  __shared__ __align__(16) float sval[kWWarps][kSortN];
  __shared__ __align__(4) unsigned char spos[kWWarps][kSortN];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = ((int64_t)blockIdx.x * kWWarps + warp) * kWTile;
  if (k0 >= nb) return;  // the whole warp
  const int64_t u0 = wstart(k0 < 1 ? 1 : k0, nb);
  // 1. keys; slot 4 lane + w starts with entry lane + 32 w (coalesced loads)
  unsigned kh[4], kl[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int e = lane + 32 * w;
    const int64_t b = u0 + e;
    kh[w] = b < nb ? __float_as_uint(cnorm(X[b])) : 0xffffffffu;
    kl[w] = (unsigned)e;
  }
#pragma unroll
  for (int size = 2; size <= kSortN; size <<= 1) {
#pragma unroll
    for (int d = size >> 1; d >= 1; d >>= 1) {
      if (d >= 4) {
        const int ld = d >> 2;
        // slots 4 lane + w, w < 4: the bits tested here (>= 4) are lane bits
        const bool asc = ((4 * lane) & size) == 0;
        const bool keep_min = ((lane & ld) == 0) == asc;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const unsigned oh = __shfl_xor_sync(0xffffffffu, kh[w], ld);
          const unsigned ol = __shfl_xor_sync(0xffffffffu, kl[w], ld);
          // strict on both sides: equal powers stay where they are, so every
          // entry keeps exactly one slot
          const bool lt = oh < kh[w], gt = kh[w] < oh;
          if ((lt && keep_min) || (gt && !keep_min)) {
            kh[w] = oh;
            kl[w] = ol;
          }
        }
      } else {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          if (w & d) continue;
          const int v = w | d;
          const bool asc = ((4 * lane + w) & size) == 0;
          const bool gt = kh[w] > kh[v];
          if (gt == asc) {
            const unsigned th = kh[w], tl = kl[w];
            kh[w] = kh[v];
            kl[w] = kl[v];
            kh[v] = th;
            kl[v] = tl;
          }
        }
      }
    }
  }
  // 2. sorted powers by slot, slot of each entry
  float* sv = sval[warp];
  unsigned char* sp = spos[warp];
  reinterpret_cast<float4*>(sv)[lane] = make_float4(__uint_as_float(kh[0]), __uint_as_float(kh[1]),
                                                    __uint_as_float(kh[2]), __uint_as_float(kh[3]));
#pragma unroll
  for (int w = 0; w < 4; ++w) sp[kl[w]] = (unsigned char)(4 * lane + w);
  __syncwarp();
  const unsigned short q01 = reinterpret_cast<const unsigned short*>(sp)[lane];
  const unsigned short q23 = reinterpret_cast<const unsigned short*>(sp)[lane + 32];
  const Bits128 b0 = bit128(q01 & 0xffu), b1 = bit128(q01 >> 8);    // entries 2l, 2l+1
  const Bits128 b2 = bit128(q23 & 0xffu), b3 = bit128(q23 >> 8);    // entries 2l+64, 2l+65
  Bits128 m0 = b0 ^ b1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    m0.lo ^= __shfl_xor_sync(0xffffffffu, m0.lo, o);
    m0.hi ^= __shfl_xor_sync(0xffffffffu, m0.hi, o);
  }
  const Bits128 D0 = b0 ^ b2, dl = D0 ^ (b1 ^ b3);
  Bits128 inc = dl;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long tlo = __shfl_up_sync(0xffffffffu, inc.lo, o);
    const unsigned long long thi = __shfl_up_sync(0xffffffffu, inc.hi, o);
    if (lane >= o) {
      inc.lo ^= tlo;
      inc.hi ^= thi;
    }
  }
  Bits128 m[2];
  m[0] = m0 ^ (inc ^ dl);  // M(2l)
  m[1] = m[0] ^ D0;        // M(2l+1)
  // 3. medians and whitened output of bins k0 + 2l, k0 + 2l + 1
  const int64_t k = k0 + 2 * lane;
  // a tile with a window shifted at either spectrum edge: offsets differ
  if (k0 < 1 + kWin / 2 || k0 + (kWTile - 1) - kWin / 2 > nb - kWin) {
    Bits128 mo[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int off = k + c < nb ? (int)(wstart(k + c, nb) - u0) : 0;  // 0..63
      const Bits128 a = shfl128(m[0], off >> 1), bb = shfl128(m[1], off >> 1);
      mo[c] = (off & 1) ? bb : a;
    }
    m[0] = mo[0];
    m[1] = mo[1];
  }
  if (k >= nb) return;  // nb is even: bins k, k + 1 are both in or both out
  float g[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const float mu = 0.5f * (sv[select128(m[c], kWin / 2 - 1)] + sv[select128(m[c], kWin / 2)]);
    g[c] = mu > 0.f ? sqrtf(0.69314718055994531f / mu) : 0.f;
  }
  if (k == 0) g[0] = 0.f;
  const float4 x = *reinterpret_cast<const float4*>(X + k);
  *reinterpret_cast<float4*>(Xw + k) = make_float4(x.x * g[0], x.y * g[0], x.z * g[1], x.w * g[1]);
}

}  // namespace

int launch_unpack(fdas_plan* p, float2* d_spec) {
  const int nt = 256;
  k_unpack<<<(unsigned)((p->M + nt - 1) / nt), nt, 0, p->stream>>>(p->spec2, d_spec, p->M,
                                                                     p->twN_lo, p->twN_hi, p->hN);
  return cuda_check(cudaGetLastError(), "k_unpack");
}

static bool pow2_in(int x, int lo, int hi) { return x >= lo && x <= hi && (x & (x - 1)) == 0; }

int launch_spectrum(fdas_plan* p, const float* d_series, float2* d_spec) {
  if (!pow2_in(p->M1, 32, 4096) || !pow2_in(p->M2, 32, 4096))
    return launch_spectrum_mixed(p, d_series, d_spec);
  const float2* z = reinterpret_cast<const float2*>(d_series);
  int rc = dispatch_cols(p, z, p->zbuf);
  if (rc) return rc;
  // the unpack reads bins k and M-k, so the packed FFT gets its own buffer
  rc = dispatch_rows(p, p->zbuf, p->spec2);
  if (rc) return rc;
  return launch_unpack(p, d_spec);
}

int launch_whiten(fdas_plan* p, const float2* d_spec, float2* d_white) {
  if (p->whiten_mode == FDAS_WHITEN_BLOCK) return launch_whiten_block(p, d_spec, d_white);
  const int64_t per_cta = (int64_t)kWTile * kWWarps;
  const unsigned nblk = (unsigned)((p->nb + per_cta - 1) / per_cta);
  k_whiten<<<nblk, 32 * kWWarps, 0, p->stream>>>(d_spec, d_white, p->nb);
  return cuda_check(cudaGetLastError(), "k_whiten");
}

}  // namespace fdas
