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
// A CTA takes 64 consecutive bins: the union of their windows (<= 127
// powers) is sorted once in shared memory as 32-bit keys - the power's bit
// pattern (powers are >= 0, so bit patterns order like values) with its low
// 7 mantissa bits replaced by the entry's index - and the medians read the
// exact powers back by index. (Two powers within 2^-16 of each other may
// swap places in that order, which moves a median by less than 2^-16
// relative.) For each run of 32 sorted entries a 128-bit mask records which
// indices it holds; a warp skips the runs below its lanes' 32nd in-window
// entries by popcount and then walks the sorted list in step, every lane
// reading the same entry.
// ----------------------------------------------------------------------------
constexpr int kWin = 64;
constexpr int kWTile = 64;
constexpr int kSortN = 128;

__device__ __forceinline__ int64_t wstart(int64_t k, int64_t nb) {
  int64_t s = k - kWin / 2;
  s = s < 1 ? 1 : s;
  return s > nb - kWin ? nb - kWin : s;
}

__global__ void __launch_bounds__(kWTile) k_whiten(const float2* __restrict__ X,
                                                   float2* __restrict__ Xw, int64_t nb) {
  __shared__ unsigned skey[kSortN];
  __shared__ float spow[kSortN];
  __shared__ unsigned long long cmask[kSortN / 32][2];
  const int tid = threadIdx.x;
  if (tid < kSortN / 16) cmask[tid >> 1][tid & 1] = 0ull;
  const int64_t k0 = (int64_t)blockIdx.x * kWTile;
  const int64_t klast = (k0 + kWTile - 1 < nb - 1) ? k0 + kWTile - 1 : nb - 1;
  const int64_t lo = wstart(k0 < 1 ? 1 : k0, nb);
  const int64_t hi = wstart(klast, nb) + kWin - 1;
  const int cnt = (int)(hi - lo + 1);
  for (int t = tid; t < kSortN; t += kWTile) {
    unsigned key = ~0u;
    if (t < cnt) {
      const float pw = cnorm(X[lo + t]);
      spow[t] = pw;
      key = (__float_as_uint(pw) & ~0x7Fu) | (unsigned)t;
    }
    skey[t] = key;
  }
  __syncthreads();
  // bitonic sort, ascending, one compare-exchange per thread per step
  for (int size = 2; size <= kSortN; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int a = 2 * stride * (tid / stride) + (tid % stride);
      const int b = a + stride;
      const bool up = (a & size) == 0;
      const unsigned ka = skey[a], kb = skey[b];
      if ((ka > kb) == up) {
        skey[a] = kb;
        skey[b] = ka;
      }
      __syncthreads();
    }
  }
  for (int t = tid; t < cnt; t += kWTile) {
    const unsigned i = skey[t] & 0x7Fu;
    atomicOr(&cmask[t >> 5][i >> 6], 1ull << (i & 63));
  }
  __syncthreads();
  const int64_t k = k0 + tid;
  const bool live = k < nb;
  const unsigned s = live ? (unsigned)(wstart(k, nb) - lo) : 0u;  // s <= 63
  // window bits [s, s + 63] of the 128 relative indices
  const unsigned long long w0 = ~0ull << s, w1 = s ? (1ull << s) - 1ull : 0ull;
  int c = 0, t0 = 0;
  for (; t0 + 32 <= cnt; t0 += 32) {
    const int n = __popcll(cmask[t0 >> 5][0] & w0) + __popcll(cmask[t0 >> 5][1] & w1);
    if (c + n >= kWin / 2) break;  // the 32nd in-window entry is in this run
    c += n;
  }
  // walk in step from the warp's lowest start; lanes before their own start
  // skip entries they have already counted
  const int tw = __reduce_min_sync(0xffffffffu, t0);
  int ia = -1, ib = -1;
  bool done = !live;
  for (int t = tw; t < cnt && !__all_sync(0xffffffffu, done); ++t) {
    const unsigned key = skey[t];
    const unsigned i = key & 0x7Fu;
    if (!done && t >= t0 && i - s < (unsigned)kWin) {
      if (c == kWin / 2 - 1) ia = (int)i;
      if (c == kWin / 2) {
        ib = (int)i;
        done = true;
      }
      ++c;
    }
  }
  if (!live) return;
  if (k == 0) {
    Xw[0] = make_float2(0.f, 0.f);
    return;
  }
  const float mu = 0.5f * (spow[ia] + spow[ib]);
  const float2 x = X[k];
  const float g = mu > 0.f ? sqrtf(0.69314718055994531f / mu) : 0.f;
  Xw[k] = make_float2(x.x * g, x.y * g);
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
  const unsigned nblk = (unsigned)((p->nb + kWTile - 1) / kWTile);
  k_whiten<<<nblk, kWTile, 0, p->stream>>>(d_spec, d_white, p->nb);
  return cuda_check(cudaGetLastError(), "k_whiten");
}

}  // namespace fdas
