// Shared device building blocks of the FDAS CUDA path: complex helpers,
// in-register radix-R DFTs and a shared-memory Stockham FFT.
//
// All FFTs here compute y_k = sum_j x_j exp(DIR * 2 pi i j k / R) with
// DIR = -1 (forward) or +1 (inverse, unnormalised). Twiddle tables are
// generated in float64 and rounded once to float32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define FDAS_DEV __device__ __forceinline__

namespace fdas {

constexpr int kFwd = -1;
constexpr int kInv = +1;

FDAS_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
FDAS_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
FDAS_DEV float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
FDAS_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
FDAS_DEV float cnorm(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// cos(2 pi k / 32), sin(2 pi k / 32) for k = 0..15 (k = 0 and 8 are never
// read: those rotations are exact swaps).
__device__ constexpr float kCos32[16] = {
    1.0f, 9.80785280403230431e-01f, 9.23879532511286738e-01f, 8.31469612302545236e-01f,
    7.07106781186547573e-01f, 5.55570233019602289e-01f, 3.82683432365089837e-01f,
    1.95090322016128331e-01f, 0.0f, -1.95090322016128193e-01f, -3.82683432365089726e-01f,
    -5.55570233019601956e-01f, -7.07106781186547462e-01f, -8.31469612302545347e-01f,
    -9.23879532511286738e-01f, -9.80785280403230431e-01f};
__device__ constexpr float kSin32[16] = {
    0.0f, 1.95090322016128248e-01f, 3.82683432365089782e-01f, 5.55570233019602178e-01f,
    7.07106781186547462e-01f, 8.31469612302545236e-01f, 9.23879532511286738e-01f,
    9.80785280403230431e-01f, 1.0f, 9.80785280403230431e-01f, 9.23879532511286738e-01f,
    8.31469612302545458e-01f, 7.07106781186547573e-01f, 5.55570233019602178e-01f,
    3.82683432365089893e-01f, 1.95090322016128609e-01f};

// v * exp(DIR * 2 pi i e / R) for 0 <= e < R/2, R | 32. After full unrolling
// e and R are constants, so the branches fold away.
template <int DIR>
FDAS_DEV float2 rot(float2 v, int e, int R) {
  const int k = e * (32 / R);
  if (k == 0) return v;
  if (k == 8) return DIR < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  const float c = kCos32[k];
  const float s = DIR < 0 ? -kSin32[k] : kSin32[k];
  return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

template <int R>
__host__ __device__ constexpr int brev(int k) {
  int r = 0;
  for (int b = 0; b < ilog2(R); ++b) r |= ((k >> b) & 1) << (ilog2(R) - 1 - b);
  return r;
}

// In-register radix-R DFT (R = 2..32, power of two), radix-2 decimation in
// frequency; on return output k sits in x[brev<R>(k)].
template <int R, int DIR>
FDAS_DEV void dft_brev(float2 (&x)[R]) {
#pragma unroll
  for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 a = x[blk + j];
        const float2 b = x[blk + j + half];
        x[blk + j] = cadd(a, b);
        x[blk + j + half] = rot<DIR>(csub(a, b), j, 2 * half);
      }
    }
  }
}

// Same, with outputs put back in natural order (register renaming only).
template <int R, int DIR>
FDAS_DEV void dft(float2 (&x)[R]) {
  dft_brev<R, DIR>(x);
  float2 y[R];
#pragma unroll
  for (int k = 0; k < R; ++k) y[k] = x[brev<R>(k)];
#pragma unroll
  for (int k = 0; k < R; ++k) x[k] = y[k];
}

// Radix used by stage s of a length-L Stockham FFT: 16 while at least 16
// remains, then the leftover factor (2, 4 or 8).
__host__ __device__ constexpr int stage_radix(int L, int ns) {
  return (L / ns) >= 16 ? 16 : (L / ns);
}

// One Stockham radix-R stage on NB transforms of length L stored back to
// back in shared memory (buf[b * L + i]); in place, with a barrier between
// the loads and the stores. tw[e] = exp(-2 pi i e / L) (float64-made).
template <int L, int R, int NS, int DIR, int NT, int NB>
FDAS_DEV void stockham_stage(float2* buf, const float2* __restrict__ tw, int tid) {
  constexpr int NBF = L / R;                 // butterflies per transform
  constexpr int TOT = NBF * NB;
  constexpr int PER = (TOT + NT - 1) / NT;
  float2 v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int g = tid + p * NT;
    if (g < TOT) {
      const int b = g / NBF;
      const int j = g - b * NBF;
      const int jm = j & (NS - 1);
      const float2* src = buf + b * L + j;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 val = src[r * NBF];
        if (NS > 1 && r > 0) {
          float2 w = __ldg(tw + jm * r * (L / (NS * R)));
          if (DIR > 0) w.y = -w.y;
          val = cmul(val, w);
        }
        v[p][r] = val;
      }
      dft_brev<R, DIR>(v[p]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int g = tid + p * NT;
    if (g < TOT) {
      const int b = g / NBF;
      const int j = g - b * NBF;
      const int jm = j & (NS - 1);
      float2* dst = buf + b * L + (j / NS) * NS * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * NS] = v[p][brev<R>(r)];
    }
  }
  __syncthreads();
}

template <int L, int NS, int DIR, int NT, int NB>
FDAS_DEV void stockham_from(float2* buf, const float2* __restrict__ tw, int tid) {
  if constexpr (NS < L) {
    constexpr int R = stage_radix(L, NS);
    stockham_stage<L, R, NS, DIR, NT, NB>(buf, tw, tid);
    stockham_from<L, NS * R, DIR, NT, NB>(buf, tw, tid);
  }
}

// Full length-L FFT (natural order in and out) of NB transforms in shared
// memory, executed by NT threads. The caller synchronises before the call.
template <int L, int DIR, int NT, int NB>
FDAS_DEV void block_fft(float2* buf, const float2* __restrict__ tw, int tid) {
  stockham_from<L, 1, DIR, NT, NB>(buf, tw, tid);
}

}  // namespace fdas
