// Shared device building blocks of the FDAS CUDA path: complex helpers,
// in-register radix-R DFTs (scalar and packed-pair) and a shared-memory
// Stockham FFT.
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

// Radix used by the stage of a length-L Stockham FFT that starts at span ns:
// 16 while more than 32 points remain, then a single radix-32 stage if
// exactly 32 remain, else the leftover factor (2, 4, 8 or 16).
__host__ __device__ constexpr int stage_radix(int L, int ns) {
  return (L / ns) == 32 ? 32 : (L / ns) >= 16 ? 16 : (L / ns);
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

// ---------------------------------------------------------------------------
// Paired complex arithmetic on packed f32x2 (sm_100 family): a c2 holds two
// independent complex values, (re0, re1) and (im0, im1), so one packed
// instruction advances two transforms at once.
// ---------------------------------------------------------------------------
namespace fdas {

struct c2 {
  float2 re, im;
};

FDAS_DEV float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
FDAS_DEV float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
FDAS_DEV float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
FDAS_DEV float2 p_sub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
FDAS_DEV float2 p_neg(float2 a) { return p_mul(a, make_float2(-1.f, -1.f)); }

FDAS_DEV c2 c2_add(c2 a, c2 b) { return c2{p_add(a.re, b.re), p_add(a.im, b.im)}; }
FDAS_DEV c2 c2_sub(c2 a, c2 b) { return c2{p_sub(a.re, b.re), p_sub(a.im, b.im)}; }
// a * b, both data
FDAS_DEV c2 c2_mul(c2 a, c2 b) {
  return c2{p_sub(p_mul(a.re, b.re), p_mul(a.im, b.im)), p_fma(a.re, b.im, p_mul(a.im, b.re))};
}
// a * (C + i S) with per-lane cosines C and sines S
FDAS_DEV c2 c2_mul_cs(c2 a, float2 C, float2 S) {
  return c2{p_sub(p_mul(a.re, C), p_mul(a.im, S)), p_fma(a.re, S, p_mul(a.im, C))};
}

// exp(DIR 2 pi i e / R) applied lane-wise, lane 0 exponent e0, lane 1 e1
// (compile-time after unrolling, 0 <= e < R, R | 32).
template <int DIR>
FDAS_DEV c2 c2_rot(c2 v, int e0, int e1, int R) {
  const int k0 = e0 * (32 / R), k1 = e1 * (32 / R);
  if (k0 == 0 && k1 == 0) return v;
  if (k0 == 8 && k1 == 8)  // times DIR * i
    return DIR < 0 ? c2{v.im, p_neg(v.re)} : c2{p_neg(v.im), v.re};
  auto cs = [](int k, float& c, float& s) {
    // cos, sin of 2 pi k / 32 for 0 <= k < 32
    const int kk = k & 15;
    c = kCos32[kk];
    s = kSin32[kk];
    if (k >= 16) {
      c = -c;
      s = -s;
    }
  };
  float c0, s0, c1, s1;
  cs(k0, c0, s0);
  cs(k1, c1, s1);
  if (DIR < 0) {
    s0 = -s0;
    s1 = -s1;
  }
  return c2_mul_cs(v, make_float2(c0, c1), make_float2(s0, s1));
}

// In-register radix-R DFT of two independent lanes (radix-2 decimation in
// frequency); output k sits in x[brev<R>(k)].
template <int R, int DIR>
FDAS_DEV void dft2_brev(c2 (&x)[R]) {
#pragma unroll
  for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const c2 a = x[blk + j];
        const c2 b = x[blk + j + half];
        x[blk + j] = c2_add(a, b);
        x[blk + j + half] = c2_rot<DIR>(c2_sub(a, b), j, j, 2 * half);
      }
    }
  }
}

// v * exp(DIR 2 pi i e / 16) for 0 <= e < 16 (e a constant after
// unrolling): quarter turns are swaps, eighth turns (|cos| = |sin|) take two
// adds and two multiplies, the rest two multiplies and two fused
// multiply-adds with the sine's negative as a constant.
template <int DIR>
FDAS_DEV c2 c2_tw16(c2 v, int e) {
  e &= 15;
  if (e == 0) return v;
  if (e == 4) return DIR > 0 ? c2{p_neg(v.im), v.re} : c2{v.im, p_neg(v.re)};
  if (e == 8) return c2{p_neg(v.re), p_neg(v.im)};
  if (e == 12) return DIR > 0 ? c2{v.im, p_neg(v.re)} : c2{p_neg(v.im), v.re};
  const int k = 2 * e;  // in 32nds of a turn
  float c = kCos32[k & 15], sn = kSin32[k & 15];
  if (k >= 16) {
    c = -c;
    sn = -sn;
  }
  if (DIR < 0) sn = -sn;
  const float2 C = make_float2(c, c);
  if (c == sn) return c2{p_mul(p_sub(v.re, v.im), C), p_mul(p_add(v.re, v.im), C)};
  if (c == -sn) return c2{p_mul(p_add(v.re, v.im), C), p_mul(p_sub(v.im, v.re), C)};
  return c2{p_fma(v.re, C, p_mul(v.im, make_float2(-sn, -sn))),
            p_fma(v.re, make_float2(sn, sn), p_mul(v.im, C))};
}

// In-place 4-point DFT of two independent lanes, a_n -> X_k (natural
// order), X_k = sum_n a_n exp(DIR 2 pi i n k / 4); the factor DIR i of the
// odd outputs is folded into the adds.
template <int DIR>
FDAS_DEV void dft4_pairs(c2& a0, c2& a1, c2& a2, c2& a3) {
  const c2 t0 = c2_add(a0, a2), t1 = c2_sub(a0, a2), t2 = c2_add(a1, a3), t3 = c2_sub(a1, a3);
  a0 = c2_add(t0, t2);
  a2 = c2_sub(t0, t2);
  if (DIR > 0) {  // X1 = t1 + i t3, X3 = t1 - i t3
    a1 = c2{p_sub(t1.re, t3.im), p_add(t1.im, t3.re)};
    a3 = c2{p_add(t1.re, t3.im), p_sub(t1.im, t3.re)};
  } else {        // X1 = t1 - i t3, X3 = t1 + i t3
    a1 = c2{p_add(t1.re, t3.im), p_sub(t1.im, t3.re)};
    a3 = c2{p_sub(t1.re, t3.im), p_add(t1.im, t3.re)};
  }
}

// 16-point DFT of two independent lanes as 4 x 4 (decimation in frequency:
// 4-point DFTs over n2 of x[n1 + 4 n2], twiddles exp(DIR 2 pi i n1 k1 / 16),
// 4-point DFTs over n1); output k sits in x[brev<16>(k)], as with
// dft2_brev<16, DIR>.
template <int DIR>
FDAS_DEV void dft16_pairs(c2 (&x)[16]) {
  c2 y[16];  // y[n1 + 4 k1]
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    c2 a0 = x[n1], a1 = x[n1 + 4], a2 = x[n1 + 8], a3 = x[n1 + 12];
    dft4_pairs<DIR>(a0, a1, a2, a3);
    y[n1] = a0;
    y[n1 + 4] = c2_tw16<DIR>(a1, n1);
    y[n1 + 8] = c2_tw16<DIR>(a2, 2 * n1);
    y[n1 + 12] = c2_tw16<DIR>(a3, 3 * n1);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    c2 a0 = y[4 * k1], a1 = y[4 * k1 + 1], a2 = y[4 * k1 + 2], a3 = y[4 * k1 + 3];
    dft4_pairs<DIR>(a0, a1, a2, a3);
    x[brev<16>(k1)] = a0;
    x[brev<16>(k1 + 4)] = a1;
    x[brev<16>(k1 + 8)] = a2;
    x[brev<16>(k1 + 12)] = a3;
  }
}

// the in-register DFT of R pairs used by the correlation (same output order
// as dft2_brev<R, DIR>)
template <int R, int DIR>
FDAS_DEV void dft_pairs(c2 (&x)[R]) {
  if constexpr (R == 16) dft16_pairs<DIR>(x);
  else dft2_brev<R, DIR>(x);
}

// Radix-32 DFT over index e = 2 p + lane held as 16 pairs (p = 0..15,
// lane 0 = even e, lane 1 = odd e). The first four radix-2 stages pair an
// element with another of equal parity, so they run packed; the last stage
// combines the two lanes of a pair and runs on scalars. On return out[e] is
// DFT output number brev<32>(e).
template <int DIR>
FDAS_DEV void dft32_pairs(c2 (&x)[16], float2 (&out)[32]) {
#pragma unroll
  for (int half = 16; half >= 2; half >>= 1) {
    const int hp = half / 2;  // distance in pairs
#pragma unroll
    for (int blk = 0; blk < 16; blk += 2 * hp) {
#pragma unroll
      for (int jp = 0; jp < hp; ++jp) {
        const c2 a = x[blk + jp];
        const c2 b = x[blk + jp + hp];
        x[blk + jp] = c2_add(a, b);
        x[blk + jp + hp] = c2_rot<DIR>(c2_sub(a, b), 2 * jp, 2 * jp + 1, 2 * half);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const c2 v = x[p];
    out[2 * p] = make_float2(v.re.x + v.re.y, v.im.x + v.im.y);
    out[2 * p + 1] = make_float2(v.re.x - v.re.y, v.im.x - v.im.y);
  }
}

// 16-byte asynchronous global -> shared copy (L2 only); with ok false the
// destination is zero-filled and nothing is read.
FDAS_DEV void cp_async16(void* dst, const void* src, bool ok = true) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
FDAS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed copy groups are pending
template <int N>
FDAS_DEV void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Radix-32 DFT by decimation in time over index e = 2 p + lane held as 16
// pairs (p = 0..15, lane 0 = even e, lane 1 = odd e): the two lanes'
// 16-point DFTs E and O run packed with the same twiddles in both lanes, then
// outputs k and k + 16 are E[k] +- exp(DIR 2 pi i k / 32) O[k] on scalars.
// f(n, value) receives output n in natural order; x is overwritten.
template <int DIR, typename F>
FDAS_DEV void dft32_dit(c2 (&x)[16], F&& f) {
  dft16_pairs<DIR>(x);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const c2 v = x[brev<16>(k)];
    const float2 E = make_float2(v.re.x, v.im.x);
    float2 t = make_float2(v.re.y, v.im.y);  // O[k]
    if (k == 8) {
      t = DIR > 0 ? make_float2(-t.y, t.x) : make_float2(t.y, -t.x);
    } else if (k != 0) {
      const float c = kCos32[k], sn = DIR < 0 ? -kSin32[k] : kSin32[k];
      t = make_float2(t.x * c - t.y * sn, t.x * sn + t.y * c);
    }
    f(k, make_float2(E.x + t.x, E.y + t.y));
    f(k + 16, make_float2(E.x - t.x, E.y - t.y));
  }
}

}  // namespace fdas
