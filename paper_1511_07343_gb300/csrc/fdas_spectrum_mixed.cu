// Step 2 of Section 4 for series lengths N = 2^a 3^b 5^c (de-dispersed DM
// trials of uneven length): the same four-step structure as the
// power-of-two path (columns with the M-point twiddle, rows, real unpack),
// with runtime-sized Stockham transforms built from radix-16, 8, 4, 2, 5 and
// 3 stages in shared memory (ping-pong buffers, one barrier per stage).
#include "fdas_common.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr int kNT = 256;
constexpr int kMaxStages = 24;

struct RtSched {
  int n;
  int r[kMaxStages];
};

// y_k = sum_j x_j exp(DIR 2 pi i j k / 3), natural order
template <int DIR>
FDAS_DEV void dft3(float2 (&x)[3]) {
  constexpr float kS = 0.86602540378443865f * DIR;  // DIR sin(2 pi / 3)
  const float2 t1 = cadd(x[1], x[2]);
  const float2 t2 = csub(x[1], x[2]);
  const float2 m = make_float2(x[0].x - 0.5f * t1.x, x[0].y - 0.5f * t1.y);
  x[0] = cadd(x[0], t1);
  // i kS t2 = (-kS t2.y, kS t2.x)
  x[1] = make_float2(m.x - kS * t2.y, m.y + kS * t2.x);
  x[2] = make_float2(m.x + kS * t2.y, m.y - kS * t2.x);
}

// y_k = sum_j x_j exp(DIR 2 pi i j k / 5), natural order
template <int DIR>
FDAS_DEV void dft5(float2 (&x)[5]) {
  constexpr float c1 = 0.30901699437494742f;   // cos(2 pi / 5)
  constexpr float c2 = -0.80901699437494742f;  // cos(4 pi / 5)
  constexpr float s1 = 0.95105651629515357f * DIR;
  constexpr float s2 = 0.58778525229247313f * DIR;
  const float2 a1 = cadd(x[1], x[4]), b1 = csub(x[1], x[4]);
  const float2 a2 = cadd(x[2], x[3]), b2 = csub(x[2], x[3]);
  const float2 x0 = x[0];
  const float2 p1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
  const float2 p2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
  const float2 q1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
  const float2 q2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
  x[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
  // p +- i q
  x[1] = make_float2(p1.x - q1.y, p1.y + q1.x);
  x[4] = make_float2(p1.x + q1.y, p1.y - q1.x);
  x[2] = make_float2(p2.x - q2.y, p2.y + q2.x);
  x[3] = make_float2(p2.x + q2.y, p2.y - q2.x);
}

template <int R, int DIR>
FDAS_DEV void dft_any(float2 (&x)[R]) {
  if constexpr (R == 3) dft3<DIR>(x);
  else if constexpr (R == 5) dft5<DIR>(x);
  else dft<R, DIR>(x);
}

// one Stockham stage of radix R on NB transforms of length len: src -> dst
template <int R, int DIR>
FDAS_DEV void rt_stage(const float2* src, float2* dst, int len, int ns, int nb_tr,
                       const float2* __restrict__ tw, int tid) {
  const int nbf = len / R;
  const int twstep = len / (ns * R);
  for (int g = tid; g < nbf * nb_tr; g += kNT) {
    const int b = g / nbf, j = g - b * nbf;
    const int jm = j % ns;
    const float2* s = src + b * len + j;
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 v = s[r * nbf];
      if (r > 0 && ns > 1) {
        float2 w = __ldg(tw + r * jm * twstep);
        if (DIR > 0) w.y = -w.y;
        v = cmul(v, w);
      }
      x[r] = v;
    }
    dft_any<R, DIR>(x);
    float2* d = dst + b * len + (j / ns) * ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * ns] = x[r];
  }
}

// full transform; returns the buffer holding the result
template <int DIR>
FDAS_DEV float2* rt_fft(float2* a, float2* b, int len, const RtSched& sch, int nb_tr,
                        const float2* __restrict__ tw, int tid) {
  int ns = 1;
  for (int s = 0; s < sch.n; ++s) {
    const int R = sch.r[s];
    switch (R) {
      case 16: rt_stage<16, DIR>(a, b, len, ns, nb_tr, tw, tid); break;
      case 8: rt_stage<8, DIR>(a, b, len, ns, nb_tr, tw, tid); break;
      case 4: rt_stage<4, DIR>(a, b, len, ns, nb_tr, tw, tid); break;
      case 2: rt_stage<2, DIR>(a, b, len, ns, nb_tr, tw, tid); break;
      case 5: rt_stage<5, DIR>(a, b, len, ns, nb_tr, tw, tid); break;
      case 3: rt_stage<3, DIR>(a, b, len, ns, nb_tr, tw, tid); break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    ns *= R;
  }
  return a;
}

// columns: for n1 in [b0, b0+NB) the DFT over n2 of z[n1 + M1 n2] (length
// M2), times exp(-2 pi i n1 k2 / M), stored as T[k2 M1 + n1]
__global__ void __launch_bounds__(kNT) k_fft_cols_rt(const float2* __restrict__ z,
                                                     float2* __restrict__ T, int M1, int M2,
                                                     int nb_tr, RtSched sch,
                                                     const float2* __restrict__ tw_len,
                                                     const float2* __restrict__ tw_lo,
                                                     const float2* __restrict__ tw_hi, int h4) {
  extern __shared__ float2 sm[];
  float2* a = sm;
  float2* b = sm + nb_tr * M2;
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * nb_tr;
  const int nt = min(nb_tr, M1 - b0);
  for (int i = tid; i < nb_tr * M2; i += kNT) {
    const int bb = i % nb_tr, e = i / nb_tr;
    a[bb * M2 + e] = bb < nt ? z[(size_t)(b0 + bb) + (size_t)M1 * e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res = rt_fft<kFwd>(a, b, M2, sch, nb_tr, tw_len, tid);
  const int mask = (1 << h4) - 1;
  for (int i = tid; i < nt * M2; i += kNT) {
    const int bb = i % nt, k2 = i / nt;
    const int n1 = b0 + bb;
    const long long e = (long long)n1 * k2;
    const float2 w = cmul(__ldg(tw_lo + (e & mask)), __ldg(tw_hi + (e >> h4)));
    T[(size_t)k2 * M1 + n1] = cmul(res[bb * M2 + k2], w);
  }
}

// rows: for k2 in [b0, b0+NB) the DFT over n1 of T[k2 M1 + n1] (length M1),
// stored as Z[k2 + M2 k1]
__global__ void __launch_bounds__(kNT) k_fft_rows_rt(const float2* __restrict__ T,
                                                     float2* __restrict__ Zo, int M1, int M2,
                                                     int nb_tr, RtSched sch,
                                                     const float2* __restrict__ tw_len) {
  extern __shared__ float2 sm[];
  float2* a = sm;
  float2* b = sm + nb_tr * M1;
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * nb_tr;
  const int nt = min(nb_tr, M2 - b0);
  for (int i = tid; i < nb_tr * M1; i += kNT) {
    const int bb = i / M1, e = i % M1;
    a[bb * M1 + e] = bb < nt ? T[(size_t)(b0 + bb) * M1 + e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* res = rt_fft<kFwd>(a, b, M1, sch, nb_tr, tw_len, tid);
  for (int i = tid; i < nt * M1; i += kNT) {
    const int bb = i % nt, k1 = i / nt;
    Zo[(size_t)(b0 + bb) + (size_t)M2 * k1] = res[bb * M1 + k1];
  }
}

RtSched schedule_of(int len) {
  RtSched s;
  s.n = 0;
  int x = len;
  while (x % 16 == 0 && s.n < kMaxStages) { s.r[s.n++] = 16; x /= 16; }
  while (x % 5 == 0 && s.n < kMaxStages) { s.r[s.n++] = 5; x /= 5; }
  while (x % 3 == 0 && s.n < kMaxStages) { s.r[s.n++] = 3; x /= 3; }
  while (x % 8 == 0 && s.n < kMaxStages) { s.r[s.n++] = 8; x /= 8; }
  while (x % 4 == 0 && s.n < kMaxStages) { s.r[s.n++] = 4; x /= 4; }
  while (x % 2 == 0 && s.n < kMaxStages) { s.r[s.n++] = 2; x /= 2; }
  return s;
}

int batch_of(int len) {
  int nb = 4096 / len;
  return nb < 1 ? 1 : nb;
}

}  // namespace

bool is_235(int64_t x) {
  if (x < 1) return false;
  for (int f : {2, 3, 5})
    while (x % f == 0) x /= f;
  return x == 1;
}

// M = M1 * M2 with both factors 2^i 3^j 5^k in [16, 8192], as balanced as
// possible; false if no such split exists.
bool split_235(int64_t M, int* M1, int* M2) {
  int best = -1;
  double best_d = 1e30;
  for (int64_t d = 16; d <= 8192; ++d) {
    if (M % d || !is_235(d)) continue;
    const int64_t e = M / d;
    if (e < 16 || e > 8192) continue;
    const double r = (double)d / (double)e;
    const double dd = r > 1 ? r : 1.0 / r;
    if (dd < best_d || (dd == best_d && d > best)) {
      best_d = dd;
      best = (int)d;
    }
  }
  if (best < 0) return false;
  // the larger factor goes to M1 (row transforms are contiguous)
  const int64_t other = M / best;
  *M1 = (int)(best > other ? best : other);
  *M2 = (int)(best > other ? other : best);
  return true;
}

int launch_spectrum_mixed(fdas_plan* p, const float* d_series, float2* d_spec) {
  const float2* z = reinterpret_cast<const float2*>(d_series);
  {
    const RtSched sch = schedule_of(p->M2);
    const int nb_tr = batch_of(p->M2);
    const size_t smem = sizeof(float2) * 2 * (size_t)nb_tr * p->M2;
    cudaError_t e = cudaFuncSetAttribute(k_fft_cols_rt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "k_fft_cols_rt attr");
    const unsigned grid = (unsigned)((p->M1 + nb_tr - 1) / nb_tr);
    k_fft_cols_rt<<<grid, kNT, smem, p->stream>>>(z, p->zbuf, p->M1, p->M2, nb_tr, sch, p->tw_M2,
                                                  p->tw4_lo, p->tw4_hi, p->h4);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(e, "k_fft_cols_rt");
  }
  {
    const RtSched sch = schedule_of(p->M1);
    const int nb_tr = batch_of(p->M1);
    const size_t smem = sizeof(float2) * 2 * (size_t)nb_tr * p->M1;
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows_rt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "k_fft_rows_rt attr");
    const unsigned grid = (unsigned)((p->M2 + nb_tr - 1) / nb_tr);
    k_fft_rows_rt<<<grid, kNT, smem, p->stream>>>(p->zbuf, p->spec2, p->M1, p->M2, nb_tr, sch,
                                                  p->tw_M1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(e, "k_fft_rows_rt");
  }
  return launch_unpack(p, d_spec);
}

}  // namespace fdas
