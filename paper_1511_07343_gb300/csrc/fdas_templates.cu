// Initialisation stage of Section 4: the z-template bank and the float64
// twiddle tables.
//
// Template (Section 2, the response of a constant-acceleration signal,
// conjugated so that correlating with it gathers the drifted power back into
// one bin, Eq. 1):
//     tau_z(d) = int_0^1 exp(2 pi i [(d + z/2) u - z u^2 / 2]) du.
// Completing the square, with q = d + z/2 and s_a = sqrt(2|z|) (a - q/z):
//     tau_z(d) = conj( exp(-i pi q^2 / z) [dC + i sgn(z) dS] ) / sqrt(2|z|),
// where dC = C(s_1) - C(s_0), dS = S(s_1) - S(s_0) are differences of the
// Fresnel integrals F(x) = C(x) + i S(x) = int_0^x exp(i pi t^2 / 2) dt.
//
// F is evaluated in float64 from its own mathematics:
//  * |x| <= 1.8: the power series F(x) = sum_k (i pi/2)^k x^(2k+1) / (k! (2k+1));
//  * |x| > 1.8: F(x) = sgn(x) [(1+i)/2 + G(|x|)], G(x) = -((1+i)/2) erfc(w),
//    w = (sqrt(pi)/2)(1-i) x, with erfc from its Laplace continued fraction
//    sqrt(pi) exp(w^2) erfc(w) = 1/(w + (1/2)/(w + 1/(w + (3/2)/(w + ...)))),
//    summed by the modified Lentz method. Differences of two tails are taken
//    as G - G so that the (1+i)/2 parts cancel exactly.
#include <math.h>

#include "fdas_common.cuh"
#include "fdas_internal.h"

namespace fdas {
namespace {

#define HD __host__ __device__ __forceinline__

struct cd {
  double re, im;
};
HD cd mk(double a, double b) { return cd{a, b}; }
HD cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
HD cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
HD cd operator*(cd a, cd b) { return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
HD cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
HD double cabs1(cd a) { return fabs(a.re) + fabs(a.im); }
// Smith's scaled complex reciprocal
HD cd crecip(cd b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return cd{1.0 / den, -r / den};
  }
  const double r = b.re / b.im, den = b.re * r + b.im;
  return cd{r / den, -1.0 / den};
}
HD cd cdiv(cd a, cd b) { return a * crecip(b); }

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr double kCut = 1.8;

HD void sincospi_d(double x, double* s, double* c) {
#ifdef __CUDA_ARCH__
  sincospi(x, s, c);
#else
  *s = sin(kPi * x);
  *c = cos(kPi * x);
#endif
}

// F(x) by its power series (0 <= x <= kCut).
HD cd fresnel_series(double x) {
  const double x2 = x * x;
  cd term = mk(x, 0.0);
  cd sum = term;
  for (int k = 1; k < 100; ++k) {
    const double f = 0.5 * kPi * x2 / k;
    term = mk(-term.im * f, term.re * f);  // * (i f)
    const double inv = 1.0 / (2 * k + 1);
    const cd add = inv * term;
    sum = sum + add;
    if (cabs1(add) <= 1e-18 * cabs1(sum)) break;
  }
  return sum;
}

// G(x) = F(x) - (1+i)/2 for x > kCut. exp(i pi x^2/2) is passed in (as
// cos, sin) so that callers with an exactly known phase can supply it.
HD cd fresnel_tail(double x, double ph_c, double ph_s) {
  const double c = 0.5 * kSqrtPi * x;
  const cd w = mk(c, -c);
  const double tiny = 1e-300;
  cd f = w, C = w, D = mk(0.0, 0.0);
  for (int n = 1; n < 20000; ++n) {
    const double a = 0.5 * n;
    D = w + a * D;
    if (cabs1(D) == 0.0) D = mk(tiny, 0.0);
    D = crecip(D);
    C = w + cdiv(mk(a, 0.0), C);
    if (cabs1(C) == 0.0) C = mk(tiny, 0.0);
    const cd delta = C * D;
    f = f * delta;
    if (cabs1(delta - mk(1.0, 0.0)) < 2e-16) break;
  }
  // erfc(w) = exp(-w^2) / (sqrt(pi) f), exp(-w^2) = exp(i pi x^2 / 2)
  const cd erfcw = (1.0 / kSqrtPi) * cdiv(mk(ph_c, ph_s), f);
  return -0.5 * (mk(1.0, 1.0) * erfcw);
}

HD cd fresnel_generic(double x) {
  const double ax = fabs(x);
  cd v;
  if (ax <= kCut) {
    v = fresnel_series(ax);
  } else {
    double s, c;
    const double h = 0.5 * ax * ax;
    sincospi_d(fmod(h, 2.0), &s, &c);
    v = mk(0.5, 0.5) + fresnel_tail(ax, c, s);
  }
  return x < 0 ? -1.0 * v : v;
}

// F(s1) - F(s0), with exact phases exp(i pi s_a^2/2) given for both points.
HD cd fresnel_diff(double s0, double c0, double sn0, double s1, double c1, double sn1) {
  const bool t0 = fabs(s0) > kCut, t1 = fabs(s1) > kCut;
  if (t0 && t1 && ((s0 > 0) == (s1 > 0))) {
    const cd g = fresnel_tail(fabs(s1), c1, sn1) - fresnel_tail(fabs(s0), c0, sn0);
    return s1 > 0 ? g : -1.0 * g;
  }
  auto F = [](double s, double c, double sn, bool tail) -> cd {
    cd v = tail ? mk(0.5, 0.5) + fresnel_tail(fabs(s), c, sn) : fresnel_series(fabs(s));
    return s < 0 ? -1.0 * v : v;
  };
  return F(s1, c1, sn1, t1) - F(s0, c0, sn0, t0);
}

// tau_z at q = d - offset + z/2 for integer z = zi, given Q = 2q (an
// integer for integer d and z and offsets 0 or 1/2), float64.
HD cd template_tap_q2(int zi, long long Q) {
  if (zi == 0) {
    // int_0^1 exp(2 pi i q u) du: delta at q = 0 for integer q; for
    // half-integer q, exp(2 pi i q) = -1 gives i / (pi q)
    if ((Q & 1) == 0) return Q == 0 ? mk(1.0, 0.0) : mk(0.0, 0.0);
    return mk(0.0, 2.0 / (3.14159265358979323846 * (double)Q));
  }
  const int az = zi < 0 ? -zi : zi;
  const double sg = zi < 0 ? -1.0 : 1.0;
  const double q = 0.5 * (double)Q;
  const double scale = sqrt(2.0 * az);
  const double s0 = scale * (0.0 - q / zi);
  const double s1 = scale * (1.0 - q / zi);
  // s0^2/2 = Q^2/(4|z|) and s1^2/2 = (2z - Q)^2/(4|z|): reduce mod 2 exactly.
  const long long den = 4LL * az;
  const long long n0 = (Q * Q) % (2 * den);
  const long long R1 = 2LL * zi - Q;
  const long long n1 = (R1 * R1) % (2 * den);
  double c0, sn0, c1, sn1;
  sincospi_d((double)n0 / (double)den, &sn0, &c0);
  sincospi_d((double)n1 / (double)den, &sn1, &c1);
  const cd dF = fresnel_diff(s0, c0, sn0, s1, c1, sn1);
  const cd dFz = mk(dF.re, sg * dF.im);  // dC + i sgn(z) dS
  // exp(-i pi q^2/z) = exp(-i pi sgn(z) n0/den)
  const cd ph = mk(c0, -sg * sn0);
  const cd t = ph * dFz;
  return mk(t.re / scale, -t.im / scale);
}

// rows = 1: row j holds tau_{z_j}; rows = 2: row 2j + e holds tau_{z_j} at
// frequency offset e/2 (the half-bin bank), q = d - e/2 + z/2.
__global__ void k_template_taps(double2* __restrict__ taps, int Z, int m, int zmax, int dz,
                                int rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (i >= m || row >= Z * rows) return;
  const int j = row / rows, e = row % rows;
  const int z = -zmax + j * dz;
  const cd t = template_tap_q2(z, 2LL * (i - m / 2) + z - e);
  taps[(size_t)row * m + i] = make_double2(t.re, t.im);
}

// bank[j][k] = (1/L) sum_i taps[j][i] exp(+2 pi i k (i - m/2) / L), float64
// accumulation, rotation by recurrence re-seeded every 32 taps.
__global__ void k_template_bank(const double2* __restrict__ taps, float2* __restrict__ bank,
                                int m, int L) {
  extern __shared__ double2 s_taps[];
  const int j = blockIdx.y;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_taps[i] = taps[(size_t)j * m + i];
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  double ss, cc;
  sincospi_d(2.0 * (double)k / (double)L, &ss, &cc);
  const cd step = mk(cc, ss);
  cd acc = mk(0.0, 0.0);
  cd w = mk(1.0, 0.0);
  for (int i = 0; i < m; ++i) {
    if ((i & 31) == 0) {
      long long e = ((long long)k * (long long)(i - m / 2)) % L;
      if (e < 0) e += L;
      sincospi_d(2.0 * (double)e / (double)L, &ss, &cc);
      w = mk(cc, ss);
    }
    const double2 t = s_taps[i];
    acc = acc + mk(t.x, t.y) * w;
    w = w * step;
  }
  const double inv = 1.0 / (double)L;
  // packed layout: slot ((k2 / RA2) RA2 + k2 % RA2) 16 + u holds
  // (re[2u], re[2u+1], im[2u], im[2u+1]) with k = (2u + e) + 32 k2
  const int RA2 = L / 512;
  const int e = k & 1, u = (k & 31) >> 1, k2 = k >> 5;
  const int slot = ((k2 / RA2) * RA2 + (k2 % RA2)) * 16 + u;
  float* f = reinterpret_cast<float*>(bank) + ((size_t)j * (L / 2) + slot) * 4;
  f[e] = (float)(acc.re * inv);
  f[2 + e] = (float)(acc.im * inv);
}

// out[i] = exp(-2 pi i ((i * mult) mod period) / period), float64 -> float32.
__global__ void k_twiddles(float2* __restrict__ out, int64_t count, int64_t mult, int64_t period) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t e = (i * mult) % period;  // i, mult < 2^26
  double s, c;
  sincospi(2.0 * (double)e / (double)period, &s, &c);
  out[i] = make_float2((float)c, (float)-s);
}

}  // namespace

int launch_twiddles(float2* out, int64_t count, int64_t mult, int64_t period, cudaStream_t s) {
  const int nt = 256;
  const int64_t nblk = (count + nt - 1) / nt;
  k_twiddles<<<(unsigned)nblk, nt, 0, s>>>(out, count, mult, period);
  return cuda_check(cudaGetLastError(), "k_twiddles");
}

int launch_template_taps(fdas_plan* p) {
  dim3 grid((p->m + 127) / 128, p->Z);
  k_template_taps<<<grid, 128, 0, p->stream>>>(p->taps, p->Z, p->m, p->zmax, p->dz, 1);
  return cuda_check(cudaGetLastError(), "k_template_taps");
}

int launch_template_bank(fdas_plan* p) {
  dim3 grid((p->L + 127) / 128, p->Z);
  const size_t smem = sizeof(double2) * p->m;
  k_template_bank<<<grid, 128, smem, p->stream>>>(p->taps, p->bank, p->m, p->L);
  return cuda_check(cudaGetLastError(), "k_template_bank");
}

int launch_template_interbin(fdas_plan* p) {
  dim3 tgrid((p->m + 127) / 128, 2 * p->Z);
  k_template_taps<<<tgrid, 128, 0, p->stream>>>(p->taps_ib, p->Z, p->m, p->zmax, p->dz, 2);
  int rc = cuda_check(cudaGetLastError(), "k_template_taps (half-bin)");
  if (rc) return rc;
  dim3 grid((p->L + 127) / 128, 2 * p->Z);
  const size_t smem = sizeof(double2) * p->m;
  k_template_bank<<<grid, 128, smem, p->stream>>>(p->taps_ib, p->bank_ib, p->m, p->L);
  return cuda_check(cudaGetLastError(), "k_template_bank (half-bin)");
}

void fresnel_host(double x, double* C, double* S) {
  const cd v = fresnel_generic(x);
  *C = v.re;
  *S = v.im;
}

}  // namespace fdas
