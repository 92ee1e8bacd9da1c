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

namespace fdas {
namespace {

constexpr int kNT = 256;

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
  float2* out = seg + (size_t)s * L;
  for (int i = tid; i < L; i += kNT) out[i] = sbuf[i];
}

// Steps 5-7, reference form: one CTA per (segment, group of ZG templates);
// the segment spectrum stays in shared memory while each template is
// multiplied in, inverse-transformed and its valid outputs squared.
template <int L, int ZG>
__global__ void __launch_bounds__(kNT) k_correlate_ref(const float2* __restrict__ seg,
                                                       const float2* __restrict__ bank,
                                                       float* __restrict__ plane, int64_t nb,
                                                       int Z, int V, int m,
                                                       const float2* __restrict__ tw) {
  extern __shared__ float2 sbuf[];
  float2* F = sbuf;
  float2* W = sbuf + L;
  const int tid = threadIdx.x;
  const int s = blockIdx.x;
  const int z0 = blockIdx.y * ZG;
  const float2* fs = seg + (size_t)s * L;
  for (int i = tid; i < L; i += kNT) F[i] = fs[i];
  const int64_t r0 = (int64_t)s * V;
  for (int j = z0; j < z0 + ZG && j < Z; ++j) {
    __syncthreads();
    const float2* tz = bank + (size_t)j * L;
    for (int i = tid; i < L; i += kNT) W[i] = cmul(F[i], __ldg(tz + i));
    __syncthreads();
    block_fft<L, kInv, kNT, 1>(W, tw, tid);
    float* prow = plane + (size_t)j * nb;
    for (int i = tid; i < V; i += kNT) {
      const int64_t r = r0 + i;
      if (r < nb) prow[r] = cnorm(W[m / 2 + i]);
    }
  }
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

template <int L>
int corr_launch(fdas_plan* p, float* plane) {
  constexpr int ZG = 8;
  const size_t smem = sizeof(float2) * 2 * L;
  cudaError_t e = cudaFuncSetAttribute(k_correlate_ref<L, ZG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "k_correlate_ref attr");
  dim3 grid(p->S, (p->Z + ZG - 1) / ZG);
  k_correlate_ref<L, ZG><<<grid, kNT, smem, p->stream>>>(p->seg, p->bank, plane, p->nb, p->Z,
                                                           p->V, p->m, p->tw_L);
  return cuda_check(cudaGetLastError(), "k_correlate_ref");
}

}  // namespace

int launch_segments(fdas_plan* p, const float2* d_white) {
  switch (p->L) {
    case 2048: return seg_launch<2048>(p, d_white);
    case 4096: return seg_launch<4096>(p, d_white);
    case 8192: return seg_launch<8192>(p, d_white);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported segment length");
}

int launch_correlate(fdas_plan* p, float* d_plane) {
  switch (p->L) {
    case 2048: return corr_launch<2048>(p, d_plane);
    case 4096: return corr_launch<4096>(p, d_plane);
    case 8192: return corr_launch<8192>(p, d_plane);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported segment length");
}

}  // namespace fdas
