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

// Steps 5-7, fused: one pass per (segment, template) pair through
//   Y = F_s * T_z  ->  inverse FFT  ->  |.|^2  ->  keep the V valid outputs,
// with the complex plane never leaving the SM. Layout of the length-L inverse
// FFT (L = 32 NA, NA = 16 RA2 threads):
//   k = k1 + 32 k2, k2 = a + RA2 b;   n = n2 + NA n1, n2 = c + 16 d
//   A1 (per thread, 2 x radix-16 over b): u = sum_b Y[k1 + 32 a + 32 RA2 b] w16^{bc},
//      times w_NA^{ac}                                   (k1 = lane, a = warp + NW h)
//   A2 (32/RA2 x radix-RA2 over a): Z[k1][c + 16 d], times w_L^{k1 (c + 16 d)}
//   B  (radix-32 over k1): c[n2 + NA n1]                 (n2 = thread index)
// Two shared-memory exchanges per pair (A1->A2, A2->B). The segment spectrum
// F_s is held in tensor memory for the whole sweep over templates; the
// template spectra stream from L2. Besides the plane row the kernel writes
// the 4-bin maximum Q4[z][r/4] (used to screen the harmonic sums) and emits
// the h = 1 candidates. Work is a static, evenly split range of pairs per
// CTA (one wave of resident CTAs).
template <int L>
struct Corr {
  static constexpr int T = L / 32;
  static constexpr int NA = L / 32;
  static constexpr int RA2 = NA / 16;
  static constexpr int NW = T / 32;
  static constexpr int XP = NA + 1;
  static constexpr int XF = (L > 32 * XP) ? L : 32 * XP;
  static constexpr int NCOLS = NW > 4 ? 128 : 64;
  static constexpr int MAXCTA = 512 / NCOLS;
  static constexpr int MINB = L == 8192 ? 2 : (L == 4096 ? 4 : 8);
  static constexpr size_t SMEM = sizeof(float2) * (XF + NA) + sizeof(float) * L;
};

template <int L>
__global__ void __launch_bounds__(Corr<L>::T, Corr<L>::MINB)
    k_correlate_fused(const float2* __restrict__ seg, const float2* __restrict__ bank,
                      float* __restrict__ plane, float* __restrict__ q4, int64_t nb, int Z, int V,
                      int m, int64_t n_pairs, const float2* __restrict__ twL, float thr1,
                      fdas_cand* __restrict__ cands, unsigned long long* count, int64_t maxc) {
  using C = Corr<L>;
  constexpr int T = C::T, NA = C::NA, RA2 = C::RA2, NW = C::NW, XP = C::XP;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* twA = smem + C::XF;  // exp(+2 pi i e / NA)
  float* Ps = reinterpret_cast<float*>(smem + C::XF + NA);  // powers of the kept outputs
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < NA; e += T) twA[e] = cconj(__ldg(twL + e * 32));
  if (warp == 0) {
    tmem_alloc(&s_tmem, C::NCOLS);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase =
      s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)(warp >> 2);

  // exp(+2 pi i 16 e lane / L) for e = 1, 2, 4, 8 (B-stage twiddle steps)
  const float2 st1 = cconj(__ldg(twL + ((16 * lane) & (L - 1))));
  const float2 st2 = cconj(__ldg(twL + ((32 * lane) & (L - 1))));
  const float2 st4 = cconj(__ldg(twL + ((64 * lane) & (L - 1))));
  const float2 st8 = cconj(__ldg(twL + ((128 * lane) & (L - 1))));
  const int half_m = m / 2;
  const int64_t nq = nb >> 2;

  const int64_t p0 = (int64_t)blockIdx.x * n_pairs / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * n_pairs / gridDim.x;
  int s_cur = -1;
  for (int64_t p = p0; p < p1; ++p) {
    const int s = (int)(p / Z);
    const int z = (int)(p - (int64_t)s * Z);
    if (s != s_cur) {  // segment spectrum -> tensor memory
      const float2* fs = seg + (size_t)s * L;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float f[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int idx = q * 8 + i;
          const float2 v = __ldg(fs + tid + T * (idx >> 4) + 2 * T * (idx & 15));
          f[2 * i] = v.x;
          f[2 * i + 1] = v.y;
        }
        tmem_st16(tbase + 16 * q, f);
      }
      tmem_wait_st();
      s_cur = s;
    }
    // ---- A1
    float2 v[2][16];
    const float2* tz = bank + (size_t)z * L;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int b = 0; b < 16; ++b) v[h][b] = __ldg(tz + tid + T * h + 2 * T * b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[16];
      tmem_ld16(tbase + 16 * q, f);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int idx = q * 8 + i;
        v[idx >> 4][idx & 15] = cmul(v[idx >> 4][idx & 15], make_float2(f[2 * i], f[2 * i + 1]));
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      dft_brev<16, kInv>(v[h]);
      const int a = warp + NW * h;
#pragma unroll
      for (int c = 1; c < 16; ++c)
        v[h][brev<16>(c)] = cmul(v[h][brev<16>(c)], twA[(a * c) & (NA - 1)]);
#pragma unroll
      for (int c = 0; c < 16; ++c) X[(a * 16 + c) * 32 + lane] = v[h][brev<16>(c)];
    }
    __syncthreads();
    // ---- A2
    constexpr int NB2 = 32 / RA2;
    float2 w[NB2][RA2];
#pragma unroll
    for (int i = 0; i < NB2; ++i) {
      const int c = warp + NW * i;
#pragma unroll
      for (int a = 0; a < RA2; ++a) w[i][a] = X[(a * 16 + c) * 32 + lane];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB2; ++i) {
      dft_brev<RA2, kInv>(w[i]);
      const int c = warp + NW * i;
      float2 W[RA2];
      W[0] = cconj(__ldg(twL + lane * c));
      if constexpr (RA2 > 1) W[1] = cmul(W[0], st1);
      if constexpr (RA2 > 2) {
        W[2] = cmul(W[0], st2);
        W[3] = cmul(W[2], st1);
      }
      if constexpr (RA2 > 4) {
        W[4] = cmul(W[0], st4);
        W[5] = cmul(W[4], st1);
        W[6] = cmul(W[4], st2);
        W[7] = cmul(W[6], st1);
      }
      if constexpr (RA2 > 8) {
#pragma unroll
        for (int k = 0; k < 8; ++k) W[8 + k] = cmul(W[k], st8);
      }
#pragma unroll
      for (int d = 0; d < RA2; ++d) X[lane * XP + c + 16 * d] = cmul(w[i][brev<RA2>(d)], W[d]);
    }
    __syncthreads();
    // ---- B
    float2 y[32];
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) y[k1] = X[k1 * XP + tid];
    dft_brev<32, kInv>(y);
    // powers of the kept outputs n in [m/2, L - m/2) -> Ps[n - m/2]
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
      const int n = tid + NA * n1;
      if (n >= half_m && n < L - half_m) Ps[n - half_m] = cnorm(y[brev<32>(n1)]);
    }
    __syncthreads();
    // coalesced float4 stores of the plane row slice, its 4-bin maxima and
    // the h = 1 candidates; r = s V + i, i < V, r < nb
    const int64_t r0 = (int64_t)s * V;
    int64_t nvalid = nb - r0;
    if (nvalid > V) nvalid = V;
    const int n4 = (int)(nvalid >> 2);
    float* prow = plane ? plane + (size_t)z * nb + r0 : nullptr;
    float* qrow = q4 ? q4 + (size_t)z * nq + (r0 >> 2) : nullptr;
    const float4* P4 = reinterpret_cast<const float4*>(Ps);
    bool hit = false;
    for (int k = tid; k < n4; k += T) {
      const float4 v4 = P4[k];
      if (prow) reinterpret_cast<float4*>(prow)[k] = v4;
      if (qrow) qrow[k] = fmaxf(fmaxf(v4.x, v4.y), fmaxf(v4.z, v4.w));
      hit |= fmaxf(fmaxf(v4.x, v4.y), fmaxf(v4.z, v4.w)) >= thr1;
    }
    if (cands && __syncthreads_or(hit)) {
      // rare: some power reached T_1; scan the slice again and append
      for (int k0 = 0; k0 < n4; k0 += T) {
        const int k = k0 + tid;
        const bool in = k < n4;
        const float4 v4 = in ? P4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int rk = (int)(r0 + 4 * k);
        emit(in && rk >= 1 && v4.x >= thr1, rk, z, 1, v4.x, cands, count, maxc);
        emit(in && v4.y >= thr1, rk + 1, z, 1, v4.y, cands, count, maxc);
        emit(in && v4.z >= thr1, rk + 2, z, 1, v4.z, cands, count, maxc);
        emit(in && v4.w >= thr1, rk + 3, z, 1, v4.w, cands, count, maxc);
      }
    }
    // no barrier needed here: the next pair's first writes to X come after
    // its own A1 work, and its Ps writes after three more barriers
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(s_tmem, C::NCOLS);
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
  cudaError_t e = cudaFuncSetAttribute(k_correlate_fused<L>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "k_correlate_fused attr");
  e = cudaFuncSetAttribute(k_correlate_fused<L>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return cuda_check(e, "k_correlate_fused carveout");
  // Resident CTAs per SM from the kernel's own resource use (registers in
  // units of 8 per thread, shared memory incl. the 1 KB per-CTA reserve,
  // threads), capped by the tensor-memory budget.
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_correlate_fused<L>);
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
  const int64_t n_pairs = (int64_t)p->S * p->Z;
  int64_t grid = (int64_t)occ * sms;
  if (grid > n_pairs) grid = n_pairs;
  p->corr_grid = (int)grid;
  k_correlate_fused<L><<<(unsigned)grid, C::T, smem, p->stream>>>(
      p->seg, p->bank, plane, q4, p->nb, p->Z, p->V, p->m, n_pairs, p->tw_L, p->thr[0], cands,
      count, p->max_cands);
  return cuda_check(cudaGetLastError(), "k_correlate_fused");
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

int launch_correlate(fdas_plan* p, float* d_plane, float* d_q4, fdas_cand* d_cands,
                     unsigned long long* d_count) {
  switch (p->L) {
    case 2048: return corr_launch<2048>(p, d_plane, d_q4, d_cands, d_count);
    case 4096: return corr_launch<4096>(p, d_plane, d_q4, d_cands, d_count);
    case 8192: return corr_launch<8192>(p, d_plane, d_q4, d_cands, d_count);
  }
  return set_error(FDAS_ERR_INVALID, "unsupported segment length");
}

}  // namespace fdas
