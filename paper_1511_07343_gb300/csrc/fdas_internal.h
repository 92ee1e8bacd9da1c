// Internal plan layout and kernel launchers of the FDAS CUDA path.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "../../include/fdas.h"

struct fdas_plan {
  // sizes
  int64_t N = 0, nb = 0, M = 0;  // M = N/2 complex points of the packed real FFT
  int M1 = 0, M2 = 0;            // four-step split M = M1 * M2
  int zmax = 0, dz = 0, Z = 0, m = 0, L = 0, V = 0, S = 0;
  int nharm = 0, n_levels = 0;
  float sigma = 6.f;
  float thr[5] = {0, 0, 0, 0, 0};
  int64_t max_cands = 0;
  cudaStream_t stream = nullptr;

  // tables (float64-made)
  float2* tw_L = nullptr;      // exp(-2 pi i e / L), e < L
  float2* tw_M1 = nullptr;     // exp(-2 pi i e / M1)
  float2* tw_M2 = nullptr;     // exp(-2 pi i e / M2)
  float2* tw4_lo = nullptr;    // four-step twiddle exp(-2 pi i e / M), e < 2^h4
  float2* tw4_hi = nullptr;    //   exp(-2 pi i (e << h4) / M)
  int h4 = 0;
  float2* twN_lo = nullptr;    // real-FFT unpack twiddle exp(-2 pi i k / N), k < 2^hN
  float2* twN_hi = nullptr;
  int hN = 0;

  // templates
  double2* taps = nullptr;     // Z x m float64 taps
  float2* bank = nullptr;      // Z x L spectra, 1/L folded in, packed layout (correlate)

  // per-trial workspaces
  float* series = nullptr;     // N floats (host-input staging)
  float2* zbuf = nullptr;      // M complex (four-step scratch)
  float2* spec = nullptr;      // nb complex spectrum
  float2* spec2 = nullptr;     // M complex packed FFT (before the real-FFT unpack)
  float2* white = nullptr;     // nb complex whitened spectrum
  float2* seg = nullptr;       // S x L segment spectra, packed layout (correlate)
  float* plane = nullptr;      // Z x nb power plane
  float* q4 = nullptr;         // Z x nb/4 maxima of 4 consecutive plane bins
  fdas_cand* cands = nullptr;  // max_cands
  unsigned long long* count = nullptr;
  // pairs of top bins the harmonic-sum screen flags, (j << 32) | r, for the
  // exact sums (kHsListCap entries; flags past the capacity are summed inline)
  unsigned long long* hs_list = nullptr;
  // [0] entries in hs_list, [1] the correlation's next chunk of pairs (each
  // zeroed on the stream before the kernel that counts it)
  unsigned long long* hs_nlist = nullptr;
  // launch order of the screen's tiles for 256- and 32-thread blocks, made
  // for plane width hs_order_w (see make_hs_order)
  uint32_t* hs_order[2] = {nullptr, nullptr};
  int64_t hs_order_w = 0;

  // tensor-core correlation (precision variant); corr_mode = FDAS_CORR_*
  int corr_mode = 0;
  int whiten_mode = 0;         // FDAS_WHITEN_*
  int hs_threads = 32;         // harmonic-sum block (32 or 256 threads)
  // half-bin planes: taps and spectra of 2Z template rows (row 2j + e at
  // frequency offset e/2); the plane and Q4 then have 2 nb columns
  int interbin = 0;
  double2* taps_ib = nullptr;
  float2* bank_ib = nullptr;
  int64_t plane_cap = 0;       // floats the plane buffer holds (Q4: plane_cap / 4)
  int64_t seg_cap = 0;         // float2 the segment buffer holds (>= S L)
  // candidate distillation: hash table of 2^dbits keys and values (on first use)
  unsigned long long* dkeys = nullptr;
  float* dvals = nullptr;
  int dbits = 0;
  uint16_t* gbank = nullptr;   // 16-bit left factor, pre-tiled (see fdas_gemm.cu)
  int* gstatus = nullptr;      // device status word of the bounded waits
  uint32_t gm_spin = 0;        // poll limit of its pipeline waits (0: the default, ~1 s)

  // host-input pipeline (more staging buffers, a second candidate list and
  // count, a copy stream and events; made on the first multi-trial host
  // call): staging slot k holds the series of trials t = k mod 4 (with the
  // trial lane; slots 0, 1 are the plan's and the lane's series buffers,
  // 2, 3 series3[0..1]) or t = k mod 2 (without it; slot 1 is series2)
  float* series2 = nullptr;
  float* series3[2] = {nullptr, nullptr};
  fdas_cand* cands2 = nullptr;
  unsigned long long* count2 = nullptr;
  // with the trial lane, two more candidate lists and counts (trial t writes
  // list t mod 4), so that the host reads trial t - 2 back while trials t - 1
  // and t run
  fdas_cand* cands3[2] = {nullptr, nullptr};
  unsigned long long* count3[2] = {nullptr, nullptr};
  cudaStream_t cstream = nullptr;
  cudaEvent_t ev_in[4] = {nullptr, nullptr, nullptr, nullptr};    // series copy landed in slot k
  cudaEvent_t ev_done[4] = {nullptr, nullptr, nullptr, nullptr};  // the trial reading slot k finished

  // second trial lane of multi-trial calls: a plan that shares this plan's
  // read-only tables and owns its own per-trial workspaces and stream, so
  // that trials t and t + 1 overlap on the GPU (made on first use); fork and
  // join events order it after and before this plan's stream
  fdas_plan* lane = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int64_t lane_key[5] = {0, 0, 0, 0, 0};  // N, Z, S * L, max_cands, plane width it was made for
  int64_t lane_gen = 0;                    // lanes made so far (a captured graph names its lane)
  bool last_on_lane = false;               // the last trial of this plan ran on the lane

  int64_t device_bytes = 0;
  int corr_ctas_per_sm = 0;  // launch shape of the correlation kernel (last launch)
  int corr_grid = 0;
};

namespace fdas {

// capacity of the harmonic-sum screen's list of flagged bin pairs
constexpr int64_t kHsListCap = (int64_t)1 << 20;

// plane columns: nb, or 2 nb (half bins) for half-bin planes
inline int64_t plane_width(const fdas_plan* p) { return p->nb << p->interbin; }

// NVTX range for the lifetime of a scope (host side: what the entry points
// enqueue); a no-op unless a profiler or tracer is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// error plumbing
int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);

// A caller's device pointer must be aligned for the vector accesses the
// kernels make through it (8 bytes where they read or write float2, 16 where
// float4, 8 for the 64-bit counters); checked before any device work, so a
// misaligned view (say a tensor sliced at an odd float) is an argument error
// rather than a misaligned-address fault.
inline int check_aligned(const void* ptr, uintptr_t bytes, const char* what) {
  if ((reinterpret_cast<uintptr_t>(ptr) & (bytes - 1)) == 0) return 0;
  return set_error(FDAS_ERR_INVALID, std::string(what) + " must be " + std::to_string(bytes) +
                                         "-byte aligned");
}

// fdas_templates.cu
int launch_twiddles(float2* out, int64_t count, int64_t mult, int64_t period, cudaStream_t s);
int launch_template_taps(fdas_plan* p);
int launch_template_bank(fdas_plan* p);
int launch_template_interbin(fdas_plan* p);
void fresnel_host(double x, double* C, double* S);

// fdas_spectrum.cu, fdas_spectrum_mixed.cu
int launch_spectrum(fdas_plan* p, const float* d_series, float2* d_spec);
int launch_unpack(fdas_plan* p, float2* d_spec);
int launch_spectrum_mixed(fdas_plan* p, const float* d_series, float2* d_spec);
bool is_235(int64_t x);
bool split_235(int64_t M, int* M1, int* M2);
int launch_whiten(fdas_plan* p, const float2* d_spec, float2* d_white);
int launch_whiten_block(fdas_plan* p, const float2* d_spec, float2* d_white);

// fdas_correlate.cu
int launch_segments(fdas_plan* p, const float2* d_white);
int launch_bank_natural(fdas_plan* p, float2* d_out);
int launch_correlate(fdas_plan* p, float* d_plane, float* d_q4, fdas_cand* d_cands,
                     unsigned long long* d_count);

// fdas_gemm.cu
size_t gemm_bank_elems(const fdas_plan* p);
int gemm_check_shape(const fdas_plan* p);
int launch_gemm_bank(fdas_plan* p);
int launch_gemm_correlate(fdas_plan* p, float* d_plane);

// fdas_distill.cu
int launch_distill(fdas_plan* p, const fdas_cand* d_cands, const int64_t* d_count,
                   fdas_peak* d_peaks, int64_t* d_npeaks);

// fdas_tune.cu
int launch_probe_noise(float* d_x, int64_t n, uint64_t seed, cudaStream_t s);

// fdas_harmsum.cu
int launch_pool4(fdas_plan* p, const float* d_plane, float* d_q4, fdas_cand* d_out,
                 unsigned long long* d_count);
int launch_harmsum(fdas_plan* p, const float* d_plane, const float* d_q4, fdas_cand* d_out,
                   unsigned long long* d_count);
int make_hs_order(fdas_plan* p);
void free_hs_order(fdas_plan* p);

}  // namespace fdas
