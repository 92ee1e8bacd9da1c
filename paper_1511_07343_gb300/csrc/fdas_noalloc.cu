// Plan-free real FFT whose scratch is a fixed, file-scope device array.
//
// Some callers cannot allocate device memory: a real-time processing loop
// that must keep a fixed device footprint once it is running, or a host
// framework that owns the device allocator and forbids other code from
// calling cudaMalloc. Such callers cannot create a plan, because
// fdas_plan_create allocates its workspaces. fdas_spectrum_noalloc runs the
// same real-FFT kernels as fdas_stage_spectrum, but keeps the four-step
// intermediate, the packed transform and the twiddle tables in the static
// array below, which exists on every GPU that loads this library until the
// process exits. Nothing here calls cudaMalloc, cudaFree or any allocating
// routine.
#include <atomic>

#include "fdas_internal.h"

namespace fdas {
namespace {

constexpr int64_t kNoallocMaxN = int64_t(1) << 20;  // samples per call, at most
constexpr int64_t kMaxM = kNoallocMaxN / 2;         // packed complex points
constexpr int64_t kMaxTab = 1 << 11;                // entries per twiddle table
// float2 slots: four-step intermediate + packed transform + 6 twiddle tables
constexpr int64_t kScratchSlots = 2 * kMaxM + 6 * (kMaxTab + 1);

static __device__ __align__(256) float2 g_noalloc_scratch[kScratchSlots];

// Device address of the array, looked up once per device (the first call on
// a device does this, with that device current). Host threads that make
// their first calls at the same time may each look it up; they store the
// same address, and the atomic slots make that well defined. The address
// belongs to the device's context at the time of the lookup: after
// cudaDeviceReset the module is loaded again, possibly elsewhere, so a
// process that resets a device must not call this entry point on it again.
constexpr int kMaxDevices = 64;
std::atomic<float2*> g_scratch_ptr[kMaxDevices];

int scratch_for_current_device(float2** out) {
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices) return set_error(FDAS_ERR_INVALID, "device ordinal too large");
  float2* cached = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!cached) {
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    if (rc) return rc;
    cached = static_cast<float2*>(p);
    g_scratch_ptr[dev].store(cached, std::memory_order_release);
  }
  *out = cached;
  return FDAS_OK;
}

int log2i64(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}

}  // namespace
}  // namespace fdas

using namespace fdas;

extern "C" int fdas_spectrum_noalloc(const float* d_series, int64_t N, float* d_spectrum,
                                     void* stream) {
  if (!d_series || !d_spectrum) return set_error(FDAS_ERR_INVALID, "NULL argument");
  // the kernels read the series and write the spectrum as float2
  if (int e = check_aligned(d_series, 8, "d_series")) return e;
  if (int e = check_aligned(d_spectrum, 8, "d_spectrum")) return e;
  if (N < (1 << 12) || N > kNoallocMaxN || (N & (N - 1)) != 0)
    return set_error(FDAS_ERR_INVALID,
                     "fdas_spectrum_noalloc: N must be a power of two in [2^12, 2^20]; larger "
                     "series need a plan (fdas_plan_create + fdas_stage_spectrum)");
  float2* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  // A plan-shaped view of the static array (host stack object, no allocation).
  fdas_plan v;
  v.N = N;
  v.nb = N / 2;
  v.M = N / 2;
  const int h = log2i64(v.M);
  v.M1 = 1 << ((h + 1) / 2);
  v.M2 = 1 << (h / 2);
  v.h4 = (h + 1) / 2;
  v.hN = (h + 1) / 2;
  v.stream = (cudaStream_t)stream;
  float2* q = base;
  v.zbuf = q;
  q += kMaxM;
  v.spec2 = q;
  q += kMaxM;
  v.tw_M1 = q;
  q += kMaxTab + 1;
  v.tw_M2 = q;
  q += kMaxTab + 1;
  v.tw4_lo = q;
  q += kMaxTab + 1;
  v.tw4_hi = q;
  q += kMaxTab + 1;
  v.twN_lo = q;
  q += kMaxTab + 1;
  v.twN_hi = q;
  // twiddle tables for this N (float64-made), written before every use: the
  // array keeps whatever the previous call left there
  cudaStream_t s = v.stream;
  if ((rc = launch_twiddles(v.tw_M1, v.M1, 1, v.M1, s))) return rc;
  if ((rc = launch_twiddles(v.tw_M2, v.M2, 1, v.M2, s))) return rc;
  if ((rc = launch_twiddles(v.tw4_lo, (int64_t)1 << v.h4, 1, v.M, s))) return rc;
  if ((rc = launch_twiddles(v.tw4_hi, (v.M >> v.h4) + 1, (int64_t)1 << v.h4, v.M, s))) return rc;
  if ((rc = launch_twiddles(v.twN_lo, (int64_t)1 << v.hN, 1, v.N, s))) return rc;
  if ((rc = launch_twiddles(v.twN_hi, (v.M >> v.hN) + 1, (int64_t)1 << v.hN, v.N, s))) return rc;
  return launch_spectrum(&v, d_series, reinterpret_cast<float2*>(d_spectrum));
}
