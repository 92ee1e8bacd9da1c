// Probe input for the autotuner: seeded Gaussian white noise generated on the
// device (splitmix64 of the sample index, Box-Muller), so that a batch can be
// tuned before any real series exists. Only its statistics matter: the
// harmonic-sum screening rate, and so the timing, depends on the whitened
// noise being Gaussian.
#include "fdas_internal.h"

namespace fdas {
namespace {

__global__ void k_probe_noise(float* __restrict__ x, int64_t n, uint64_t seed) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u1 = ((float)(z >> 40) + 0.5f) * (1.0f / 16777216.0f);
  const float u2 = ((float)(z & 0xFFFFFFull) + 0.5f) * (1.0f / 16777216.0f);
  x[i] = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

}  // namespace

int launch_probe_noise(float* d_x, int64_t n, uint64_t seed, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  k_probe_noise<<<(unsigned)blocks, 256, 0, s>>>(d_x, n, seed);
  return cuda_check(cudaGetLastError(), "k_probe_noise");
}

}  // namespace fdas
