// Correlation of Eq. 1 as a dense contraction on the 5th-generation tensor
// cores (tcgen05): the precision variant of steps 5-7 of Section 4.
//
// For a block of 512 consecutive Fourier bins r0..r0+511, Eq. 1 is
//   A[z][n] = sum_d tau_z(d) * X^[r0 + n + d],   d = -m/2 .. m/2-1,
// a (Z x m) x (m x 512) complex product whose right factor is a Hankel
// matrix (its entry depends on n + d only). In real arithmetic each template
// z gives two rows (Re A, Im A) over K = [Re X^; Im X^]; the float32 inputs
// are split into 16-bit hi + lo parts and the three products hi*hi, hi*lo and
// lo*hi are stacked along K, so one GEMM with K = 6m computes A to about 16
// (bf16) or 22 (fp16) bits:
//
//   K section   right factor   left factor (row 2z: Re A | row 2z+1: Im A)
//   0           Re X^_lo       Re t_hi | Im t_hi          (t = tau_z)
//   1           Im X^_lo      -Im t_hi | Re t_hi
//   2           Re X^_hi       Re t_lo | Im t_lo
//   3           Im X^_hi      -Im t_lo | Re t_lo
//   4           Re X^_hi       Re t_hi | Im t_hi
//   5           Im X^_hi      -Im t_hi | Re t_hi
//
// For fp16 the lo parts are stored scaled by s = 2^11 (so they stay normal
// numbers) and sections 4-5 carry t_hi * s: the accumulator holds s * A
// exactly and the epilogue multiplies the power by s^-2. bf16 has the range
// of float32 and uses s = 1.
//
// Tile: 128 rows of the left factor (64 templates, TMEM lanes) x 512 bins
// (TMEM columns, two N = 256 MMAs per K step), K streamed in blocks of 64.
// The left factor (the template bank, built once per plan from the float64
// taps) is stored pre-tiled in the no-swizzle K-major core-matrix layout, so
// one 16 KB bulk copy (cp.async.bulk) fills one pipeline stage. The Hankel
// factor is never materialised: for each part (Re/Im x hi/lo) shared memory
// holds W[j] = (x[j], ..., x[j+7]) as one 16-byte chunk per j, and the
// matrix descriptor with both core-matrix strides equal to 128 bytes
// (8 chunks) addresses row n, column d of the Hankel matrix at chunk n + d.
//
// Warp roles (192 threads, one CTA per SM, persistent over bin blocks):
//   warps 0-3  build W for upcoming bin blocks; drain the accumulator
//              (tcgen05.ld), form |A|^2 and store the plane rows
//   warp 4     producer: bulk copies of template-bank blocks
//   warp 5     issues tcgen05.mma (one thread) and the commits
// Every wait is bounded; a pipeline wait that gives up (after the plan's
// poll limit, 2^23 polls by default) sets the plan's status word and all
// roles leave their loops; the kernel still waits, with the full fixed bound
// and whatever the plan's limit, for the bulk copies it issued and the MMAs
// it committed, and frees TMEM, before it returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "fdas_internal.h"
#include "fdas_tmem.cuh"

namespace fdas {
namespace {

constexpr int kGmNT = 512;                     // bins per tile = TMEM columns
constexpr int kGmMT = 128;                     // left-factor rows per tile = TMEM lanes
constexpr int kGmKB = 64;                      // K per pipeline stage
constexpr int kGmStages = 8;
constexpr int kGmWBufs = 1;                    // Hankel buffers (the room goes to stages)
constexpr int kGmStageBytes = kGmMT * kGmKB * 2;  // 16 KB
constexpr int kGmThreads = 192;
constexpr uint32_t kGmSpin = 1u << 23;         // polls of one bounded wait (~1 s)
// (kGmSpin is the default pipeline limit and the fixed bound of the drains)

// K sections 0..5 read shared-memory parts 2, 3, 0, 1, 0, 1 (0 Re hi, 1 Im hi,
// 2 Re lo, 3 Im lo)

struct GemmLayout {
  uint32_t w_part, w_buf, w_off, bar_off, total;
};

__host__ __device__ inline GemmLayout gemm_layout(int m) {
  GemmLayout g;
  g.w_part = (uint32_t)(kGmNT + m) * 16u;
  g.w_buf = 4u * g.w_part;
  g.w_off = kGmStages * kGmStageBytes;
  g.bar_off = g.w_off + kGmWBufs * g.w_buf;
  g.total = g.bar_off + 256u;  // 2 x kGmStages + 5 barriers, TMEM slot, abort flag
  return g;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded pipeline wait for the phase of parity `parity` (at most `limit`
// polls); false when it gave up or another role already did (the abort word
// is then set).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* status,
                          uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63u) == 63u) {
      if (*abort) return false;
      __nanosleep(64);
    }
  }
  *abort = 1;
  atomicExch(status, FDAS_ERR_TIMEOUT);
  return false;
}

// Wait for a completion that arrives on its own (a bulk copy landing, a
// commit of MMAs already issued) before the CTA frees what it uses: the full
// fixed bound, not the plan's limit, and no early exit on abort.
__device__ void mbar_drain(uint32_t bar, uint32_t parity, int* status) {
  for (uint32_t i = 0; i < kGmSpin; ++i) {
    if (mbar_test(bar, parity)) return;
    if ((i & 63u) == 63u) __nanosleep(64);
  }
  atomicExch(status, FDAS_ERR_TIMEOUT);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between core matrices adjacent in K (lbo) and in M/N (sbo).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator, both operands bf16
// or both f16, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive columns of this thread's lane, twice (64 columns), one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
      "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]),
        "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]),
        "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
        "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]),
        "=r"(r[62]), "=r"(r[63])
      : "r"(taddr), "r"(taddr + 32u)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ element types
template <typename T>
struct Elt;

template <>
struct Elt<__nv_bfloat16> {
  static constexpr bool kBf16 = true;
  static constexpr float kScale = 1.f;
  __device__ static uint16_t bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  }
  __device__ static float value(uint16_t b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
  }
  __device__ static uint16_t bits_d(double x) { return __bfloat16_as_ushort(__double2bfloat16(x)); }
  __device__ static double value_d(uint16_t b) { return (double)value(b); }
};

template <>
struct Elt<__half> {
  static constexpr bool kBf16 = false;
  static constexpr float kScale = 2048.f;
  __device__ static uint16_t bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
  __device__ static float value(uint16_t b) { return __half2float(__ushort_as_half(b)); }
  __device__ static uint16_t bits_d(double x) { return __half_as_ushort(__double2half(x)); }
  __device__ static double value_d(uint16_t b) { return (double)value(b); }
};

// ---------------------------------------------------------------- the bank
// bank[mt][kb] = 128 x 64 block of the left factor, element (i, kk) at
// (i/8)*512 + (kk/8)*64 + (i%8)*8 + kk%8 (16-bit elements): core matrices of
// 8 rows x 16 bytes, K-adjacent ones 128 B apart, row groups 1024 B apart.
template <typename T>
__global__ void k_gemm_bank(const double2* __restrict__ taps, uint16_t* __restrict__ bank,
                            int Z, int m, int nKB) {
  using E = Elt<T>;
  const int tile = blockIdx.x;
  const int mt = tile / nKB, kb = tile % nKB;
  const double s = (double)E::kScale;
  for (int e = threadIdx.x; e < kGmMT * kGmKB; e += blockDim.x) {
    const int i = e / kGmKB, kk = e % kGmKB;
    const int row = mt * kGmMT + i;
    const int k = kb * kGmKB + kk;
    const int sec = k / m, d = k % m;
    uint16_t out = 0;
    if (row < 2 * Z) {
      const double2 t = taps[(size_t)(row >> 1) * m + d];
      const bool odd = row & 1;
      // X_re sections take Re t (row 2z) / Im t (row 2z+1); X_im sections
      // take -Im t / Re t.
      const double c = (sec % 2 == 0) ? (odd ? t.y : t.x) : (odd ? t.x : -t.y);
      const uint16_t hi = E::bits_d(c);
      if (sec < 2) {
        out = hi;
      } else if (sec < 4) {
        out = E::bits_d((c - E::value_d(hi)) * s);
      } else {
        out = E::bits_d(E::value_d(hi) * s);
      }
    }
    const size_t off = (size_t)tile * (kGmMT * kGmKB) + (i / 8) * 512 + (kk / 8) * 64 +
                       (i % 8) * 8 + (kk % 8);
    bank[off] = out;
  }
}

// ---------------------------------------------------------------- the GEMM
template <typename T>
__global__ void __launch_bounds__(kGmThreads, 1)
    k_gemm_correlate(const uint16_t* __restrict__ bank, const float2* __restrict__ white,
                     float* __restrict__ plane, int* __restrict__ status, int64_t nb, int Z,
                     int m, int nMT, int nKB, int nRT, uint32_t spin) {
  using E = Elt<T>;
  extern __shared__ __align__(1024) uint8_t smem[];
  const GemmLayout g = gemm_layout(m);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t a_base = sbase;
  const uint32_t w_base = sbase + g.w_off;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + g.bar_off);
  const uint32_t bar0 = smem_u32(bars);
  auto bar_full = [&](int s) { return bar0 + 8u * s; };
  auto bar_empty = [&](int s) { return bar0 + 8u * (kGmStages + s); };
  const uint32_t bar_tfull = bar0 + 8u * (2 * kGmStages);
  const uint32_t bar_tempty = bar_tfull + 8u;
  const uint32_t bar_wfull0 = bar_tfull + 16u;  // two: one per W buffer
  const uint32_t bar_done = bar_tfull + 32u;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + g.bar_off + 8 * (2 * kGmStages + 5));
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGmStages; ++s) {
      mbar_init(bar_full(s), 1);
      mbar_init(bar_empty(s), 1);
    }
    mbar_init(bar_tfull, 1);
    mbar_init(bar_tempty, 4);
    mbar_init(bar_wfull0, 4);
    mbar_init(bar_wfull0 + 8u, 4);
    mbar_init(bar_done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int my_tiles = nRT > (int)blockIdx.x ? (nRT - (int)blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (warp < 4) {
    // ---------------------------------------------- W builder + epilogue
    const int tid = threadIdx.x;
    auto build_w = [&](int q) {
      const int64_t r0 = (int64_t)(blockIdx.x + (int64_t)q * gridDim.x) * kGmNT;
      const int64_t base = r0 - m / 2;
      uint8_t* wp = smem + g.w_off + (size_t)(q % kGmWBufs) * g.w_buf;
      const int nch = kGmNT + m;
      for (int j = tid; j < nch; j += 128) {
        uint32_t p[4][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          float2 x[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int64_t idx = base + j + e + u;
            x[u] = (idx >= 0 && idx < nb) ? __ldg(white + idx) : make_float2(0.f, 0.f);
          }
          uint16_t h[4][2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            h[0][u] = E::bits(x[u].x);
            h[1][u] = E::bits(x[u].y);
            h[2][u] = E::bits((x[u].x - E::value(h[0][u])) * E::kScale);
            h[3][u] = E::bits((x[u].y - E::value(h[1][u])) * E::kScale);
          }
#pragma unroll
          for (int pt = 0; pt < 4; ++pt) p[pt][e >> 1] = (uint32_t)h[pt][0] | ((uint32_t)h[pt][1] << 16);
        }
#pragma unroll
        for (int pt = 0; pt < 4; ++pt)
          *reinterpret_cast<uint4*>(wp + (size_t)pt * g.w_part + (size_t)j * 16) =
              make_uint4(p[pt][0], p[pt][1], p[pt][2], p[pt][3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_wfull0 + 8u * (q % kGmWBufs));
    };

    for (int q = 0; q < kGmWBufs && q < my_tiles; ++q) build_w(q);
    const float pscale = 1.f / (E::kScale * E::kScale);
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t tile = 0;
    bool ok = true;
    for (int q = 0; q < my_tiles && ok; ++q) {
      const int64_t r0 = (int64_t)(blockIdx.x + (int64_t)q * gridDim.x) * kGmNT;
      for (int mt = 0; mt < nMT; ++mt, ++tile) {
        int got = 0;
        if (lane == 0) got = mbar_wait(bar_tfull, tile & 1u, abort, status, spin) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          ok = false;
          break;
        }
        tmem_fence_after_sync();
        const int row = mt * kGmMT + tid;
        const bool valid = row < 2 * Z;
        float* dst = plane + (size_t)(row >> 1) * nb + r0 + ((lane & 1) ? 32 : 0);
#pragma unroll 1
        for (int c = 0; c < kGmNT; c += 64) {
          float v[64];
          tmem_ld64(lane_addr + (uint32_t)c, v);
          float pw[64];
#pragma unroll
          for (int i = 0; i < 64; ++i) {
            const float o = __shfl_xor_sync(0xffffffffu, v[i], 1);
            pw[i] = (v[i] * v[i] + o * o) * pscale;
          }
          if (valid) {
            const bool odd = lane & 1;
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(dst + c + i) = make_float4(
                  odd ? pw[32 + i] : pw[i], odd ? pw[33 + i] : pw[i + 1],
                  odd ? pw[34 + i] : pw[i + 2], odd ? pw[35 + i] : pw[i + 3]);
          }
        }
        tmem_fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_tempty);
      }
      // the MMAs of bin block q are retired: its W buffer takes block q + kGmWBufs
      if (ok && q + kGmWBufs < my_tiles) build_w(q + kGmWBufs);
    }
  } else if (warp == 4) {
    // ---------------------------------------------- producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      const int per_block = nMT * nKB;
      for (int q = 0; q < my_tiles && ok; ++q)
        for (int b = 0; b < per_block; ++b, ++it) {
          const int s = it % kGmStages;
          if (it >= (uint32_t)kGmStages &&
              !mbar_wait(bar_empty(s), ((it / kGmStages) - 1) & 1u, abort, status, spin)) {
            ok = false;
            break;
          }
          mbar_expect_tx(bar_full(s), kGmStageBytes);
          bulk_g2s(a_base + (uint32_t)s * kGmStageBytes, bank + (size_t)b * (kGmMT * kGmKB),
                   kGmStageBytes, bar_full(s));
        }
      // copies still in flight land before the CTA may exit
      const uint32_t first = it > (uint32_t)kGmStages ? it - kGmStages : 0;
      for (uint32_t k = first; k < it; ++k)
        mbar_drain(bar_full(k % kGmStages), (k / kGmStages) & 1u, status);
    }
  } else {
    // ---------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(E::kBf16, kGmMT, 256);
      uint32_t it = 0, tile = 0;
      bool ok = true;
      // descriptors advance by adding to their start-address field (16-byte
      // units): the A stage by 16 per K step, the Hankel part by 1 per bin
      const uint64_t a_desc0 = sdesc(a_base, 128u, 1024u);
      for (int q = 0; q < my_tiles && ok; ++q) {
        const uint32_t wb = w_base + (uint32_t)(q % kGmWBufs) * g.w_buf;
        const uint64_t w_desc0 = sdesc(wb, 128u, 128u);  // part pt at + pt * w_part / 16
        if (!mbar_wait(bar_wfull0 + 8u * (q % kGmWBufs), (uint32_t)(q / kGmWBufs) & 1u, abort,
                       status, spin))
          break;
        for (int mt = 0; mt < nMT && ok; ++mt, ++tile) {
          if (tile > 0 && !mbar_wait(bar_tempty, (tile - 1) & 1u, abort, status, spin)) {
            ok = false;
            break;
          }
          tmem_fence_after_sync();
          int sec = 0, d0 = 0;  // K section and tap offset of the next K step
          for (int kb = 0; kb < nKB; ++kb, ++it) {
            const int s = it % kGmStages;
            if (!mbar_wait(bar_full(s), (it / kGmStages) & 1u, abort, status, spin)) {
              ok = false;
              break;
            }
            tmem_fence_after_sync();
            const uint64_t ad = a_desc0 + (uint64_t)((s * kGmStageBytes) >> 4);
#pragma unroll
            for (int i = 0; i < kGmKB / 16; ++i) {
              // sections 0, 1 read parts 2, 3 (lo); 2, 4 part 0; 3, 5 part 1
              const int pt = sec < 2 ? sec + 2 : (sec & 1);
              const uint64_t bd = w_desc0 + (uint64_t)(pt * (g.w_part >> 4) + d0);
              const uint32_t acc = (kb | i) != 0;
              umma(tmem, ad + 16u * i, bd, idesc, acc);
              umma(tmem + 256u, ad + 16u * i, bd + 256u, idesc, acc);
              d0 += 16;
              if (d0 == m) {
                d0 = 0;
                ++sec;
              }
            }
            umma_commit(bar_empty(s));
          }
          if (ok) umma_commit(bar_tfull);
        }
        if (!ok) break;
      }
      // every MMA issued above has retired once this commit lands
      umma_commit(bar_done);
      mbar_drain(bar_done, 0, status);
    }
  }
  tmem_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tmem_fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

template <typename T>
int gemm_bank(fdas_plan* p) {
  const int nMT = (2 * p->Z + kGmMT - 1) / kGmMT;
  const int nKB = 6 * p->m / kGmKB;
  k_gemm_bank<T><<<nMT * nKB, 256, 0, p->stream>>>(p->taps, p->gbank, p->Z, p->m, nKB);
  return cuda_check(cudaGetLastError(), "k_gemm_bank");
}

template <typename T>
int gemm_run(fdas_plan* p, float* d_plane) {
  const int nMT = (2 * p->Z + kGmMT - 1) / kGmMT;
  const int nKB = 6 * p->m / kGmKB;
  const int nRT = (int)(p->nb / kGmNT);
  const GemmLayout g = gemm_layout(p->m);
  static int attr_dev[2] = {-1, -1};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
  const int slot = Elt<T>::kBf16 ? 0 : 1;
  if (attr_dev[slot] != dev) {
    // the largest shared-memory size any template width may ask for
    e = cudaFuncSetAttribute(k_gemm_correlate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
    if (e != cudaSuccess) return cuda_check(e, "k_gemm_correlate attr");
    attr_dev[slot] = dev;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_check(e, "SM count");
  const int grid = std::min(sms, nRT);
  k_gemm_correlate<T><<<grid, kGmThreads, g.total, p->stream>>>(
      p->gbank, p->white, d_plane, p->gstatus, p->nb, p->Z, p->m, nMT, nKB, nRT,
      p->gm_spin ? p->gm_spin : kGmSpin);
  return cuda_check(cudaGetLastError(), "k_gemm_correlate");
}

}  // namespace

size_t gemm_bank_elems(const fdas_plan* p) {
  const int nMT = (2 * p->Z + kGmMT - 1) / kGmMT;
  return (size_t)nMT * (6 * p->m / kGmKB) * kGmMT * kGmKB;
}

int gemm_check_shape(const fdas_plan* p) {
  if (p->m % 32 != 0)
    return set_error(FDAS_ERR_INVALID, "the tensor-core correlation needs m % 32 == 0");
  if (p->nb % kGmNT != 0)
    return set_error(FDAS_ERR_INVALID, "the tensor-core correlation needs nb % 512 == 0");
  if (gemm_layout(p->m).total > 227u * 1024u)
    return set_error(FDAS_ERR_INVALID, "template width too large for the tensor-core correlation");
  return FDAS_OK;
}

int launch_gemm_bank(fdas_plan* p) {
  return p->corr_mode == FDAS_CORR_GEMM_FP16 ? gemm_bank<__half>(p)
                                             : gemm_bank<__nv_bfloat16>(p);
}

int launch_gemm_correlate(fdas_plan* p, float* d_plane) {
  return p->corr_mode == FDAS_CORR_GEMM_FP16 ? gemm_run<__half>(p, d_plane)
                                             : gemm_run<__nv_bfloat16>(p, d_plane);
}

}  // namespace fdas
