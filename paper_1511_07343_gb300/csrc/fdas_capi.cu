// C ABI of the FDAS library: plan lifetime, the search entry points and the
// per-stage hooks. Host logic only; every arithmetic step of the path runs in
// the kernels of the other translation units.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fdas_internal.h"

namespace fdas {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FDAS_OK;
  return set_error(e == cudaErrorMemoryAllocation ? FDAS_ERR_NOMEM : FDAS_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int log2i(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}

// Upper tail of Gamma(h, 1) for integer h: Q(h, x) = exp(-x) sum_{i<h} x^i / i!.
double gamma_q_int(int h, double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < h; ++i) {
    term *= x / i;
    sum += term;
  }
  return exp(-x) * sum;
}

// T with Q(h, T) = p: bisection on log Q (monotone), then Newton polish.
double gamma_q_inv_int(int h, double p) {
  double lo = 0.0, hi = 1.0;
  while (gamma_q_int(h, hi) > p) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (gamma_q_int(h, mid) > p) lo = mid; else hi = mid;
  }
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 3; ++it) {
    double lf = 1.0;
    for (int i = 1; i < h; ++i) lf *= i;
    const double dq = -exp(-x) * pow(x, h - 1) / lf;  // dQ/dx
    const double f = log(gamma_q_int(h, x)) - log(p);
    const double df = dq / gamma_q_int(h, x);
    if (df != 0.0) x -= f / df;
  }
  return x;
}

template <typename T>
int dalloc(fdas_plan* p, T** ptr, size_t count) {
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // a refused allocation must not surface at a later launch check
    *ptr = nullptr;
    return set_error(FDAS_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                         cudaGetErrorString(e));
  }
  p->device_bytes += (int64_t)bytes;
  return FDAS_OK;
}

void free_lane(fdas_plan* p);

void free_plan(fdas_plan* p) {
  if (!p) return;
  free_lane(p);
  for (int k = 0; k < 4; ++k) {
    if (p->ev_in[k]) cudaEventDestroy(p->ev_in[k]);
    if (p->ev_done[k]) cudaEventDestroy(p->ev_done[k]);
  }
  if (p->cstream) cudaStreamDestroy(p->cstream);
  if (p->series2) cudaFree(p->series2);
  for (float* b : p->series3)
    if (b) cudaFree(b);
  if (p->cands2) cudaFree(p->cands2);
  if (p->count2) cudaFree(p->count2);
  for (int e = 0; e < 2; ++e) {
    if (p->cands3[e]) cudaFree(p->cands3[e]);
    if (p->count3[e]) cudaFree(p->count3[e]);
  }
  void* ptrs[] = {p->tw_L, p->tw_M1, p->tw_M2, p->tw4_lo, p->tw4_hi, p->twN_lo, p->twN_hi,
                  p->taps, p->bank, p->series, p->zbuf, p->spec, p->spec2, p->white, p->seg,
                  p->plane, p->q4, p->cands, p->count, p->hs_list, p->hs_nlist,
                  p->hs_order[0], p->hs_order[1], p->gbank, p->gstatus,
                  p->dkeys, p->dvals, p->taps_ib, p->bank_ib};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p;
}

int launch_plane(fdas_plan* p, float* d_plane, float* d_q4, fdas_cand* d_out,
                 unsigned long long* d_count);

// The path for one trial; the plane goes to p->plane, candidates to d_out.
int run_trial(fdas_plan* p, const float* d_x, fdas_cand* d_out, unsigned long long* d_count) {
  NvtxRange range("fdas trial");
  int rc;
  p->last_on_lane = false;
  if ((rc = cuda_check(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), p->stream),
                       "memset count")))
    return rc;
  if ((rc = launch_spectrum(p, d_x, p->spec))) return rc;
  if ((rc = launch_whiten(p, p->spec, p->white))) return rc;
  if ((rc = launch_plane(p, p->plane, p->q4, d_out, d_count))) return rc;
  return launch_harmsum(p, p->plane, p->q4, d_out, d_count);
}

// Steps 3-7 for the plan's correlation mode: the plane, its 4-bin maxima and
// the h = 1 candidates (when d_q4 is given).
int launch_plane(fdas_plan* p, float* d_plane, float* d_q4, fdas_cand* d_out,
                 unsigned long long* d_count) {
  int rc;
  if (p->corr_mode == FDAS_CORR_FFT) {
    if ((rc = launch_segments(p, p->white))) return rc;
    if ((rc = launch_correlate(p, d_plane, d_q4, d_out, d_count))) return rc;
    // half-bin planes: maxima and h = 1 candidates of the interleaved plane
    return p->interbin && d_q4 ? launch_pool4(p, d_plane, d_q4, d_out, d_count) : FDAS_OK;
  }
  if ((rc = launch_gemm_correlate(p, d_plane))) return rc;
  return d_q4 ? launch_pool4(p, d_plane, d_q4, d_out, d_count) : FDAS_OK;
}

// Status word of the tensor-core kernel's bounded waits (0 when none gave up).
int gemm_status(fdas_plan* p) {
  if (p->corr_mode == FDAS_CORR_FFT) return FDAS_OK;
  int st = 0;
  int rc = cuda_check(cudaMemcpyAsync(&st, p->gstatus, sizeof(int), cudaMemcpyDeviceToHost,
                                      p->stream), "copy status");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(p->stream), "sync status");
  if (rc) return rc;
  if (st) {
    cudaMemsetAsync(p->gstatus, 0, sizeof(int), p->stream);
    return set_error(FDAS_ERR_TIMEOUT, "a bounded wait of the tensor-core correlation gave up");
  }
  return FDAS_OK;
}

// N-dependent geometry of a plan: spectrum length, four-step split and the
// segment count. N = 2^a 3^b 5^c with a >= 12 (the power-of-two path splits
// M = N/2 into equal powers of two; other lengths use a balanced 2-3-5 split).
int set_geometry(fdas_plan* p, int64_t N) {
  if (N < (1 << 12) || N > (1 << 24) || N % 4096 != 0 || !is_235(N))
    return set_error(FDAS_ERR_INVALID,
                     "N must be 2^a 3^b 5^c with a >= 12 and 2^12 <= N <= 2^24");
  p->N = N;
  p->nb = N / 2;
  p->M = N / 2;
  const int h = log2i(p->M);
  if (is_pow2(N)) {
    p->M1 = 1 << ((h + 1) / 2);
    p->M2 = 1 << (h / 2);
  } else if (!split_235(p->M, &p->M1, &p->M2)) {
    return set_error(FDAS_ERR_INVALID, "N has no supported four-step split");
  }
  p->h4 = (h + 1) / 2;
  p->hN = (h + 1) / 2;
  p->S = (int)((p->nb + p->V - 1) / p->V);
  return FDAS_OK;
}

// the six N-dependent twiddle tables (float64-made) of the real FFT
int alloc_geometry_tables(fdas_plan* p) {
  int rc;
  if ((rc = dalloc(p, &p->tw_M1, p->M1))) return rc;
  if ((rc = dalloc(p, &p->tw_M2, p->M2))) return rc;
  if ((rc = dalloc(p, &p->tw4_lo, (size_t)1 << p->h4))) return rc;
  if ((rc = dalloc(p, &p->tw4_hi, (size_t)(p->M >> p->h4) + 1))) return rc;
  if ((rc = dalloc(p, &p->twN_lo, (size_t)1 << p->hN))) return rc;
  if ((rc = dalloc(p, &p->twN_hi, (size_t)(p->M >> p->hN) + 1))) return rc;
  cudaStream_t s = p->stream;
  if ((rc = launch_twiddles(p->tw_M1, p->M1, 1, p->M1, s))) return rc;
  if ((rc = launch_twiddles(p->tw_M2, p->M2, 1, p->M2, s))) return rc;
  if ((rc = launch_twiddles(p->tw4_lo, (int64_t)1 << p->h4, 1, p->M, s))) return rc;
  if ((rc = launch_twiddles(p->tw4_hi, (p->M >> p->h4) + 1, (int64_t)1 << p->h4, p->M, s)))
    return rc;
  if ((rc = launch_twiddles(p->twN_lo, (int64_t)1 << p->hN, 1, p->N, s))) return rc;
  return launch_twiddles(p->twN_hi, (p->M >> p->hN) + 1, (int64_t)1 << p->hN, p->N, s);
}

void free_geometry_tables(fdas_plan* p) {
  void* ptrs[] = {p->tw_M1, p->tw_M2, p->tw4_lo, p->tw4_hi, p->twN_lo, p->twN_hi};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->tw_M1 = p->tw_M2 = p->tw4_lo = p->tw4_hi = p->twN_lo = p->twN_hi = nullptr;
}

bool cand_less(const fdas_cand& a, const fdas_cand& b) {
  if (a.h != b.h) return a.h < b.h;
  if (a.r_top != b.r_top) return a.r_top < b.r_top;
  return a.z_idx < b.z_idx;
}

// ---------------------------------------------------------------------------
// Second trial lane (multi-trial calls of the FFT correlation on integer-bin
// planes). The lane is a copy of the plan whose per-trial workspaces, stream
// and candidate list are its own; the templates, twiddle and tile-order
// tables are the plan's (read-only during a search).
// ---------------------------------------------------------------------------
bool lanes_usable(const fdas_plan* p) {
  return p->stream != nullptr && p->corr_mode == FDAS_CORR_FFT && !p->interbin;
}

void free_lane(fdas_plan* p) {
  fdas_plan* l = p->lane;
  if (!l) return;
  if (l->stream) {
    cudaStreamSynchronize(l->stream);
    cudaStreamDestroy(l->stream);
  }
  void* ptrs[] = {l->series, l->zbuf, l->spec, l->spec2, l->white, l->seg, l->plane,
                  l->q4, l->cands, l->count, l->hs_list, l->hs_nlist};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  p->ev_fork = p->ev_join = nullptr;
  p->device_bytes -= l->device_bytes;
  delete l;
  p->lane = nullptr;
}

// The lane for the plan's current shape, made or remade as needed, with the
// plan's shared fields copied in. Its plane, 4-bin maxima and segment buffers
// have the plan's capacities (a batch with several zmax classes sizes those
// for its largest class).
int ensure_lane(fdas_plan* p) {
  const int64_t key[5] = {p->N, p->plane_cap, p->seg_cap, p->max_cands, plane_width(p)};
  if (p->lane && !std::equal(key, key + 5, p->lane_key)) free_lane(p);
  if (!p->lane) {
    fdas_plan* l = new fdas_plan(*p);
    // nothing the plan owns may be freed through the lane
    l->series = nullptr; l->zbuf = nullptr; l->spec = nullptr; l->spec2 = nullptr;
    l->white = nullptr; l->seg = nullptr; l->plane = nullptr; l->q4 = nullptr;
    l->cands = nullptr; l->count = nullptr; l->hs_list = nullptr; l->hs_nlist = nullptr;
    l->stream = nullptr; l->lane = nullptr; l->device_bytes = 0;
    p->lane = l;
    int rc = 0;
    if (!rc) rc = dalloc(l, &l->series, (size_t)p->N);
    if (!rc) rc = dalloc(l, &l->zbuf, (size_t)p->M);
    if (!rc) rc = dalloc(l, &l->spec, (size_t)p->nb);
    if (!rc) rc = dalloc(l, &l->spec2, (size_t)p->M);
    if (!rc) rc = dalloc(l, &l->white, (size_t)p->nb);
    if (!rc) rc = dalloc(l, &l->seg, (size_t)p->seg_cap);
    if (!rc) rc = dalloc(l, &l->plane, (size_t)p->plane_cap);
    if (!rc) rc = dalloc(l, &l->q4, (size_t)p->plane_cap / 4);
    if (!rc) rc = dalloc(l, &l->cands, (size_t)p->max_cands);
    if (!rc) rc = dalloc(l, &l->count, 1);
    if (!rc) rc = dalloc(l, &l->hs_list, (size_t)kHsListCap);
    if (!rc) rc = dalloc(l, &l->hs_nlist, 2);
    if (!rc)
      rc = cuda_check(cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking), "lane stream");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming), "event");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming), "event");
    p->device_bytes += l->device_bytes;
    if (rc) {
      free_lane(p);
      return rc;
    }
    std::copy(key, key + 5, p->lane_key);
    ++p->lane_gen;
  }
  // shared fields (modes, tables, templates) as the plan has them now
  fdas_plan* l = p->lane;
  fdas_plan own = *l;
  *l = *p;
  l->series = own.series; l->zbuf = own.zbuf; l->spec = own.spec; l->spec2 = own.spec2;
  l->white = own.white; l->seg = own.seg; l->plane = own.plane; l->q4 = own.q4;
  l->plane_cap = p->plane_cap;
  l->seg_cap = p->seg_cap;
  l->cands = own.cands; l->count = own.count; l->hs_list = own.hs_list;
  l->hs_nlist = own.hs_nlist; l->stream = own.stream; l->device_bytes = own.device_bytes;
  l->series2 = nullptr; l->cands2 = nullptr; l->count2 = nullptr; l->cstream = nullptr;
  l->series3[0] = l->series3[1] = nullptr;
  l->cands3[0] = l->cands3[1] = nullptr;
  l->count3[0] = l->count3[1] = nullptr;
  for (int k = 0; k < 4; ++k) l->ev_in[k] = l->ev_done[k] = nullptr;
  l->lane = nullptr; l->ev_fork = l->ev_join = nullptr;
  l->dkeys = nullptr; l->dvals = nullptr; l->dbits = 0;
  return FDAS_OK;
}

int search_impl(fdas_plan* p, const float* d_series, int32_t n_trials, fdas_cand* h_out,
                int64_t* h_counts) {
  bool overflow = false;
  for (int32_t t = 0; t < n_trials; ++t) {
    int rc = run_trial(p, d_series + (size_t)t * p->N, p->cands, p->count);
    if (rc) return rc;
    unsigned long long cnt = 0;
    rc = cuda_check(cudaMemcpyAsync(&cnt, p->count, sizeof(cnt), cudaMemcpyDeviceToHost,
                                    p->stream),
                    "copy count");
    if (rc) return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(p->stream), "sync count"))) return rc;
    if ((rc = gemm_status(p))) return rc;
    h_counts[t] = (int64_t)cnt;
    const int64_t keep = std::min<int64_t>((int64_t)cnt, p->max_cands);
    if ((int64_t)cnt > p->max_cands) overflow = true;
    fdas_cand* dst = h_out + (size_t)t * p->max_cands;
    if (keep > 0) {
      rc = cuda_check(cudaMemcpyAsync(dst, p->cands, sizeof(fdas_cand) * keep,
                                      cudaMemcpyDeviceToHost, p->stream),
                      "copy candidates");
      if (rc) return rc;
      if ((rc = cuda_check(cudaStreamSynchronize(p->stream), "sync candidates"))) return rc;
      std::sort(dst, dst + keep, cand_less);
    }
  }
  return overflow ? set_error(FDAS_ERR_OVERFLOW, "candidate list overflow") : FDAS_OK;
}

// Several host series through one plan with the copies overlapped: while
// trial t runs on the plan stream, the copy stream brings in series t+1
// (into the other staging buffer, once trial t-1 has finished reading it)
// and the host reads back and sorts the candidates of trial t-1 (from the
// other candidate buffer). Page-locked host memory makes the copies overlap.
// (d_series != nullptr: the series are already on the device, nothing is
// copied in and only the read-back overlaps)
int host_pipeline(fdas_plan* p, const float* h_series, int32_t n_trials, fdas_cand* h_out,
                  int64_t* h_counts, const float* d_series = nullptr) {
  int rc = FDAS_OK;
  if (!p->cstream) {
    if ((rc = cuda_check(cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking),
                         "copy stream")))
      return rc;
    for (int k = 0; k < 4 && !rc; ++k) {
      rc = cuda_check(cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming), "event");
      if (!rc)
        rc = cuda_check(cudaEventCreateWithFlags(&p->ev_done[k], cudaEventDisableTiming), "event");
    }
    if (rc) return rc;
  }
  // trial t runs on lane t % 2: the plan itself, then the second lane (its
  // own workspaces and stream) where usable, else the plan again with a
  // second staging buffer and candidate list of its own
  fdas_plan* q[2] = {p, p};
  if (lanes_usable(p)) {
    if ((rc = ensure_lane(p))) return rc;
    q[1] = p->lane;
  } else if (!p->series2 || !p->cands2 || !p->count2) {
    if (!p->series2 && (rc = dalloc(p, &p->series2, (size_t)p->N))) return rc;
    if (!p->cands2 && (rc = dalloc(p, &p->cands2, (size_t)p->max_cands))) return rc;
    if (!p->count2 && (rc = dalloc(p, &p->count2, 1))) return rc;
  }
  const bool lanes = q[1] != p;
  // staging slots: with two lanes, 4, so that the copy of trial t + 1 waits
  // for trial t - 3 (long done) rather than for trial t - 1 of its lane
  const int K = lanes ? 4 : 2;
  if (lanes && !d_series)
    for (int e = 0; e < 2; ++e)
      if (!p->series3[e] && (rc = dalloc(p, &p->series3[e], (size_t)p->N))) return rc;
  if (lanes)
    for (int e = 0; e < 2; ++e) {
      if (!p->cands3[e] && (rc = dalloc(p, &p->cands3[e], (size_t)p->max_cands))) return rc;
      if (!p->count3[e] && (rc = dalloc(p, &p->count3[e], 1))) return rc;
    }
  float* buf[4] = {p->series, lanes ? q[1]->series : p->series2, p->series3[0], p->series3[1]};
  // candidate list of trial t: cbuf[t % K] (with lanes, t mod 4: the read-back
  // of trial t - 2 overlaps trials t - 1 and t; without, t mod 2)
  fdas_cand* cbuf[4] = {p->cands, lanes ? q[1]->cands : p->cands2, p->cands3[0], p->cands3[1]};
  unsigned long long* nbuf[4] = {p->count, lanes ? q[1]->count : p->count2, p->count3[0],
                                 p->count3[1]};
  const int D = lanes ? 2 : 1;  // trials enqueued ahead of the one read back
  if (lanes) {  // the lane starts after the caller's work on the plan stream
    rc = cuda_check(cudaEventRecord(p->ev_fork, p->stream), "event");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(q[1]->stream, p->ev_fork, 0), "wait");
    if (rc) return rc;
  }
  const size_t bytes = sizeof(float) * (size_t)p->N;
  bool overflow = false;
  // read back and sort trial t (its kernels are done once ev_done fires)
  auto finish = [&](int32_t t) -> int {
    const int b = t % K;
    int r = cuda_check(cudaEventSynchronize(p->ev_done[t % K]), "trial done");
    unsigned long long cnt = 0;
    if (!r)
      r = cuda_check(cudaMemcpyAsync(&cnt, nbuf[b], sizeof(cnt), cudaMemcpyDeviceToHost, p->cstream),
                     "copy count");
    if (!r) r = cuda_check(cudaStreamSynchronize(p->cstream), "sync count");
    if (r) return r;
    h_counts[t] = (int64_t)cnt;
    const int64_t keep = std::min<int64_t>((int64_t)cnt, p->max_cands);
    if ((int64_t)cnt > p->max_cands) overflow = true;
    fdas_cand* dst = h_out + (size_t)t * p->max_cands;
    if (keep > 0) {
      r = cuda_check(cudaMemcpyAsync(dst, cbuf[b], sizeof(fdas_cand) * keep,
                                     cudaMemcpyDeviceToHost, p->cstream),
                     "copy candidates");
      if (!r) r = cuda_check(cudaStreamSynchronize(p->cstream), "sync candidates");
      if (r) return r;
      std::sort(dst, dst + keep, cand_less);
    }
    return FDAS_OK;
  };
  if (!d_series) {
    rc = cuda_check(cudaMemcpyAsync(buf[0], h_series, bytes, cudaMemcpyHostToDevice, p->cstream),
                    "copy series");
    if (!rc) rc = cuda_check(cudaEventRecord(p->ev_in[0], p->cstream), "event");
  }
  for (int32_t t = 0; t < n_trials && !rc; ++t) {
    const int b = t & 1, k = t % K;
    if (d_series) {
      rc = run_trial(q[b], d_series + (size_t)t * p->N, cbuf[k], nbuf[k]);
      if (!rc) rc = cuda_check(cudaEventRecord(p->ev_done[k], q[b]->stream), "event");
      if (!rc && t >= D) rc = finish(t - D);
      continue;
    }
    if (t + 1 < n_trials) {
      // staging slot k1 was last read by trial t + 1 - K
      const int k1 = (t + 1) % K;
      if (t + 1 >= K) rc = cuda_check(cudaStreamWaitEvent(p->cstream, p->ev_done[k1], 0), "wait");
      if (!rc)
        rc = cuda_check(cudaMemcpyAsync(buf[k1], h_series + (size_t)(t + 1) * p->N, bytes,
                                        cudaMemcpyHostToDevice, p->cstream),
                        "copy series");
      if (!rc) rc = cuda_check(cudaEventRecord(p->ev_in[k1], p->cstream), "event");
    }
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(q[b]->stream, p->ev_in[k], 0), "wait");
    if (!rc) rc = run_trial(q[b], buf[k], cbuf[k], nbuf[k]);
    if (!rc) rc = cuda_check(cudaEventRecord(p->ev_done[k], q[b]->stream), "event");
    // the host reads back trial t - D while the trials after it run; the
    // next trial to use its candidate list is enqueued only after this returns
    if (!rc && t >= D) rc = finish(t - D);
  }
  for (int32_t t = std::max(0, n_trials - D); t < n_trials && !rc; ++t) rc = finish(t);
  if (!rc && lanes) {  // the plan stream continues after the lane's work
    rc = cuda_check(cudaEventRecord(p->ev_join, q[1]->stream), "event");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(p->stream, p->ev_join, 0), "wait");
    p->last_on_lane = n_trials >= 2 && ((n_trials - 1) & 1);
  }
  if (!rc) rc = gemm_status(p);
  if (rc) {
    cudaStreamSynchronize(p->cstream);
    cudaStreamSynchronize(p->stream);
    if (lanes) cudaStreamSynchronize(q[1]->stream);
    return rc;
  }
  return overflow ? set_error(FDAS_ERR_OVERFLOW, "candidate list overflow") : FDAS_OK;
}

}  // namespace
}  // namespace fdas

using namespace fdas;

extern "C" {

int fdas_plan_create(fdas_plan** out, int64_t N, int32_t zmax, int32_t dz, int32_t m,
                     int32_t L, int32_t nharm, float sigma, int64_t max_cands, void* stream) {
  NvtxRange range("fdas_plan_create");
  if (!out) return set_error(FDAS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (zmax < 0 || dz <= 0 || zmax % dz != 0)
    return set_error(FDAS_ERR_INVALID, "need zmax >= 0, dz > 0 and dz | zmax");
  if (m < 8 || (m & 7)) return set_error(FDAS_ERR_INVALID, "template width must be a multiple of 8");
  if (L != 2048 && L != 4096 && L != 8192)
    return set_error(FDAS_ERR_INVALID, "segment length must be 2048, 4096 or 8192");
  if (L < 2 * m) return set_error(FDAS_ERR_INVALID, "segment length must be >= 2 * width");
  if (nharm != 1 && nharm != 2 && nharm != 4 && nharm != 8 && nharm != 16)
    return set_error(FDAS_ERR_INVALID, "nharm must be 1, 2, 4, 8 or 16");
  if (!(sigma > 0.f)) return set_error(FDAS_ERR_INVALID, "sigma must be > 0");
  if (max_cands < 1) return set_error(FDAS_ERR_INVALID, "max_cands must be >= 1");
  if (N < 0 || (int64_t)(2 * (zmax / dz) + 1) * (N / 2) > (int64_t(1) << 40))
    return set_error(FDAS_ERR_INVALID, "plane too large");

  fdas_plan* p = new fdas_plan();
  p->zmax = zmax;
  p->dz = dz;
  p->Z = 2 * (zmax / dz) + 1;
  p->m = m;
  p->L = L;
  p->V = L - m;
  p->nharm = nharm;
  p->n_levels = log2i(nharm) + 1;
  p->sigma = sigma;
  p->max_cands = max_cands;
  p->stream = (cudaStream_t)stream;
  {
    const int grc = set_geometry(p, N);
    if (grc) {
      delete p;
      return grc;
    }
  }
  const double ptail = 0.5 * erfc((double)sigma / sqrt(2.0));
  for (int i = 0; i < p->n_levels; ++i) p->thr[i] = (float)gamma_q_inv_int(1 << i, ptail);

  int rc = FDAS_OK;
#define TRY(x)            \
  do {                    \
    if ((rc = (x))) {     \
      free_plan(p);       \
      return rc;          \
    }                     \
  } while (0)
  TRY(dalloc(p, &p->tw_L, L));
  TRY(alloc_geometry_tables(p));
  TRY(dalloc(p, &p->taps, (size_t)p->Z * m));
  TRY(dalloc(p, &p->bank, (size_t)p->Z * L));
  TRY(dalloc(p, &p->series, (size_t)N));
  TRY(dalloc(p, &p->zbuf, (size_t)p->M));
  TRY(dalloc(p, &p->spec, (size_t)p->nb));
  TRY(dalloc(p, &p->spec2, (size_t)p->M));
  TRY(dalloc(p, &p->white, (size_t)p->nb));
  TRY(dalloc(p, &p->seg, (size_t)p->S * L));
  p->seg_cap = (int64_t)p->S * L;
  TRY(dalloc(p, &p->plane, (size_t)p->Z * p->nb));
  TRY(dalloc(p, &p->q4, (size_t)p->Z * (p->nb / 4)));
  p->plane_cap = (int64_t)p->Z * p->nb;
  TRY(dalloc(p, &p->cands, (size_t)max_cands));
  TRY(dalloc(p, &p->count, 1));
  TRY(dalloc(p, &p->hs_list, (size_t)fdas::kHsListCap));
  TRY(dalloc(p, &p->hs_nlist, 2));
  TRY(make_hs_order(p));

  cudaStream_t s = p->stream;
  TRY(launch_twiddles(p->tw_L, L, 1, L, s));
  TRY(launch_template_taps(p));
  TRY(launch_template_bank(p));
  TRY(cuda_check(cudaStreamSynchronize(s), "plan initialisation"));
#undef TRY
  *out = p;
  return FDAS_OK;
}

int fdas_plan_destroy(fdas_plan* p) {
  if (!p) return FDAS_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  free_plan(p);
  return FDAS_OK;
}

int fdas_plan_get_info(const fdas_plan* p, fdas_plan_info* info) {
  if (!p || !info) return set_error(FDAS_ERR_INVALID, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->N = p->N;
  info->nb = p->nb;
  info->zmax = p->zmax;
  info->dz = p->dz;
  info->Z = p->Z;
  info->m = p->m;
  info->L = p->L;
  info->V = p->V;
  info->S = p->S;
  info->nharm = p->nharm;
  info->n_levels = p->n_levels;
  for (int i = 0; i < 5; ++i) info->thresholds[i] = p->thr[i];
  info->max_cands = p->max_cands;
  info->device_bytes = p->device_bytes;
  info->plane_floats = (int64_t)p->Z * plane_width(p);
  info->corr_ctas_per_sm = p->corr_ctas_per_sm;
  info->corr_grid = p->corr_grid;
  return FDAS_OK;
}

int fdas_search(fdas_plan* p, const float* d_series, int32_t n_trials, fdas_cand* h_out,
                int64_t* h_counts) {
  NvtxRange range("fdas_search");
  if (!p || !d_series || n_trials < 0 || (n_trials > 0 && (!h_out || !h_counts)))
    return set_error(FDAS_ERR_INVALID, "bad argument to fdas_search");
  if (int rc = check_aligned(d_series, 8, "d_series")) return rc;
  if (n_trials > 1 && p->stream != nullptr)  // read-back of trial t-1 overlaps trial t
    return host_pipeline(p, nullptr, n_trials, h_out, h_counts, d_series);
  return search_impl(p, d_series, n_trials, h_out, h_counts);
}

int fdas_search_host(fdas_plan* p, const float* h_series, int32_t n_trials, fdas_cand* h_out,
                     int64_t* h_counts) {
  NvtxRange range("fdas_search_host");
  if (!p || !h_series || n_trials < 0 || (n_trials > 0 && (!h_out || !h_counts)))
    return set_error(FDAS_ERR_INVALID, "bad argument to fdas_search_host");
  if (n_trials == 1 || p->stream == nullptr) {
    // one trial (or the legacy default stream, which orders every copy after
    // every kernel): copy, run, read back in sequence
    bool overflow = false;
    for (int32_t t = 0; t < n_trials; ++t) {
      int rc = cuda_check(cudaMemcpyAsync(p->series, h_series + (size_t)t * p->N,
                                          sizeof(float) * p->N, cudaMemcpyHostToDevice,
                                          p->stream),
                          "copy series");
      if (rc) return rc;
      rc = search_impl(p, p->series, 1, h_out + (size_t)t * p->max_cands, h_counts + t);
      if (rc == FDAS_ERR_OVERFLOW) overflow = true;
      else if (rc) return rc;
    }
    return overflow ? set_error(FDAS_ERR_OVERFLOW, "candidate list overflow") : FDAS_OK;
  }
  return host_pipeline(p, h_series, n_trials, h_out, h_counts);
}

int fdas_search_device(fdas_plan* p, const float* d_series, int32_t n_trials, fdas_cand* d_out,
                       int64_t* d_counts) {
  NvtxRange range("fdas_search_device");
  if (!p || !d_series || n_trials < 0 || (n_trials > 0 && (!d_out || !d_counts)))
    return set_error(FDAS_ERR_INVALID, "bad argument to fdas_search_device");
  if (int rc = check_aligned(d_series, 8, "d_series")) return rc;
  if (int rc = check_aligned(d_out, 4, "d_out")) return rc;
  if (int rc = check_aligned(d_counts, 8, "d_counts")) return rc;
  fdas_plan* q[2] = {p, p};
  if (n_trials > 1 && lanes_usable(p)) {
    // odd trials on the second lane: it starts after the caller's work on
    // the plan stream, which continues once both lanes are done
    int rc = ensure_lane(p);
    if (!rc) rc = cuda_check(cudaEventRecord(p->ev_fork, p->stream), "event");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(p->lane->stream, p->ev_fork, 0), "wait");
    if (rc) return rc;
    q[1] = p->lane;
  }
  for (int32_t t = 0; t < n_trials; ++t) {
    int rc = run_trial(q[t & 1], d_series + (size_t)t * p->N, d_out + (size_t)t * p->max_cands,
                       reinterpret_cast<unsigned long long*>(d_counts + t));
    if (rc) return rc;
  }
  if (q[1] != p) {
    int rc = cuda_check(cudaEventRecord(p->ev_join, q[1]->stream), "event");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(p->stream, p->ev_join, 0), "wait");
    if (rc) return rc;
    p->last_on_lane = (n_trials - 1) & 1;
  }
  return FDAS_OK;
}

int fdas_plane_debug(fdas_plan* p, float* d_plane) {
  if (!p || !d_plane) return set_error(FDAS_ERR_INVALID, "NULL argument");
  // the lane's plane if the last trial ran there (its work is ordered
  // before the plan stream's by the join of that call)
  const float* src = p->last_on_lane && p->lane ? p->lane->plane : p->plane;
  return cuda_check(cudaMemcpyAsync(d_plane, src, sizeof(float) * (size_t)p->Z * plane_width(p),
                                    cudaMemcpyDeviceToDevice, p->stream),
                    "copy plane");
}

int fdas_stage_spectrum(fdas_plan* p, const float* d_series, float* d_spectrum) {
  if (!p || !d_series || !d_spectrum) return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int rc = check_aligned(d_series, 8, "d_series")) return rc;
  if (int rc = check_aligned(d_spectrum, 8, "d_spectrum")) return rc;
  return launch_spectrum(p, d_series, reinterpret_cast<float2*>(d_spectrum));
}

int fdas_stage_whiten(fdas_plan* p, const float* d_spectrum, float* d_white) {
  if (!p || !d_spectrum || !d_white) return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int rc = check_aligned(d_spectrum, 16, "d_spectrum")) return rc;
  if (int rc = check_aligned(d_white, 16, "d_white")) return rc;
  return launch_whiten(p, reinterpret_cast<const float2*>(d_spectrum),
                       reinterpret_cast<float2*>(d_white));
}

int fdas_stage_plane(fdas_plan* p, const float* d_white, float* d_plane) {
  if (!p || !d_white || !d_plane) return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int rc = check_aligned(d_white, 8, "d_white")) return rc;
  if (int rc = check_aligned(d_plane, 16, "d_plane")) return rc;
  if (p->corr_mode != FDAS_CORR_FFT) {
    // the tensor-core kernel reads the plan's whitened spectrum
    int rc = cuda_check(cudaMemcpyAsync(p->white, d_white, sizeof(float2) * (size_t)p->nb,
                                        cudaMemcpyDeviceToDevice, p->stream), "copy spectrum");
    if (rc) return rc;
    if ((rc = launch_gemm_correlate(p, d_plane))) return rc;
    return gemm_status(p);
  }
  int rc = launch_segments(p, reinterpret_cast<const float2*>(d_white));
  if (rc) return rc;
  return launch_correlate(p, d_plane, nullptr, nullptr, nullptr);
}

int fdas_distill(fdas_plan* p, const fdas_cand* d_cands, const int64_t* d_count,
                 fdas_peak* d_peaks, int64_t* d_npeaks) {
  if (!p || !d_cands || !d_count || !d_peaks || !d_npeaks)
    return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int rc = check_aligned(d_cands, 4, "d_cands")) return rc;
  if (int rc = check_aligned(d_peaks, 4, "d_peaks")) return rc;
  if (int rc = check_aligned(d_count, 8, "d_count")) return rc;
  if (int rc = check_aligned(d_npeaks, 8, "d_npeaks")) return rc;
  return launch_distill(p, d_cands, d_count, d_peaks, d_npeaks);
}

int fdas_plan_set_interbin(fdas_plan* p, int32_t enable) {
  if (!p) return set_error(FDAS_ERR_INVALID, "NULL plan");
  if (!enable) {
    p->interbin = 0;
    return make_hs_order(p);
  }
  if (p->corr_mode != FDAS_CORR_FFT)
    return set_error(FDAS_ERR_INVALID, "half-bin planes use the FFT correlation only");
  int rc;
  if (!p->taps_ib) {
    if ((rc = dalloc(p, &p->taps_ib, (size_t)2 * p->Z * p->m))) return rc;
    if ((rc = dalloc(p, &p->bank_ib, (size_t)2 * p->Z * p->L))) return rc;
    if ((rc = launch_template_interbin(p))) return rc;
  }
  const int64_t need = (int64_t)p->Z * 2 * p->nb;
  if (p->plane_cap < need) {
    // the larger buffers first: a refused allocation leaves the plan as it was
    float *plane = nullptr, *q4 = nullptr;
    if ((rc = dalloc(p, &plane, (size_t)need))) return rc;
    if ((rc = dalloc(p, &q4, (size_t)need / 4))) {
      cudaFree(plane);
      p->device_bytes -= (int64_t)sizeof(float) * need;
      return rc;
    }
    if ((rc = cuda_check(cudaStreamSynchronize(p->stream), "sync"))) {
      cudaFree(plane);
      cudaFree(q4);
      p->device_bytes -= (int64_t)sizeof(float) * (need + need / 4);
      return rc;
    }
    cudaFree(p->plane);
    cudaFree(p->q4);
    p->device_bytes -= (int64_t)sizeof(float) * (p->plane_cap + p->plane_cap / 4);
    p->plane = plane;
    p->q4 = q4;
    p->plane_cap = need;
  }
  p->interbin = 1;
  if ((rc = make_hs_order(p))) return rc;
  return cuda_check(cudaStreamSynchronize(p->stream), "half-bin templates");
}

int fdas_plan_set_whitening(fdas_plan* p, int32_t mode) {
  if (!p) return set_error(FDAS_ERR_INVALID, "NULL plan");
  if (mode != FDAS_WHITEN_RUNNING && mode != FDAS_WHITEN_BLOCK)
    return set_error(FDAS_ERR_INVALID, "unknown whitening mode");
  p->whiten_mode = mode;
  return FDAS_OK;
}

int fdas_plan_set_harmsum_block(fdas_plan* p, int32_t threads) {
  if (!p) return set_error(FDAS_ERR_INVALID, "NULL plan");
  if (threads != 32 && threads != 256)
    return set_error(FDAS_ERR_INVALID, "harmonic-sum block must be 32 or 256 threads");
  p->hs_threads = threads;
  return FDAS_OK;
}

int fdas_plan_set_correlation(fdas_plan* p, int32_t mode) {
  if (!p) return set_error(FDAS_ERR_INVALID, "NULL plan");
  if (mode != FDAS_CORR_FFT && mode != FDAS_CORR_GEMM_BF16 && mode != FDAS_CORR_GEMM_FP16)
    return set_error(FDAS_ERR_INVALID, "unknown correlation mode");
  if (mode == FDAS_CORR_FFT) {
    p->corr_mode = mode;
    return FDAS_OK;
  }
  if (p->interbin)
    return set_error(FDAS_ERR_INVALID, "half-bin planes use the FFT correlation only");
  int rc = gemm_check_shape(p);
  if (rc) return rc;
  if (!p->gbank && (rc = dalloc(p, &p->gbank, gemm_bank_elems(p)))) return rc;
  if (!p->gstatus && (rc = dalloc(p, &p->gstatus, 1))) return rc;
  if ((rc = cuda_check(cudaMemsetAsync(p->gstatus, 0, sizeof(int), p->stream), "memset status")))
    return rc;
  const int old = p->corr_mode;
  p->corr_mode = mode;
  if ((rc = launch_gemm_bank(p))) {
    p->corr_mode = old;
    return rc;
  }
  return cuda_check(cudaStreamSynchronize(p->stream), "template matrix");
}

int fdas_plan_set_wait_limit(fdas_plan* p, uint32_t polls) {
  if (!p) return set_error(FDAS_ERR_INVALID, "NULL plan");
  p->gm_spin = polls;
  return FDAS_OK;
}

int fdas_stage_harmsum(fdas_plan* p, const float* d_plane, fdas_cand* d_out, int64_t* d_count) {
  if (!p || !d_plane || !d_out || !d_count) return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int e = check_aligned(d_plane, 16, "d_plane")) return e;
  if (int e = check_aligned(d_out, 4, "d_out")) return e;
  if (int e = check_aligned(d_count, 8, "d_count")) return e;
  int rc = cuda_check(cudaMemsetAsync(d_count, 0, sizeof(int64_t), p->stream), "memset count");
  if (rc) return rc;
  auto* cnt = reinterpret_cast<unsigned long long*>(d_count);
  if ((rc = launch_pool4(p, d_plane, p->q4, d_out, cnt))) return rc;
  return launch_harmsum(p, d_plane, p->q4, d_out, cnt);
}

int fdas_template_taps(fdas_plan* p, double* d_taps) {
  if (!p || !d_taps) return set_error(FDAS_ERR_INVALID, "NULL argument");
  return cuda_check(cudaMemcpyAsync(d_taps, p->taps, sizeof(double2) * (size_t)p->Z * p->m,
                                    cudaMemcpyDeviceToDevice, p->stream),
                    "copy taps");
}

int fdas_template_bank(fdas_plan* p, float* d_bank) {
  if (!p || !d_bank) return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int rc = check_aligned(d_bank, 8, "d_bank")) return rc;
  return launch_bank_natural(p, reinterpret_cast<float2*>(d_bank));
}

int fdas_profile_trial(fdas_plan* p, const float* d_series, float* h_ms) {
  if (!p || !d_series || !h_ms) return set_error(FDAS_ERR_INVALID, "NULL argument");
  if (int rc = check_aligned(d_series, 8, "d_series")) return rc;
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) {
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
      return set_error(FDAS_ERR_CUDA, "cudaEventCreate failed");
    }
  }
  p->last_on_lane = false;
  int rc = cuda_check(cudaMemsetAsync(p->count, 0, sizeof(unsigned long long), p->stream),
                      "memset count");
  if (!rc) rc = cuda_check(cudaEventRecord(ev[0], p->stream), "event");
  if (!rc) rc = launch_spectrum(p, d_series, p->spec);
  if (!rc) rc = cuda_check(cudaEventRecord(ev[1], p->stream), "event");
  if (!rc) rc = launch_whiten(p, p->spec, p->white);
  if (!rc) rc = cuda_check(cudaEventRecord(ev[2], p->stream), "event");
  // the tensor-core modes have no segment FFTs; their 4-bin maxima and h = 1
  // threshold (a separate kernel there) count as harmonic-sum time
  const bool fft = p->corr_mode == FDAS_CORR_FFT && !p->interbin;
  if (!rc && p->corr_mode == FDAS_CORR_FFT) rc = launch_segments(p, p->white);
  if (!rc) rc = cuda_check(cudaEventRecord(ev[3], p->stream), "event");
  if (!rc) rc = fft ? launch_correlate(p, p->plane, p->q4, p->cands, p->count)
                    : p->interbin ? launch_correlate(p, p->plane, nullptr, nullptr, nullptr)
                                  : launch_gemm_correlate(p, p->plane);
  if (!rc) rc = cuda_check(cudaEventRecord(ev[4], p->stream), "event");
  if (!rc && !fft) rc = launch_pool4(p, p->plane, p->q4, p->cands, p->count);
  if (!rc) rc = launch_harmsum(p, p->plane, p->q4, p->cands, p->count);
  if (!rc) rc = cuda_check(cudaEventRecord(ev[5], p->stream), "event");
  if (!rc) rc = cuda_check(cudaEventSynchronize(ev[5]), "event sync");
  for (int i = 0; i < 5 && !rc; ++i)
    rc = cuda_check(cudaEventElapsedTime(&h_ms[i], ev[i], ev[i + 1]), "elapsed");
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

int fdas_host_fresnel(double x, double* C, double* S) {
  if (!C || !S) return set_error(FDAS_ERR_INVALID, "NULL argument");
  fresnel_host(x, C, S);
  return FDAS_OK;
}

// ---------------------------------------------------------------------------
// Batches of DM trials (Section 1: the search runs once per de-dispersed
// trial, ~6000 per observation) of uneven length and mixed acceleration
// range. One plan's per-trial workspaces, sized for the longest series and
// the largest zmax class, serve every trial. A zmax class owns only its
// templates (taps and spectra), L-point twiddles and harmonic-sum tile
// orders; per length only the real-FFT geometry and its twiddle tables
// differ, cached as lightweight views of a class.
// ---------------------------------------------------------------------------
}  // extern "C"

struct fdas_batch {
  fdas_plan* base = nullptr;          // class 0; owns every workspace
  std::vector<fdas_plan*> classes;    // classes[0] == base; others share its workspaces
  std::vector<fdas_plan*> views;      // (length, class) views other than the classes themselves
  std::vector<int> view_cls;          // class of each view
  // captured CUDA graph of the last batch and the arguments it was made for
  bool graphs = true;
  cudaGraphExec_t exec = nullptr;
  std::vector<const float*> key_series;
  std::vector<int64_t> key_N;
  std::vector<int32_t> key_zmax;
  fdas_cand* key_out = nullptr;
  int64_t* key_counts = nullptr;
  int64_t key_lane_gen = 0;  // the base's trial lane the graph was captured with (0: none)
  int64_t graph_builds = 0, graph_launches = 0;
  // autotuner record
  int n_tuned = 0;
  int32_t tuned_segment[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t tuned_hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float tuned_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

// The per-trial workspaces of a class or view are the base plan's.
void share_workspaces(fdas_plan* d, const fdas_plan* b) {
  d->series = b->series; d->zbuf = b->zbuf; d->spec = b->spec; d->spec2 = b->spec2;
  d->white = b->white; d->seg = b->seg; d->plane = b->plane; d->q4 = b->q4;
  d->cands = b->cands; d->count = b->count; d->hs_list = b->hs_list; d->hs_nlist = b->hs_nlist;
  d->plane_cap = b->plane_cap; d->seg_cap = b->seg_cap;
}

// A copy of plan b that owns nothing yet: every pointer it may free, and
// every per-plan resource a search would make on first use, is cleared.
fdas_plan* unowned_copy(const fdas_plan* b) {
  fdas_plan* v = new fdas_plan(*b);
  v->hs_order[0] = v->hs_order[1] = nullptr;
  v->hs_order_w = 0;
  v->lane = nullptr;  // batches fork the base's lane themselves
  v->ev_fork = v->ev_join = nullptr;
  v->lane_gen = 0;
  v->series2 = nullptr; v->series3[0] = v->series3[1] = nullptr;
  v->cands2 = nullptr; v->count2 = nullptr; v->cstream = nullptr;
  v->cands3[0] = v->cands3[1] = nullptr;
  v->count3[0] = v->count3[1] = nullptr;
  for (int k = 0; k < 4; ++k) v->ev_in[k] = v->ev_done[k] = nullptr;
  v->dkeys = nullptr; v->dvals = nullptr; v->dbits = 0;
  v->gbank = nullptr; v->gstatus = nullptr; v->taps_ib = nullptr; v->bank_ib = nullptr;
  v->device_bytes = 0;
  return v;
}

void free_class(fdas_plan* c) {
  void* ptrs[] = {c->tw_L, c->taps, c->bank};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  free_hs_order(c);
  delete c;
}

void free_view(fdas_plan* v) {
  free_geometry_tables(v);
  free_hs_order(v);
  delete v;
}

int class_index(const fdas_batch* b, int32_t zmax) {
  for (size_t k = 0; k < b->classes.size(); ++k)
    if (b->classes[k]->zmax == zmax) return (int)k;
  return -1;
}

// Replaces one of the base plan's workspaces by a larger one (the stream is
// idle: the caller synchronised it). The new buffer is allocated before the
// old one is freed, so a refused allocation leaves the batch as it was.
template <typename T>
int replace_buffer(fdas_plan* base, T** buf, int64_t elem_now, int64_t need) {
  T* fresh = nullptr;
  int rc = dalloc(base, &fresh, (size_t)need);
  if (rc) return rc;
  cudaFree(*buf);
  base->device_bytes -= (int64_t)sizeof(T) * elem_now;
  *buf = fresh;
  return FDAS_OK;
}

// The lane and any captured graph name the old workspaces: drop them.
void drop_workspace_users(fdas_batch* b) {
  free_lane(b->base);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
}

// Adds the zmax class (zmax, m, L) to the batch: templates and tables of its
// own, the base's workspaces grown to fit its plane and segment spectra.
int add_class(fdas_batch* b, int32_t zmax, int32_t m, int32_t L) {
  fdas_plan* base = b->base;
  const int32_t dz = base->dz;
  if (zmax < 0 || zmax % dz != 0)
    return set_error(FDAS_ERR_INVALID, "class zmax must be >= 0 and a multiple of the batch's dz");
  if (m < 8 || (m & 7)) return set_error(FDAS_ERR_INVALID, "template width must be a multiple of 8");
  if (L != 2048 && L != 4096 && L != 8192)
    return set_error(FDAS_ERR_INVALID, "segment length must be 2048, 4096 or 8192");
  if (L < 2 * m) return set_error(FDAS_ERR_INVALID, "segment length must be >= 2 * width");
  if (class_index(b, zmax) >= 0)
    return set_error(FDAS_ERR_INVALID, "the batch already has a class for this zmax");
  if ((int64_t)(2 * (zmax / dz) + 1) * base->nb > (int64_t(1) << 40))
    return set_error(FDAS_ERR_INVALID, "plane too large");
  int rc = cuda_check(cudaStreamSynchronize(base->stream), "sync");
  if (rc) return rc;
  fdas_plan* c = unowned_copy(base);
  c->tw_L = nullptr; c->taps = nullptr; c->bank = nullptr;
  c->zmax = zmax;
  c->Z = 2 * (zmax / dz) + 1;
  c->m = m;
  c->L = L;
  c->V = L - m;
  c->S = (int)((c->nb + c->V - 1) / c->V);
  if (!rc) rc = dalloc(c, &c->tw_L, (size_t)L);
  if (!rc) rc = dalloc(c, &c->taps, (size_t)c->Z * m);
  if (!rc) rc = dalloc(c, &c->bank, (size_t)c->Z * L);
  if (!rc) rc = make_hs_order(c);
  if (!rc) rc = launch_twiddles(c->tw_L, L, 1, L, c->stream);
  if (!rc) rc = launch_template_taps(c);
  if (!rc) rc = launch_template_bank(c);
  if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream), "class templates");
  const int64_t seg_need = (int64_t)c->S * L;
  if (!rc && base->seg_cap < seg_need) {
    rc = replace_buffer(base, &base->seg, base->seg_cap, seg_need);
    if (!rc) {
      base->seg_cap = seg_need;
      drop_workspace_users(b);
    }
  }
  const int64_t plane_need = (int64_t)c->Z * base->nb;
  if (!rc && base->plane_cap < plane_need) {
    // the 4-bin maxima first: if the plane is then refused, the larger
    // maxima buffer still serves the old plane
    rc = replace_buffer(base, &base->q4, base->plane_cap / 4, plane_need / 4);
    if (!rc) {
      drop_workspace_users(b);  // the maxima buffer moved, whatever comes next
      rc = replace_buffer(base, &base->plane, base->plane_cap, plane_need);
    }
    if (!rc) base->plane_cap = plane_need;
  }
  if (rc) {
    free_class(c);
    return rc;
  }
  base->device_bytes += c->device_bytes;
  share_workspaces(c, base);
  b->classes.push_back(c);
  return FDAS_OK;
}

// The plan that runs a trial of length N in the class of zmax: the class
// itself for N = N_max, else a cached view with that length's geometry.
int batch_view(fdas_batch* b, int64_t N, int32_t zmax, fdas_plan** out) {
  fdas_plan* base = b->base;
  const int k = class_index(b, zmax);
  if (k < 0) return set_error(FDAS_ERR_INVALID, "no class for this zmax (fdas_batch_add_class)");
  if (N > base->N) return set_error(FDAS_ERR_INVALID, "series longer than the batch's N_max");
  fdas_plan* c = b->classes[(size_t)k];
  if (N == base->N) {
    *out = c;
    return FDAS_OK;
  }
  for (size_t i = 0; i < b->views.size(); ++i)
    if (b->views[i]->N == N && b->view_cls[i] == k) {
      *out = b->views[i];
      return FDAS_OK;
    }
  fdas_plan* v = unowned_copy(c);  // shares the class's templates and tables
  v->tw_M1 = v->tw_M2 = v->tw4_lo = v->tw4_hi = v->twN_lo = v->twN_hi = nullptr;
  int rc = set_geometry(v, N);
  if (!rc) rc = alloc_geometry_tables(v);
  if (!rc) rc = make_hs_order(v);
  if (rc) {
    free_view(v);
    return rc;
  }
  base->device_bytes += v->device_bytes;
  b->views.push_back(v);
  b->view_cls.push_back(k);
  *out = v;
  return FDAS_OK;
}

// Median times of one trial (3 timed after 1 warm-up) of a fresh plan with
// segment length L on the probe series, for each harmonic-sum block size in
// hs[0..nhs).
int time_segment(int64_t N, int32_t zmax, int32_t dz, int32_t m, int32_t L, int32_t nharm,
                 float sigma, int64_t max_cands, const float* d_probe, cudaStream_t s,
                 const int* hs, int nhs, float* ms_out) {
  fdas_plan* p = nullptr;
  int rc = fdas_plan_create(&p, N, zmax, dz, m, L, nharm, sigma, max_cands, s);
  if (rc) return rc;
  cudaEvent_t ev[2];
  int made = 0;
  for (; made < 2 && !rc; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) rc = set_error(FDAS_ERR_CUDA, "cudaEventCreate failed");
  for (int c = 0; c < nhs && !rc; ++c) {
    p->hs_threads = hs[c];
    float t[3] = {0, 0, 0};
    rc = run_trial(p, d_probe, p->cands, p->count);
    for (int i = 0; i < 3 && !rc; ++i) {
      rc = cuda_check(cudaEventRecord(ev[0], s), "event");
      if (!rc) rc = run_trial(p, d_probe, p->cands, p->count);
      if (!rc) rc = cuda_check(cudaEventRecord(ev[1], s), "event");
      if (!rc) rc = cuda_check(cudaEventSynchronize(ev[1]), "event sync");
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&t[i], ev[0], ev[1]), "elapsed");
    }
    std::sort(t, t + 3);
    ms_out[c] = t[1];
  }
  for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  fdas_plan_destroy(p);
  return rc;
}

// Trials of a batch in order, launched directly on the plan's stream.
// The trials of a batch in order; with a lane (base->lane, made before any
// capture), odd trials run on it: their length's view with the lane's
// workspaces and stream, forked from and joined to the base stream.
int batch_direct(fdas_plan* base, const std::vector<fdas_plan*>& vs,
                 const float* const* d_series, fdas_cand* d_out, int64_t* d_counts) {
  fdas_plan* lane = vs.size() > 1 && lanes_usable(base) ? base->lane : nullptr;
  int rc = FDAS_OK;
  if (lane) {
    rc = cuda_check(cudaEventRecord(base->ev_fork, base->stream), "event");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(lane->stream, base->ev_fork, 0), "wait");
  }
  for (size_t t = 0; t < vs.size() && !rc; ++t) {
    fdas_cand* out = d_out + t * vs[t]->max_cands;
    auto* cnt = reinterpret_cast<unsigned long long*>(d_counts + t);
    if (lane && (t & 1)) {
      fdas_plan lv = *vs[t];  // this length's geometry and tables
      lv.series = lane->series; lv.zbuf = lane->zbuf; lv.spec = lane->spec;
      lv.spec2 = lane->spec2; lv.white = lane->white; lv.seg = lane->seg;
      lv.plane = lane->plane; lv.q4 = lane->q4; lv.hs_list = lane->hs_list;
      lv.hs_nlist = lane->hs_nlist; lv.stream = lane->stream;
      rc = run_trial(&lv, d_series[t], out, cnt);
    } else {
      rc = run_trial(vs[t], d_series[t], out, cnt);
    }
  }
  if (!rc && lane) {
    rc = cuda_check(cudaEventRecord(base->ev_join, lane->stream), "event");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(base->stream, base->ev_join, 0), "wait");
  }
  return rc;
}

}  // namespace

extern "C" {

int fdas_batch_create(fdas_batch** out, int64_t N_max, int32_t zmax, int32_t dz, int32_t m,
                      int32_t L, int32_t nharm, float sigma, int64_t max_cands, void* stream) {
  if (!out) return set_error(FDAS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  fdas_plan* base = nullptr;
  int rc = fdas_plan_create(&base, N_max, zmax, dz, m, L, nharm, sigma, max_cands, stream);
  if (rc) return rc;
  fdas_batch* b = new fdas_batch();
  b->base = base;
  b->classes.push_back(base);
  *out = b;
  return FDAS_OK;
}

int fdas_batch_add_class(fdas_batch* b, int32_t zmax, int32_t template_width, int32_t segment) {
  if (!b) return set_error(FDAS_ERR_INVALID, "NULL batch");
  return add_class(b, zmax, template_width, segment);
}

int fdas_batch_create_tuned(fdas_batch** out, int64_t N_max, int32_t zmax, int32_t dz,
                            int32_t m, int32_t nharm, float sigma, int64_t max_cands,
                            const float* d_probe, void* stream) {
  if (!out) return set_error(FDAS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (int e = check_aligned(d_probe, 8, "d_probe")) return e;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t cand[3] = {2048, 4096, 8192};
  float* own = nullptr;
  int rc = FDAS_OK;
  if (!d_probe) {
    if (N_max < (1 << 12) || N_max > (1 << 24))
      return set_error(FDAS_ERR_INVALID, "N must be 2^a 3^b 5^c with a >= 12 and 2^12 <= N <= 2^24");
    cudaError_t e = cudaMalloc((void**)&own, sizeof(float) * (size_t)N_max);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(FDAS_ERR_NOMEM, "probe series allocation failed");
    }
    rc = launch_probe_noise(own, N_max, 0x5eedull, s);
    d_probe = own;
  }
  const int hs[2] = {256, 32};  // harmonic-sum block sizes
  int n = 0, best = -1;
  int32_t Ls[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 3 && !rc; ++i) {
    if (cand[i] < 2 * m) continue;
    rc = time_segment(N_max, zmax, dz, m, cand[i], nharm, sigma, max_cands, d_probe, s, hs, 2,
                      &ms[n]);
    if (rc) break;
    for (int c = 0; c < 2; ++c, ++n) {
      Ls[n] = cand[i];
      Hs[n] = hs[c];
      if (best < 0 || ms[n] < ms[best]) best = n;
    }
  }
  if (own) {
    cudaStreamSynchronize(s);
    cudaFree(own);
  }
  if (rc) return rc;
  if (best < 0) return set_error(FDAS_ERR_INVALID, "no segment length with L >= 2m");
  rc = fdas_batch_create(out, N_max, zmax, dz, m, Ls[best], nharm, sigma, max_cands, stream);
  if (rc) return rc;
  (*out)->base->hs_threads = Hs[best];
  (*out)->n_tuned = n;
  for (int i = 0; i < n; ++i) {
    (*out)->tuned_segment[i] = Ls[i];
    (*out)->tuned_hs[i] = Hs[i];
    (*out)->tuned_ms[i] = ms[i];
  }
  return FDAS_OK;
}

int fdas_batch_set_graphs(fdas_batch* b, int32_t enable) {
  if (!b) return set_error(FDAS_ERR_INVALID, "NULL batch");
  b->graphs = enable != 0;
  return FDAS_OK;
}

int fdas_batch_get_info(const fdas_batch* b, fdas_batch_info* info) {
  if (!b || !info) return set_error(FDAS_ERR_INVALID, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->N_max = b->base->N;
  info->segment = b->base->L;
  // distinct series lengths with a geometry
  std::vector<int64_t> lens{b->base->N};
  for (const fdas_plan* v : b->views)
    if (std::find(lens.begin(), lens.end(), v->N) == lens.end()) lens.push_back(v->N);
  info->n_lengths = (int32_t)lens.size();
  info->graphs = b->graphs && b->base->stream != nullptr;
  info->graph_builds = b->graph_builds;
  info->graph_launches = b->graph_launches;
  info->hs_block = b->base->hs_threads;
  info->n_tuned = b->n_tuned;
  for (int i = 0; i < 8; ++i) {
    info->tuned_segment[i] = b->tuned_segment[i];
    info->tuned_hs_block[i] = b->tuned_hs[i];
    info->tuned_ms[i] = b->tuned_ms[i];
  }
  info->n_classes = (int32_t)b->classes.size();
  info->device_bytes = b->base->device_bytes;
  return FDAS_OK;
}

int fdas_batch_destroy(fdas_batch* b) {
  if (!b) return FDAS_OK;
  if (b->base && b->base->stream) cudaStreamSynchronize(b->base->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (fdas_plan* v : b->views) free_view(v);
  for (size_t k = 1; k < b->classes.size(); ++k) free_class(b->classes[k]);
  fdas_plan_destroy(b->base);
  delete b;
  return FDAS_OK;
}

int fdas_search_batch(fdas_batch* b, const float* const* d_series, const int64_t* N,
                      const int32_t* zmax, int32_t n_trials, fdas_cand* d_out,
                      int64_t* d_counts) {
  NvtxRange range("fdas_search_batch");
  if (!b || !d_series || !N || n_trials < 0 || (n_trials > 0 && (!d_out || !d_counts)))
    return set_error(FDAS_ERR_INVALID, "bad argument to fdas_search_batch");
  if (n_trials > 0) {
    if (int rc = check_aligned(d_out, 4, "d_out")) return rc;
    if (int rc = check_aligned(d_counts, 8, "d_counts")) return rc;
  }
  // every (length, class) geometry first: allocations cannot be captured
  std::vector<fdas_plan*> vs((size_t)n_trials);
  std::vector<int32_t> zs((size_t)n_trials);
  for (int32_t t = 0; t < n_trials; ++t) {
    if (!d_series[t]) return set_error(FDAS_ERR_INVALID, "NULL series in batch");
    if (int rc = check_aligned(d_series[t], 8, "d_series[t]")) return rc;
    zs[(size_t)t] = zmax ? zmax[t] : b->base->zmax;
    int rc = batch_view(b, N[t], zs[(size_t)t], &vs[(size_t)t]);
    if (rc) return rc;
  }
  for (size_t k = 1; k < b->classes.size(); ++k) share_workspaces(b->classes[k], b->base);
  for (fdas_plan* v : b->views) share_workspaces(v, b->base);
  if (n_trials > 1 && lanes_usable(b->base)) {
    int rc = ensure_lane(b->base);
    if (rc) return rc;
  }
  cudaStream_t s = b->base->stream;
  // the legacy default stream cannot be captured
  if (!b->graphs || s == nullptr || n_trials == 0)
    return batch_direct(b->base, vs, d_series, d_out, d_counts);
  const bool same = b->exec && b->key_out == d_out && b->key_counts == d_counts &&
                    b->key_lane_gen == (b->base->lane ? b->base->lane_gen : 0) &&
                    b->key_series.size() == (size_t)n_trials &&
                    std::equal(b->key_series.begin(), b->key_series.end(), d_series) &&
                    std::equal(b->key_N.begin(), b->key_N.end(), N) &&
                    std::equal(b->key_zmax.begin(), b->key_zmax.end(), zs.begin());
  if (!same) {
    int rc = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal),
                        "begin capture");
    if (rc) return rc;
    const int trc = batch_direct(b->base, vs, d_series, d_out, d_counts);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (trc || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return trc ? trc : cuda_check(ce, "end capture");
    }
    if (b->exec) {
      cudaGraphExecUpdateResultInfo upd;
      if (cudaGraphExecUpdate(b->exec, g, &upd) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
    }
    if (!b->exec) {
      const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
      if (ie != cudaSuccess) {
        b->exec = nullptr;
        cudaGraphDestroy(g);
        return cuda_check(ie, "graph instantiate");
      }
    }
    cudaGraphDestroy(g);
    ++b->graph_builds;
    b->key_series.assign(d_series, d_series + n_trials);
    b->key_N.assign(N, N + n_trials);
    b->key_zmax = zs;
    b->key_out = d_out;
    b->key_counts = d_counts;
    b->key_lane_gen = b->base->lane ? b->base->lane_gen : 0;
  }
  ++b->graph_launches;
  return cuda_check(cudaGraphLaunch(b->exec, s), "graph launch");
}

const char* fdas_strerror(int status) {
  switch (status) {
    case FDAS_OK: return "ok";
    case FDAS_ERR_INVALID: return "invalid argument";
    case FDAS_ERR_NOMEM: return "out of memory";
    case FDAS_ERR_CUDA: return "CUDA error";
    case FDAS_ERR_TIMEOUT: return "device wait timed out";
    case FDAS_ERR_OVERFLOW: return "candidate list overflow";
  }
  return "unknown status";
}

const char* fdas_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
