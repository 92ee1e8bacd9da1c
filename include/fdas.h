/*
 * fdas.h - C ABI of the GB300 (sm_103a) Fourier Domain Acceleration Search.
 *
 * The library implements the hot path of the FDAS method of Dimoudi &
 * Armour, "Pulsar Acceleration Searches on the GPU for the Square Kilometre
 * Array" (Sections 2 and 4): for each de-dispersed time series
 *   real FFT (step 2) -> 64-bin running-median whitening ->
 *   overlapped segments (step 3) -> segment FFT (step 4) ->
 *   multiply by the conjugated z-templates (step 5) -> inverse FFT (step 6) ->
 *   power and edge removal (step 7) = the f-fdot power plane of Eq. 1 ->
 *   harmonic sums h = 1, 2, 4, 8, 16 -> threshold -> compacted candidate list.
 *
 * Conventions (all entry points):
 *  - Every function returns an int status: FDAS_OK (0) or a negative
 *    FDAS_ERR_* code; nothing throws across the ABI. fdas_strerror() maps a
 *    code to text, fdas_last_error() gives the detail of the last failure on
 *    the calling thread.
 *  - Pointers named d_* are device pointers, h_* host pointers. The caller
 *    owns every buffer it passes; the plan owns everything it allocates on
 *    the device (templates, twiddle tables, workspaces) and frees it in
 *    fdas_plan_destroy().
 *  - A plan is bound to the CUDA stream given at creation (NULL = the legacy
 *    default stream) and is not thread-safe; use one plan per stream.
 *  - Complex data are interleaved float32 (re, im) pairs, i.e. float2.
 *  - Device pointers must be aligned for the vector accesses the kernels
 *    make through them: series and spectra 8 bytes (float2), the whitening
 *    stage's input and output and every plane 16 bytes (float4), 64-bit
 *    counts 8 bytes, candidate and peak lists 4 bytes. Memory from
 *    cudaMalloc (or a torch tensor's storage) is aligned; a view that starts
 *    at an odd element may not be. A misaligned pointer returns
 *    FDAS_ERR_INVALID before any device work.
 *
 * Notation: N samples per series, nb = N/2 Fourier bins (Nyquist dropped),
 * z_j = -zmax + j*dz for j = 0..Z-1 (Z = 2*zmax/dz + 1, z = fdot*T^2 in bins,
 * Section 2), m template taps, L segment length, V = L - m valid outputs per
 * segment, S = ceil(nb / V) segments.
 */
#ifndef FDAS_H
#define FDAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum fdas_status {
  FDAS_OK = 0,
  FDAS_ERR_INVALID = -1,  /* bad argument or unsupported size */
  FDAS_ERR_NOMEM = -2,    /* a device or host allocation failed */
  FDAS_ERR_CUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  FDAS_ERR_TIMEOUT = -4,  /* a bounded device wait gave up */
  FDAS_ERR_OVERFLOW = -5  /* more candidates than max_cands (count still exact) */
};

typedef struct fdas_plan fdas_plan;

/* One detection: the harmonic sum H_h at top-harmonic bin r_top and template
 * index z_idx (z = -zmax + z_idx*dz) reached the threshold T_h. */
typedef struct {
  int32_t r_top;
  int32_t z_idx;
  int32_t h;
  float power;
} fdas_cand;

typedef struct {
  int64_t N, nb;
  int32_t zmax, dz, Z, m, L, V, S, nharm, n_levels;
  float thresholds[5];      /* T_h for h = 1, 2, 4, 8, 16 (first n_levels used) */
  int64_t max_cands;
  int64_t device_bytes;     /* device memory the plan holds */
  int64_t plane_floats;     /* Z * nb */
  int32_t corr_ctas_per_sm; /* launch shape of the correlation kernel (0 before the first search) */
  int32_t corr_grid;
} fdas_plan_info;

/* Creates a plan: validates sizes, allocates the device workspaces and runs
 * the initialisation stage of Section 4 (template computation): the Fresnel
 * response tau_z(d) of Section 2 for d = -m/2..m/2-1 in float64 on the GPU,
 * its length-L spectrum (float64 DFT, scaled by 1/L and rounded to float32),
 * and the float64-generated FFT twiddle tables.
 *   N: 2^a 3^b 5^c with a >= 12, 2^12 <= N <= 2^24.  zmax >= 0, dz > 0, dz | zmax.
 *   template_width m: multiple of 8, m >= 8.  segment L: 2048, 4096 or 8192, L >= 2m.
 *   nharm: 1, 2, 4, 8 or 16.  sigma > 0: Gaussian-equivalent threshold.
 *   max_cands >= 1: capacity of the candidate list per trial.
 *   stream: a cudaStream_t (may be NULL).
 * On error *out is NULL and nothing is leaked. */
int fdas_plan_create(fdas_plan** out, int64_t N, int32_t zmax, int32_t dz,
                     int32_t template_width, int32_t segment, int32_t nharm,
                     float sigma, int64_t max_cands, void* stream);

int fdas_plan_destroy(fdas_plan* plan);

int fdas_plan_get_info(const fdas_plan* plan, fdas_plan_info* info);

/* The full path (Section 4 steps 2-7, harmonic sum, threshold, compaction)
 * on n_trials series stored back to back at d_series (N floats each, device).
 * Candidates of trial t go to h_out + t*max_cands (host, caller-owned),
 * sorted by (h, r_top, z_idx); h_counts[t] is the exact number found, which
 * may exceed max_cands: then only max_cands are stored and the call returns
 * FDAS_ERR_OVERFLOW after finishing every trial. Synchronises the stream.
 * With n_trials > 1 on a stream other than the legacy default stream, earlier
 * trials' candidates are read back and sorted while later trials run: with
 * the second trial lane (below) trial t-2 while trials t-1 and t run, through
 * four candidate lists (the plan's, the lane's and two allocated on first
 * use); without it trial t-1 while trial t runs, through two. */
int fdas_search(fdas_plan* plan, const float* d_series, int32_t n_trials,
                fdas_cand* h_out, int64_t* h_counts);

/* As fdas_search, but the series are in host memory (step 1 of Section 4:
 * the transfer to the GPU is part of the call). With n_trials > 1 on a
 * stream other than the legacy default stream, the copies overlap the
 * kernels: series t+1 is copied in (on a copy stream of the plan, into a
 * second staging buffer) and trial t-1's candidates are read back and
 * sorted while trial t runs; page-locked host memory is needed for the
 * copies to overlap. With the second trial lane (below) the series go
 * through four staging buffers (the plan's, the lane's and two allocated on
 * the first such call, 8N bytes), so the copy of trial t+1 never waits for
 * a running trial, and the candidates through four lists (two more allocated
 * then, 32 max_cands + 16 bytes), so trial t-2 is read back while trials
 * t-1 and t run; where no lane is used (tensor-core or half-bin modes)
 * the first such call allocates a second staging buffer and candidate list
 * (4N + 16 max_cands bytes). */
int fdas_search_host(fdas_plan* plan, const float* h_series, int32_t n_trials,
                     fdas_cand* h_out, int64_t* h_counts);

/* Device-resident variant: enqueues the whole path on the plan's stream and
 * returns without synchronising. Candidates of trial t go, unsorted, to
 * d_out + t*max_cands and d_counts[t] (device int64) receives the exact count
 * (entries past max_cands are dropped). */
int fdas_search_device(fdas_plan* plan, const float* d_series, int32_t n_trials,
                       fdas_cand* d_out, int64_t* d_counts);

/* Trial lanes. When fdas_search, fdas_search_host, fdas_search_device or
 * fdas_search_batch runs 2 or more trials on a stream other than the legacy
 * default stream, with the FFT correlation on integer-bin planes, the odd
 * trials run on a second lane of the plan: its own per-trial workspaces
 * (series staging, spectra, segment spectra, plane, 4-bin maxima and lists;
 * about 4N + 36N + 8 S L + 5 Z N/2 + 16 max_cands + 8 MiB bytes, 4.4 GB for
 * N = 2^23, zmax = 200, L = 8192) and its own stream, sharing the plan's
 * templates and tables, so that consecutive trials overlap on the GPU. The
 * lane is forked from the plan stream at the start of the call and joined
 * back at the end: work enqueued on the plan stream before the call is done
 * before any trial starts, and work enqueued after it waits for every trial.
 * The first such call allocates the lane (counted in device_bytes); it is
 * remade if the plan's shape changes and freed with the plan. */

/* Batches of DM trials (Section 1: the search runs once per de-dispersed
 * trial, about 6000 per 530 s observation for the SKA) of uneven length and
 * mixed acceleration range, each trial through the whole path of Section 4
 * (steps 2-7) plus the harmonic sum, threshold and compaction.
 * fdas_batch_create makes one plan for the longest series N_max (same
 * arguments and limits as fdas_plan_create); its zmax, template width and
 * segment length are the batch's first zmax class. fdas_batch_add_class adds
 * another class (zmax, template_width, segment) under the same dz, nharm,
 * sigma and max_cands (same limits as fdas_plan_create; one class per zmax):
 * it makes that class's template bank (Section 4, initialisation) and grows
 * the shared workspaces (plane, 4-bin maxima, segment spectra) to fit the
 * largest class; every class uses the one set of per-trial workspaces, so a
 * batch holds one plane of the largest class, not one per class. It
 * synchronises the batch's stream; call it between searches.
 * fdas_search_batch runs trial t of length N[t] (N[t] <= N_max,
 * N[t] = 2^a 3^b 5^c with a >= 12) in the class of zmax[t] (host array; NULL
 * = the first class for every trial) from d_series[t] (host array of device
 * pointers, N[t] floats each) and, like fdas_search_device, enqueues the
 * whole path asynchronously with unsorted candidates at d_out + t*max_cands
 * and the exact count in d_counts[t] (device int64). A zmax with no class
 * returns FDAS_ERR_INVALID before any device work. The real-FFT geometry of
 * each new (length, class) pair is built (and cached) on first use, which
 * allocates its small twiddle tables. */
typedef struct fdas_batch fdas_batch;
int fdas_batch_create(fdas_batch** out, int64_t N_max, int32_t zmax, int32_t dz,
                      int32_t template_width, int32_t segment, int32_t nharm, float sigma,
                      int64_t max_cands, void* stream);
int fdas_batch_add_class(fdas_batch* batch, int32_t zmax, int32_t template_width,
                         int32_t segment);
int fdas_batch_destroy(fdas_batch* batch);
int fdas_search_batch(fdas_batch* batch, const float* const* d_series, const int64_t* N,
                      const int32_t* zmax, int32_t n_trials, fdas_cand* d_out,
                      int64_t* d_counts);
/* On a stream other than the legacy default stream, fdas_search_batch
 * captures the whole batch (every trial's kernels and count resets, in
 * order) into one CUDA graph and launches it as a single graph launch. The
 * executable graph is kept: a later call with the same series pointers,
 * lengths, zmax values and output pointers replays it without capturing; other
 * arguments re-capture and update it in place when the topology allows.
 * fdas_batch_set_graphs(batch, 0) launches the kernels directly instead. */
int fdas_batch_set_graphs(fdas_batch* batch, int32_t enable);

/* Autotuned batch (first class only; classes added later keep the segment
 * length they are given): times one trial of every combination of segment length
 * L in {2048, 4096, 8192} with L >= 2m and harmonic-sum block of 256 or 32
 * threads (16384 or 2048 top bins per block) on a probe series of N_max
 * samples (d_probe, device; NULL = seeded Gaussian white noise made on the
 * device), on a fresh plan per L (median of 3 after a warm-up), and creates
 * the batch with the fastest. L sets the segment FFT size, the number of
 * segments and the correlation kernel's occupancy; the plane is the same up
 * to float32 rounding for every L, and the candidates do not depend on the
 * block size. Other arguments as fdas_batch_create. */
int fdas_batch_create_tuned(fdas_batch** out, int64_t N_max, int32_t zmax, int32_t dz,
                            int32_t template_width, int32_t nharm, float sigma,
                            int64_t max_cands, const float* d_probe, void* stream);

typedef struct {
  int64_t N_max;
  int32_t segment;           /* L in use */
  int32_t n_lengths;         /* distinct series lengths with a geometry */
  int32_t graphs;            /* 1 when batches run as captured CUDA graphs */
  int32_t n_tuned;           /* configurations the autotuner timed (0: not tuned) */
  int64_t graph_builds;      /* captures made */
  int64_t graph_launches;    /* graph launches */
  int32_t hs_block;          /* harmonic-sum block in use (threads) */
  int32_t tuned_segment[8];  /* the configurations timed: L ... */
  int32_t tuned_hs_block[8]; /* ... harmonic-sum block ... */
  float tuned_ms[8];         /* ... and their median trial times (ms) */
  int32_t n_classes;         /* zmax classes (1 + fdas_batch_add_class calls) */
  int64_t device_bytes;      /* device memory the batch holds */
} fdas_batch_info;
int fdas_batch_get_info(const fdas_batch* batch, fdas_batch_info* info);

/* Test hook: copies the float32 power plane of the last trial processed,
 * Z x nb row-major by z (P[j*nb + r] = |A(r, z_j)|^2, Eq. 1), to d_plane. */
int fdas_plane_debug(fdas_plan* plan, float* d_plane);

/* Stage entry points (device pointers, asynchronous on the plan's stream),
 * used by the per-stage parity tests. */
/* Step 2: X_k = sum_n x_n exp(-2 pi i k n/N), k = 0..nb-1 -> d_spectrum (nb float2). */
int fdas_stage_spectrum(fdas_plan* plan, const float* d_series, float* d_spectrum);
/* Whitening: mu_k = median of |X|^2 over the 64-bin window [k-32, k+31]
 * shifted into [1, nb-1]; Xw_k = X_k sqrt(ln2/mu_k), Xw_0 = 0 (nb float2). */
int fdas_stage_whiten(fdas_plan* plan, const float* d_spectrum, float* d_white);
/* Steps 3-7 on a whitened spectrum: writes the Z x nb float32 plane. */
int fdas_stage_plane(fdas_plan* plan, const float* d_white, float* d_plane);
/* Harmonic sum + threshold + compaction on a caller-supplied Z x nb plane;
 * d_count: one device int64. */
int fdas_stage_harmsum(fdas_plan* plan, const float* d_plane, fdas_cand* d_out,
                       int64_t* d_count);
/* Template taps tau_{z_j}(d), float64 complex, Z x m (d = -m/2..m/2-1). */
int fdas_template_taps(fdas_plan* plan, double* d_taps);
/* Template spectra (1/L) sum_d tau(d) exp(+2 pi i k d/L), float2, Z x L. */
int fdas_template_bank(fdas_plan* plan, float* d_bank);

/* Per-stage timing of one trial on the plan's stream (CUDA events around
 * each kernel launch group; synchronises). h_ms[0..4] receive milliseconds
 * for: spectrum (step 2), whitening, segment FFTs (steps 3-4), correlation
 * (steps 5-7), harmonic sum + threshold + compaction. */
int fdas_profile_trial(fdas_plan* plan, const float* d_series, float* h_ms);
/* (In the tensor-core correlation modes the segment entry is 0, the
 * correlation entry is the GEMM kernel alone, and the harmonic-sum entry
 * includes the 4-bin maxima and h = 1 threshold kernel.) */

/* Correlation modes (steps 5-7 of Section 4, Eq. 1). */
enum fdas_corr_mode {
  FDAS_CORR_FFT = 0,       /* overlap-save FFT correlation, float32 (default) */
  FDAS_CORR_GEMM_BF16 = 1, /* tensor-core GEMM, bf16 hi/lo split, float32 accumulation */
  FDAS_CORR_GEMM_FP16 = 2  /* tensor-core GEMM, fp16 hi/lo split, float32 accumulation */
};

/* Selects how the plan computes the power plane of Eq. 1. The GEMM modes
 * evaluate Eq. 1 directly as a dense contraction: for each block of 512
 * consecutive bins, (2Z x 6m template matrix) x (6m x 512 Hankel-blocked
 * spectrum) on the tcgen05 tensor cores. Each float32 operand is split into
 * a 16-bit hi part and a lo part (fp16: lo scaled by 2^11 to stay normal);
 * the products hi*hi + hi*lo + lo*hi are summed in float32, so the plane
 * carries about 16 (bf16) or 22 (fp16) significant bits. The whitened
 * spectrum must stay below 65504 in magnitude for the fp16 mode. Both modes
 * feed the same harmonic sum and threshold. The left factor is built from the
 * plan's float64 taps when the mode is selected and held until the plan is
 * destroyed (2Z rounded up to 128 rows x 6m x 2 bytes).
 *   mode: an fdas_corr_mode. The GEMM modes need m % 32 == 0 and m <= 768.
 * A bounded device wait that gives up makes the next fdas_search return
 * FDAS_ERR_TIMEOUT. */
int fdas_plan_set_correlation(fdas_plan* plan, int32_t mode);

/* Test hook for the bounded device waits of the tensor-core correlation
 * (the paper has no counterpart; this exercises the failure handling): every
 * pipeline wait of k_gemm_correlate (bulk copies landing, MMA commits,
 * hand-offs between its warp roles) gives up after `polls` polls of its
 * mbarrier (0 = the default, 2^23 polls with back-off, about a second), after
 * which every role leaves its loop and the next fdas_search (or
 * fdas_stage_plane) returns FDAS_ERR_TIMEOUT and clears the status. Whatever
 * the limit, the kernel then waits with the full default bound for the bulk
 * copies it issued and the MMAs it committed (they complete on their own)
 * and frees its tensor memory before it returns, so the context stays
 * usable. polls = 1 makes the first wait run out; a test uses it to check
 * the error path. No effect on the FFT correlation, which waits on nothing. */
int fdas_plan_set_wait_limit(fdas_plan* plan, uint32_t polls);

/* One distilled detection: a local maximum of the candidate list with its
 * Gaussian-equivalent significance. */
typedef struct {
  int32_t r_top;
  int32_t z_idx;
  int32_t h;
  float power;    /* H_h */
  float sigma;    /* Phi_bar(sigma) = Q(h, H_h), Q the Gamma(h, 1) upper tail */
  float log10_p;  /* log10 Q(h, H_h), the per-cell false-alarm probability */
} fdas_peak;

/* Candidate distillation (after the threshold; not in the paper). From the
 * first min(*d_count, max_cands) candidates at d_cands (device; the output
 * of fdas_search_device or of one trial of fdas_search_batch), keeps those
 * that are
 *   - local maxima in H within their level: no candidate of the same h at
 *     (r + dr, j + dj), |dr|, |dj| <= 1, has a larger H (equal H: the
 *     smaller (j, r) wins), and
 *   - the most significant rendering of their signal across adjacent levels:
 *     candidates (r, jc) at level h and (r', jc') at level 2h, jc = j - zc,
 *     zc = (Z-1)/2, count as one signal when |r' - 2r| <= 2 and
 *     |jc' - 2 jc| <= 2; the larger sigma wins (equal: the lower level),
 * writing them to d_peaks (device, max_cands entries, append order) and
 * their exact number to *d_npeaks (device int64). Asynchronous on the plan's
 * stream. The first call allocates a hash table of 2 x max_cands entries
 * (12 bytes each), held by the plan. */
int fdas_distill(fdas_plan* plan, const fdas_cand* d_cands, const int64_t* d_count,
                 fdas_peak* d_peaks, int64_t* d_npeaks);

/* Half-bin (interbinned) planes, the resolution of the paper's Fig. 1:
 * with enable != 0 the plan also evaluates Eq. 1 at the half-integer
 * frequencies r + 1/2, with templates tau_z at frequency offset 1/2 (the same
 * m taps d = -m/2..m/2-1 around bin r; Fresnel form with q = d - 1/2 + z/2),
 * and the plane becomes P[j][2r + e] = |A(r + e/2, z_j)|^2, e = 0, 1: Z rows
 * of 2 nb columns counted in half bins. Harmonic sums and thresholds run
 * unchanged on that plane, so candidate r_top is in half bins (frequency
 * r_top / 2 bins). The first call builds the 2Z-row template bank and
 * doubles the plane and 4-bin-maxima buffers (synchronises the stream);
 * fdas_plane_debug then copies Z x 2nb floats, and fdas_stage_plane writes
 * that many. FFT correlation only (FDAS_ERR_INVALID in a tensor-core mode).
 * enable = 0 returns to the integer plane. */
int fdas_plan_set_interbin(fdas_plan* plan, int32_t enable);

/* Whitening modes (the stage before step 3; not specified by the paper). */
enum fdas_whiten_mode {
  FDAS_WHITEN_RUNNING = 0, /* 64-bin running median, window [k-32, k+31] shifted into [1, nb-1] */
  FDAS_WHITEN_BLOCK = 1    /* medians of 64-bin blocks from bin 1, linearly interpolated */
};

/* Selects the whitening of the plan. FDAS_WHITEN_BLOCK: mu_b = median of
 * |X_k|^2 over [1 + 64 b, min(1 + 64 (b+1), nb)) (mean of the two middle
 * values for an even count), placed at the block centre; mu_k interpolates
 * linearly between adjacent centres and is constant beyond the first and
 * last centre; Xw_k = X_k sqrt(ln 2 / mu_k), Xw_0 = 0. Cheaper than the
 * running median but a different estimate, so candidate lists differ. */
int fdas_plan_set_whitening(fdas_plan* plan, int32_t mode);

/* Block size of the harmonic-sum screen (the stage after step 7 of Section
 * 4): 32 threads (one warp per block, the default) or 256 (eight warps per
 * block; fdas_batch_create_tuned times both). Candidate lists do not depend
 * on it. Any other value returns FDAS_ERR_INVALID. */
int fdas_plan_set_harmsum_block(fdas_plan* plan, int32_t threads);

/* Real FFT of one series without a plan and without allocating device memory.
 * The paper has no counterpart; this exists for callers that must not
 * allocate device memory (for example a real-time loop with a fixed device
 * footprint, or a host framework that owns the device allocator) and so
 * cannot create a plan. Computes the same X_k as fdas_stage_spectrum,
 * k = 0..N/2-1, from d_series (N floats, device) into d_spectrum (N/2 float2,
 * device), asynchronously on `stream` (a cudaStream_t, may be NULL).
 *   N: power of two, 2^12 <= N <= 2^20; larger N returns FDAS_ERR_INVALID.
 * Scratch: a fixed 8.5 MB array in device memory that every GPU loading this
 * library holds until the process exits; no call allocates or frees memory.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture. The
 * address is cached for the life of the process: after cudaDeviceReset on a
 * device, do not call this entry point on that device again. All
 * calls share the one array: calls whose work overlaps on a GPU (different
 * streams or host threads) race and give wrong results; serialise them.
 * Every value the kernels read from the array is written earlier in the same
 * call, so nothing needs clearing between calls. */
int fdas_spectrum_noalloc(const float* d_series, int64_t N, float* d_spectrum, void* stream);

/* Host-side Fresnel integrals C(x), S(x) of the library's own float64
 * implementation (the one the template kernel runs), for CPU checks. */
int fdas_host_fresnel(double x, double* C, double* S);

const char* fdas_strerror(int status);
const char* fdas_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FDAS_H */
