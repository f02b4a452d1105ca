/*
 * fdas.h -- C ABI of the GB300 (sm_103a) Fourier Domain Acceleration Search.
 *
 * Method: arXiv:2211.13517 (White, Adamek, Armour).  §2.1 "FDAS": a matched
 * filter over a grid of constant-acceleration (constant-fdot) templates whose
 * cost grows linearly with the number of templates; §2.2 "Mixed-Precision":
 * the filter is an FFT-based (frequency-domain) convolution, the stage moved
 * from FP32 to bfloat16, with at most 2.7% error in detection strength.
 * The paper does not spell out the normalisation, the template formula, the
 * harmonic sum or the threshold; the readings used here are written next to
 * each entry point below.
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" are CUDA device (or managed) memory of the
 *    current device; "host" pointers are ordinary CPU memory.  Nothing is
 *    retained after the call returns unless stated.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is queued on it in order.
 *  - Every call returns an fdas_status; no C++ exception crosses the ABI.
 *    fdas_last_error() returns a thread-local message for the last failure.
 *  - Arguments are validated before any GPU work is queued; an invalid
 *    argument returns FDAS_ERR_ARG and queues nothing.
 *  - There is no CPU fallback: without a usable CUDA device the calls that
 *    need one return FDAS_ERR_CUDA.
 *
 * Notation: N = n_samples, N_r = N/2 spectral bins r = 0..N_r-1;
 * z_i = (i - K) z_step, K = z_max/z_step, i = 0..n_z-1 (n_z = 2K+1, iz0 = K);
 * m(z) = 8 + ceil(|z|/2) template half-width; H = n_harm.
 */
#ifndef FDAS_H
#define FDAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDAS_OK = 0,
    FDAS_ERR_ARG = 1,            /* invalid argument; nothing was queued     */
    FDAS_ERR_CUDA = 2,           /* a CUDA runtime call failed               */
    FDAS_ERR_OOM = 3,            /* device allocation failed                 */
    FDAS_ERR_CAND_OVERFLOW = 4,  /* more candidates than the caller's buffer */
    FDAS_ERR_NONFINITE = 5,      /* NaN or Inf in an input series, or a
                                    spectral power beyond the FP32 range    */
    FDAS_ERR_TIMEOUT = 6,        /* a bounded device wait gave up            */
    FDAS_ERR_UNSUPPORTED = 7,    /* valid request the library does not serve */
    FDAS_ERR_CAND_STORE_FULL = 8, /* more crossings than the plan's device
                                    store (fdas_opts.max_candidates)         */
    FDAS_ERR_BOUNDS = 9          /* checked build only: a device bounds check
                                    failed or a workspace canary was
                                    overwritten (see fdas_checked_build)     */
} fdas_status;

/* storage precision of spectra, templates and the power plane; the
 * arithmetic (butterflies, products, sums) is FP32 in every mode */
enum { FDAS_FP32 = 0, FDAS_BF16 = 1, FDAS_FP16 = 2 };
/* threshold rule */
enum { FDAS_THRESH_GAMMA_TAIL = 0, FDAS_THRESH_MEAN_PLUS_KSIGMA = 1 };
/* spectral normalisation */
enum { FDAS_NORM_MEDIAN = 0, FDAS_NORM_NONE = 1 };
/* how the power plane is computed (the same P(r, z) either way):
 * FDAS_CORR_FFT: overlap-save, segment FFT x template spectrum, inverse FFT
 *   (FP32 arithmetic on the CUDA cores; every precision);
 * FDAS_CORR_TENSOR: the direct correlation sum_e g_z[e] X'_{r-e} as a GEMM
 *   on the tensor cores (16-bit operands, FP32 accumulation; FDAS_BF16 and
 *   FDAS_FP16 only, with m_overlap <= 112, i.e. z_max <= 208);
 * FDAS_CORR_TENSOR_SPLIT: FP32 storage on the tensor cores: spectrum and
 *   taps each as the sum of two BF16 parts (hi = bf16(x), lo = bf16(x - hi)),
 *   three products per term (hi*hi + hi*lo + lo*hi; the dropped lo*lo term
 *   is about 2^-16 of each product), FP32 accumulation and FP32 plane; P
 *   within about 1e-4 of the FP32 result (FDAS_FP32 only, m_overlap <= 56,
 *   i.e. z_max <= 96 at the default bank);
 * FDAS_CORR_AUTO: TENSOR where it applies, else FFT (never the split mode). */
enum { FDAS_CORR_AUTO = 0, FDAS_CORR_FFT = 1, FDAS_CORR_TENSOR = 2, FDAS_CORR_TENSOR_SPLIT = 3 };
/* harmonic sum:
 * FDAS_HARM_TOP (default): top-harmonic indexed, every plane cell (ir, iz) is
 *   the top harmonic; harmonic j of H reads the rounded sub-multiple
 *   (iz0 + sign(o) floor((|o| j + H/2)/H), floor((ir j + H/2)/H));
 * FDAS_HARM_FUNDAMENTAL: a candidate is labelled by its fundamental (ir, iz)
 *   and stage h sums the exact multiples P[iz0 + k o][k ir], k = 1..h, on the
 *   cells where every multiple lies in the plane (h ir <= N_r - 1,
 *   |h o| <= K); fewer gathers and additions, a different candidate list. */
enum { FDAS_HARM_TOP = 0, FDAS_HARM_FUNDAMENTAL = 1 };
/* order of the templates in the tensor-core correlation's chunks of 28 (the
 * same plane either way; the time differs):
 * FDAS_TORDER_Z: consecutive z;
 * FDAS_TORDER_PAIRED: 14 templates with z <= 0 and 14 with z > 0 of about
 *   the same |z|, so that a chunk's templates have similar widths and less of
 *   the K dimension is padding;
 * FDAS_TORDER_DEFAULT: PAIRED, or with autotune the faster of the two. */
enum { FDAS_TORDER_DEFAULT = 0, FDAS_TORDER_Z = 1, FDAS_TORDER_PAIRED = 2 };
/* Interbinning (fdas_opts.interbin = 1; the paper does not use it, an
 * option of the search): the power plane is sampled every half bin, n_z x
 * 2 N_r cells.  With F(r, z) the complex correlation (the matched-filter
 * output before |.|^2), column 2r holds |F(r)|^2 and column 2r + 1 holds
 * (pi/4)^2 |F(r) - F(r+1)|^2, with F(N_r) = 0: a sinusoid half-way between
 * two bins, which keeps only (2/pi)^2 of its power in either bin, is
 * recovered in full there.  Statistics, harmonic sums (the index formulas
 * applied to columns) and thresholds run on that plane; a candidate's `ir`
 * is its column, the spectral bin ir/2. */

typedef struct {
    int32_t precision;       /* FDAS_FP32 (default), FDAS_BF16, FDAS_FP16          */
    double threshold_sigma;  /* Gaussian-equivalent significance, default 6         */
    int32_t threshold_mode;  /* FDAS_THRESH_GAMMA_TAIL (default)                    */
    int32_t norm_mode;       /* FDAS_NORM_MEDIAN (default)                          */
    int32_t norm_block;      /* bins per median block, power of 2 in [16, 8192]; 2048 */
    int64_t max_candidates;  /* device candidate store per search call; 1<<20     */
    int32_t autotune;        /* 1: pick the correlator, seg_len (among 2048, 4096,
                                8192 and the one asked for) and the template chunking,
                                or the tensor-core template order, by timing the
                                correlation at plan creation; 0 (default): as given */
    int32_t use_graph;       /* 1: fdas_search captures each batch's launches into
                                one CUDA graph and replays it (device or pinned
                                series, a non-default stream); 0 (default): direct */
    int32_t correlator;      /* FDAS_CORR_AUTO (default), _FFT or _TENSOR; asking
                                for _TENSOR where it does not apply is FDAS_ERR_ARG */
    int32_t harmonic_mode;   /* FDAS_HARM_TOP (default) or FDAS_HARM_FUNDAMENTAL */
    int32_t interbin;        /* 1: the plane on the half-bin grid (see below);
                                0 (default): whole bins.  Needs n_samples <= 2^23 */
    int32_t template_order;  /* tensor-core correlation: FDAS_TORDER_DEFAULT (0),
                                _Z or _PAIRED (below); other correlators ignore it */
} fdas_opts;

/* One dedispersed time series (one DM trial).  `data` points to n_samples
 * FP32 values (16-byte aligned) in device memory, or in host memory (pinned
 * or pageable), which the search copies to the device itself; it is only
 * read.  n_samples may be the plan's length or that length divided by a
 * power of two (a series decimated in time: same observation, so the same
 * z grid and templates, half the bins per halving), down to 2^10. */
typedef struct {
    const float *data;
    int64_t n_samples;   /* plan's n_samples / 2^d, d >= 0, at least 2^10   */
    int32_t decimation;  /* informational (1 = full time resolution)        */
    uint32_t trial_id;   /* caller's DM-trial id, echoed into candidates    */
} fdas_series;

/* One threshold crossing.  `harm` is the number of summed harmonics h (the
 * stage), (ir, iz) the top-harmonic cell: spectral bin ir, z = (iz-K) z_step;
 * the fundamental is at ir/h.  `power` is S_h, `sigma` its Gaussian-equivalent
 * significance (see fdas_search). */
typedef struct {
    uint32_t trial_id;
    uint32_t ir;
    uint16_t iz;
    uint16_t harm;
    float power;
    float sigma;
} fdas_candidate;

/* Read-only description of a plan (all derived from the create arguments). */
typedef struct {
    int64_t n_samples, n_r;
    int32_t n_z, iz0, m_max, m_overlap, seg_len, valid_per_seg, n_seg;
    int32_t n_harm, n_stages, precision, norm_block, threshold_mode;
    double tsamp, z_max, z_step, threshold_sigma;
    double stage_factor[6];   /* G_h = Q^-1(h, Phibar(sigma)) per stage h = 2^s */
    int64_t workspace_bytes;  /* device memory the plan holds                  */
    int32_t z_chunks;         /* template chunks per segment in the correlation */
    int32_t use_graph;
    double tuned_ms;          /* autotune: correlation time per series (ms), else 0 */
    int32_t correlator;       /* FDAS_CORR_FFT, _TENSOR or _TENSOR_SPLIT, as built */
    int32_t harmonic_mode;    /* FDAS_HARM_TOP or FDAS_HARM_FUNDAMENTAL         */
    int32_t interbin;         /* 1: half-bin plane                             */
    int32_t template_order;   /* FDAS_TORDER_Z or _PAIRED as built (tensor-core
                                 correlation), 0 for the FFT correlator          */
    int64_t plane_cols;       /* columns of the power plane: N_r or 2 N_r      */
} fdas_plan_info;

typedef struct fdas_plan fdas_plan;

/* Fill *opts with the defaults listed in fdas_opts. */
void fdas_opts_default(fdas_opts *opts);

/*
 * Build a search plan on the current device: geometry, the frequency-domain
 * template bank and all device workspace for one series at a time (two
 * power planes, so consecutive series overlap).
 *
 * Templates (paper §2.1 matched filter; template formula is a reading): the
 * response of a sinusoid whose frequency drifts by z bins over the
 * observation, rho(q,z) = int_0^1 exp(2 pi i [(q - z/2)u + z u^2/2]) du,
 * evaluated in FP64 on the GPU from Fresnel integrals; g_z[e] =
 * conj(rho(e,z))/sqrt(E_z) for |e| <= m(z), E_z = sum_e |rho(e,z)|^2, placed
 * circularly in seg_len points, transformed with an FP64 DFT, divided by
 * seg_len and stored at the plan's precision.
 *
 * n_samples: power of 2 in [2^10, 2^24]. tsamp: sampling time in s (> 0,
 * informational). z_max >= 0, z_step > 0 with z_max/z_step an integer and
 * n_z <= 65535. seg_len: power of 2 in [1024, 16384], larger than
 * 2*m_overlap + 64 where m_overlap = m(z_max) rounded up to a multiple of 8;
 * 16384 only with the tensor-core correlation, whose direct sum has no
 * segments (FDAS_ERR_UNSUPPORTED for the overlap-save correlator).
 * n_harm in {1,2,4,8,16,32}.  opts may be NULL (defaults).
 * On success *out owns device memory until fdas_plan_destroy.
 * Errors: FDAS_ERR_ARG, FDAS_ERR_UNSUPPORTED, FDAS_ERR_OOM, FDAS_ERR_CUDA
 * (nothing is leaked).
 * Synchronises the device before returning.
 */
fdas_status fdas_plan_create(fdas_plan **out, int64_t n_samples, double tsamp,
                             double z_max, double z_step, int32_t seg_len,
                             int32_t n_harm, const fdas_opts *opts);

/* Release a plan (NULL is ignored).  Synchronises the plan's streams. */
void fdas_plan_destroy(fdas_plan *plan);

/* Copy the plan description into *info (host). */
fdas_status fdas_plan_get_info(const fdas_plan *plan, fdas_plan_info *info);

/*
 * Full search of a batch of series: for each series, R2C FFT, median
 * normalisation, overlap-save correlation with every template, |.|^2 power
 * plane with FP64 mean/std, harmonic sum and threshold (the data-parallel hot
 * path of the paper's FDAS, §2.1-§2.2).
 *
 * batch: host array of n_series descriptors.
 * cands: caller-owned buffer (host or device) for `capacity` entries.
 * n_found: host; receives the total number of threshold crossings.
 * Candidates are every cell with S_h > T_h (strict), h = 1,2,4..H, ordered by
 * (trial_id, harm, iz, ir).  T_h = mean * G_h (GAMMA_TAIL: G_h inverts the
 * Gamma(h,1) upper tail at Phibar(threshold_sigma)) or h*mean +
 * threshold_sigma*sqrt(h)*std (MEAN_PLUS_KSIGMA), with mean/std of the
 * series' own plane.  sigma = Phibar^-1(Q(h, S/mean)) or
 * (S - h mean)/(sqrt(h) std).
 * Blocking: returns after the results are in `cands` (fdas_search_async
 * below is the stream-ordered form).
 * Errors: FDAS_ERR_ARG; FDAS_ERR_NONFINITE (a series holds NaN/Inf, or
 * a power |X_k|^2 of its spectrum exceeds the FP32 range, about 3.4e38, as
 * for samples of about 1e20 at N = 2^23: no candidates are returned); FDAS_ERR_CAND_OVERFLOW (more crossings than
 * `capacity` but no more than the plan's max_candidates: *n_found is the true
 * total and the first `capacity` entries in the order above are written);
 * FDAS_ERR_CAND_STORE_FULL (more crossings than the plan's max_candidates:
 * the device store kept only some of them, in an order that depends on
 * scheduling, so no entry is written; *n_found is the true total; search
 * again with a larger max_candidates or a higher threshold); FDAS_ERR_CUDA.
 * FDAS_ERR_CAND_STORE_FULL takes precedence over FDAS_ERR_CAND_OVERFLOW.
 */
fdas_status fdas_search(fdas_plan *plan, const fdas_series *batch,
                        int32_t n_series, fdas_candidate *cands,
                        int64_t capacity, int64_t *n_found, void *stream);

/*
 * The same search, stream-ordered: every step is queued on `stream` and
 * the call returns without waiting for the device; the caller synchronises
 * the stream (or waits on an event recorded after the call) before reading
 * the results.  It computes what fdas_search computes (same candidates,
 * same order, same statuses), with the count and the status decided on the
 * device:
 *   cands:   device memory or page-locked host memory for `capacity`
 *            entries (written by the device directly);
 *   n_found: device or page-locked host int64, receives the total number
 *            of crossings (0 after a NONFINITE or TIMEOUT status);
 *   status:  device or page-locked host int32, receives the fdas_status
 *            fdas_search would have returned for this batch (FDAS_OK,
 *            FDAS_ERR_CAND_OVERFLOW, FDAS_ERR_CAND_STORE_FULL,
 *            FDAS_ERR_NONFINITE or FDAS_ERR_TIMEOUT, with the same meaning
 *            for `cands` and `n_found`).
 * The series may be in device or host memory as for fdas_search; a series
 * in pageable host memory makes its copy, and so the call, wait for it.
 * The series and the three outputs must stay valid until the stream has
 * completed the search (`batch`, the descriptor array, is read during the
 * call only).
 * The return value covers only what the host can check at the call:
 * FDAS_OK (everything queued), FDAS_ERR_ARG (also: cands, n_found or status
 * in pageable memory, or tracing enabled with fdas_profile_enable), or
 * FDAS_ERR_CUDA (a launch failed).
 * The candidates are ordered on the device without knowing their number on
 * the host, so the sort network is queued for up to the plan's
 * max_candidates records and its unused steps return at once (about 40
 * launches for max_candidates = 2^20).
 * The plan's buffers are reused by the next search: calls on one plan must
 * be ordered by the caller (one stream, or a synchronisation in between).
 * A call with more series than any earlier call on the plan first grows the
 * plan's per-trial buffers, which waits for the device once.
 */
fdas_status fdas_search_async(fdas_plan *plan, const fdas_series *batch,
                              int32_t n_series, fdas_candidate *cands,
                              int64_t capacity, int64_t *n_found,
                              int32_t *status, void *stream);

/* ---------------------------------------------------------------------
 * Candidate refinement with the Fourier-interpolated power.
 *
 * The search grid samples r in whole bins and z in steps of z_step; a
 * signal between grid points loses power to the grid (the paper's §2.1
 * matched filter evaluated off-grid).  For continuous (r, z), with k0 =
 * floor(r + 1/2), delta = r - k0 and m = 32 + ceil(|z|/2) (at most 255):
 *   F(r, z) = sum_{e=-m..m} X_{k0+e} conj(rho(delta - e, z)),   P = |F|^2,
 * rho the unnormalised response above (so a signal c rho(r0 - k, z0) gives
 * P(r0, z0) ~ |c|^2 at any z0), bins outside [0, N_r) counted as 0.  The
 * integrals are Gauss-Legendre sums with 512 nodes, FP32 arithmetic.  The
 * window is held fixed when differentiating.
 * `spectrum` is always FP32 complex (N_r float pairs, device), e.g. the
 * output of fdas_spectrum on an FP32 plan.
 * --------------------------------------------------------------------- */
typedef struct {
    double r;           /* spectral bin (continuous)                       */
    double z;           /* drift in bins over the observation               */
    uint32_t trial_id;  /* echoed into the result                           */
    uint32_t reserved;
} fdas_seed;

typedef struct {
    double r, z;        /* refined location                                 */
    float power;        /* P(r, z)                                          */
    float dpdr, dpdz;   /* gradient at the refined location                 */
    int32_t steps;      /* accepted ascent steps                            */
    uint32_t trial_id;
    uint32_t reserved;
} fdas_refined;

/* P at n points; rz: device double[n][2] (r, z); power: device float[n];
 * grad_rz: device float[n][2] (dP/dr, dP/dz) or NULL.  Asynchronous. */
fdas_status fdas_fourier_power(fdas_plan *plan, const float *spectrum,
                               const double *rz, int32_t n, float *power,
                               float *grad_rz, void *stream);

/* Backward of fdas_fourier_power for an upstream gradient g_s = dL/dP_s
 * (device float[n]): adds sum_s g_s * 2 F_s rho(r_s - k, z_s) to
 * grad_spectrum[k] (device float[N_r][2], complex; the gradient of a real
 * loss with respect to a complex input in the convention of PyTorch,
 * dL/dRe + i dL/dIm), if not NULL, and writes g_s * (dP/dr, dP/dz) to grad_rz
 * (device double[n][2]), if not NULL.  Asynchronous; atomically accumulating
 * (the summation order of overlapping windows is not fixed). */
fdas_status fdas_fourier_power_backward(fdas_plan *plan, const float *spectrum,
                                        const double *rz, int32_t n,
                                        const float *grad_power,
                                        float *grad_spectrum, double *grad_rz,
                                        void *stream);

/* Refine n seeds by n_steps of gradient ascent on P(r, z) with
 * backtracking (one point per CTA; steps along the gradient in the scaled
 * coordinates (r, z/4), shortened fourfold on a decrease, lengthened 1.5
 * times on an increase; stops early when no step increases P).  seeds and
 * out may be host or device memory.  Blocking. */
fdas_status fdas_refine(fdas_plan *plan, const float *spectrum,
                        const fdas_seed *seeds, int32_t n, int32_t n_steps,
                        fdas_refined *out, void *stream);

/* ---------------------------------------------------------------------
 * Stage entry points: one step of the path each, on device buffers, so each
 * step can be checked on its own.  All are asynchronous on `stream`.
 * --------------------------------------------------------------------- */

/* Element type of spectra (complex pairs) and planes at each precision:
 *   FDAS_FP32: float2 spectrum, float plane
 *   FDAS_BF16: __nv_bfloat162 spectrum, __nv_bfloat16 plane
 *   FDAS_FP16: __half2 spectrum, __half plane holding P/16 (range).       */

/*
 * R2C FFT + median normalisation of one series.  X_k = sum_n x_n
 * exp(-2 pi i k n/N) for k in [0, N_r), X_0 set to 0; per block of
 * norm_block bins the median mu_b of |X_k|^2 (block 0 without k = 0; the mean
 * of the two middle values for an even count) gives X'_k = X_k sqrt(ln2/mu_b)
 * (0 when mu_b = 0).  Exponential noise has median ln2 times its mean, so
 * white noise leaves with unit mean power.
 * series: device, N floats.  spectrum_out: device, N_r complex elements of
 * the plan's precision.  medians_out: device float[N_r / norm_block] or NULL.
 * Non-finite input is not reported by this call (a NaN or Inf propagates
 * into the spectrum); fdas_search reports it as FDAS_ERR_NONFINITE.
 */
fdas_status fdas_spectrum(fdas_plan *plan, const float *series,
                          void *spectrum_out, float *medians_out, void *stream);

/*
 * Overlap-save correlation and power plane of one normalised spectrum:
 * P[iz][r] = |sum_{|e|<=m(z_iz)} X'_{r-e} g_z[e]|^2 for r in [0, N_r), with
 * X'_k = 0 outside [0, N_r), computed per segment of seg_len bins (forward
 * FFT, product with the template bank, inverse FFT, keep the valid part).
 * spectrum: device, N_r complex elements (plan precision).  plane_out:
 * device, n_z * N_r elements (plan precision, row-major, r contiguous).
 * stats_out: device double[2] = {mean, population std} of P in FP64 (may be
 * NULL).
 */
fdas_status fdas_power_plane(fdas_plan *plan, const void *spectrum,
                             void *plane_out, double *stats_out, void *stream);
/* (With interbinning, plane_out holds n_z * 2 N_r elements: the half-bin
 * plane, and stats_out its mean/std.) */

/*
 * The complex correlation itself, F[iz][r] = sum_{|e|<=m(z_iz)} X'_{r-e}
 * g_z[e] for r in [0, N_r) (the same correlator as fdas_power_plane, before
 * |.|^2; the input of interbinning).  spectrum: device, N_r complex elements
 * (plan precision).  corr_out: device, n_z * N_r complex elements of the
 * plan precision (FP16 unscaled).  Any plan.  Asynchronous.
 */
fdas_status fdas_correlation_plane(fdas_plan *plan, const void *spectrum,
                                   void *corr_out, void *stream);

/*
 * Harmonic sums of a plane, written out (for checking; the search itself
 * never stores them).  Top-harmonic indexing: for the cell (ir, iz), o =
 * iz - iz0, harmonic j of H reads (iz0 + sign(o) floor((|o| j + H/2)/H),
 * floor((ir j + H/2)/H)); stage h = 2^s sums the harmonics j = kH/h, k=1..h.
 * plane: device (plan precision).  sums_out: device float[n_stages][n_z][N_r]
 * (plane_cols columns with interbinning).
 */
fdas_status fdas_harmonic_sums(fdas_plan *plan, const void *plane,
                               float *sums_out, void *stream);

/*
 * Harmonic sum + threshold of one plane with given statistics.
 * stats: device double[2] {mean, std} (e.g. from fdas_power_plane).
 * cands/capacity/n_found and the statuses FDAS_ERR_CAND_OVERFLOW /
 * FDAS_ERR_CAND_STORE_FULL as in fdas_search (one trial, id `trial_id`).
 * Blocking.
 */
fdas_status fdas_threshold(fdas_plan *plan, const void *plane,
                           const double *stats, uint32_t trial_id,
                           fdas_candidate *cands, int64_t capacity,
                           int64_t *n_found, void *stream);

/*
 * The template bank as the plan holds it.
 * taps_out: host double[2 * sum_iz (2 m(z_iz) + 1)] or NULL -- the FP64
 *   taps g_z[e] (re, im) for iz = 0.., e = -m..m, concatenated.
 * energy_out: host double[n_z] or NULL -- E_z.
 * bank_out: device, n_z * seg_len complex elements of the plan precision or
 *   NULL -- the stored frequency-domain bank (FP16 holds seg_len times it).
 * Blocking.
 */
fdas_status fdas_template_bank(fdas_plan *plan, double *taps_out,
                               double *energy_out, void *bank_out,
                               void *stream);

/*
 * Allocation-free spectrum (no counterpart in the paper; an addition for
 * callers that must not allocate device memory when they call in, such as a
 * real-time pipeline that reserves all of its GPU memory up front and forbids
 * allocation afterwards, or a host whose device memory is handed out by
 * another allocator that must not be bypassed).
 *
 * Computes exactly what fdas_spectrum computes (R2C FFT, X_0 = 0, median
 * normalisation with blocks of norm_block bins) without a plan: the FFT
 * intermediates live in a fixed array of device memory defined by the
 * library, 2^20 complex FP32 values (8 MiB) plus a flag word, which every
 * device that loads the library keeps reserved until the process exits.
 * The call allocates nothing and calls no allocating routine.
 *
 * series: device, n_samples floats, 16-byte aligned.  n_samples: power of
 * two in [2^10, 2^20]; longer series are rejected with FDAS_ERR_ARG (the fixed
 * array holds at most 2^20 samples).  precision, norm_mode, norm_block as in
 * fdas_opts.  spectrum_out: device, n_samples/2 complex elements of
 * `precision`.  medians_out: device float[n_samples/2 / min(norm_block,
 * n_samples/2)] or NULL.  Asynchronous on `stream`.
 *
 * The first call on a device looks up the array's device address and caches
 * it; make that first call before any stream capture.  All calls share the
 * one array and each call overwrites what the previous left there, so calls
 * whose work may overlap on the GPU (different streams without ordering, or
 * several host threads) race with one another: order them on one stream.
 * Like fdas_spectrum, it does not report non-finite input (a NaN or Inf in
 * the series propagates into the spectrum; fdas_search reports it).
 */
fdas_status fdas_spectrum_static(const float *series, int64_t n_samples,
                                 int32_t precision, int32_t norm_mode,
                                 int32_t norm_block, void *spectrum_out,
                                 float *medians_out, void *stream);

/* ---------------------------------------------------------------------
 * Tracing: per-kernel-group launch counts (always kept) and CUDA-event
 * durations (kept while enabled).  While tracing is enabled fdas_search
 * runs every group on the caller's stream (otherwise the harmonic sum of one
 * series runs on a second stream beside the next series), so that each
 * event interval holds one group's kernels only.
 * Groups: [0] R2C FFT + normalisation, [1] fused correlation/power,
 * [2] statistics + harmonic sum/threshold, [3] candidate ordering/output.
 * --------------------------------------------------------------------- */
enum { FDAS_PROF_SPECTRUM = 0, FDAS_PROF_CORRELATE = 1, FDAS_PROF_HARMONIC = 2,
       FDAS_PROF_FINISH = 3 };

typedef struct {
    int64_t trials;        /* series searched since the last reset           */
    int64_t launches[4];   /* kernel launches per group                      */
    int64_t timed[4];      /* timed intervals per group                      */
    double ms[4];          /* summed event-timed milliseconds per group      */
} fdas_profile;

/* Reset the counters; on != 0 also times every group of later fdas_search
 * calls with CUDA events (a few microseconds per series). */
fdas_status fdas_profile_enable(fdas_plan *plan, int32_t on);

/* Copy the counters into *out (host). */
fdas_status fdas_profile_read(const fdas_plan *plan, fdas_profile *out);

/* ---------------------------------------------------------------------
 * Failure-path check for the bounded device waits (no counterpart in the
 * paper).  Every kernel that waits for an asynchronous copy (an mbarrier
 * phase) gives up after a bounded number of clock cycles, records the fact
 * in the plan's flag word and returns; the call that launched it then
 * returns FDAS_ERR_TIMEOUT and the plan stays usable.  This call exercises
 * that path without any fault: one CTA arms a barrier for 16 bytes that no
 * copy delivers and waits at most `limit_cycles` SM clock cycles
 * (1 <= limit_cycles <= 2e9, else FDAS_ERR_ARG).  Blocking.  Returns
 * FDAS_ERR_TIMEOUT when the wait gave up (the expected outcome), FDAS_OK if
 * it did not, FDAS_ERR_CUDA on a CUDA error.
 */
fdas_status fdas_selftest_wait_timeout(fdas_plan *plan, int64_t limit_cycles, void *stream);

/* ---------------------------------------------------------------------
 * Incoherent dedispersion: the stage upstream of the search that turns a
 * filterbank into DM-trial series (the paper searches 5925 DM trials, §3,
 * but does not describe this stage; the textbook definition is used).
 *
 * Channel c (0 = top of the band) has frequency f_c = f_top_mhz - c df_mhz.
 * At DM_d = dm_lo + d dm_step (pc cm^-3) its cold-plasma delay relative to
 * the top of the band, in samples, is
 *   Delta(c, d) = floor(K DM_d (f_c^-2 - f_top^-2) / tsamp + 1/2),
 *   K = 4.148808e3 MHz^2 pc^-1 cm^3 s,
 * evaluated once per plan in FP64 with each operation rounded on its own in
 * that order (f_c, 1/f_c^2, 1/f_top^2, DM_d, (K DM_d)(a - b), / tsamp,
 * + 1/2, floor), and the series is
 *   out[d][t] = sum_{c} in[c][t + Delta(c, d)],  t < n_out,
 * with samples at or past n_t counted as 0 (FP32 sums in channel order).
 * --------------------------------------------------------------------- */
typedef struct fdas_dedisp_plan fdas_dedisp_plan;

typedef struct {
    int32_t n_chan, n_dm;
    int64_t n_t, n_out;
    double f_top_mhz, df_mhz, tsamp, dm_lo, dm_step;
    int32_t max_delay;        /* largest Delta(c, d)                           */
    int32_t tile_span;        /* largest delay spread over 32 consecutive DMs  */
    int64_t workspace_bytes;  /* device memory the plan holds (delay table)   */
} fdas_dedisp_info;

/* n_chan in [1, 65536], n_dm in [1, 65536], 1 <= n_out <= n_t,
 * n_chan * n_t <= 2^36, tsamp > 0, f_top_mhz > 0, df_mhz > 0 with the lowest
 * channel above 0 MHz, dm_lo >= 0, dm_step >= 0: else FDAS_ERR_ARG.  The delay
 * spread of 32 consecutive DM trials must stay below 25088 samples, else
 * FDAS_ERR_UNSUPPORTED.  Computes the delay table on the current device
 * (blocking); *out owns it until fdas_dedisp_plan_destroy. */
fdas_status fdas_dedisp_plan_create(fdas_dedisp_plan **out, int32_t n_chan, int64_t n_t,
                                    double f_top_mhz, double df_mhz, double tsamp,
                                    double dm_lo, double dm_step, int32_t n_dm,
                                    int64_t n_out);
void fdas_dedisp_plan_destroy(fdas_dedisp_plan *plan);
fdas_status fdas_dedisp_get_info(const fdas_dedisp_plan *plan, fdas_dedisp_info *info);

/* The delay table, host int32[n_dm][n_chan]. */
fdas_status fdas_dedisp_delays(const fdas_dedisp_plan *plan, int32_t *delays_out);

/* filterbank: device float[n_chan][n_t] (channel-major, each channel a time
 * series).  out: device float[n_dm][n_out]; row d is DM trial d, ready to be
 * a fdas_series (16-byte aligned when n_out is a multiple of 4).
 * Asynchronous on `stream`. */
fdas_status fdas_dedisperse(fdas_dedisp_plan *plan, const float *filterbank, float *out,
                            void *stream);

/* The same for 8-bit samples (the usual filterbank format): filterbank is
 * device uint8[n_chan][n_t], 16-byte aligned, with n_t a multiple of 16
 * (else FDAS_ERR_ARG).  The channel sums are exact int32 sums, stored as
 * FP32 (exact: n_chan * 255 < 2^24). */
fdas_status fdas_dedisperse_u8(fdas_dedisp_plan *plan, const uint8_t *filterbank, float *out,
                               void *stream);

/* ---------------------------------------------------------------------
 * Host-side fault injection (no counterpart in the paper): the environment
 * variable FDAS_FAULT, read at every call, makes the library take an error
 * path on purpose, without any fault on the device, so that callers and
 * tests can check how failures are reported and cleaned up:
 *   "alloc:N"   the N-th device allocation made for a plan (counted from
 *               fdas_plan_create, N >= 1; "alloc" means "alloc:1") fails as
 *               if the device were out of memory: FDAS_ERR_OOM, and a failed
 *               fdas_plan_create frees everything it had allocated;
 *   "capacity"  fdas_search / fdas_threshold run with a device candidate
 *               store of one record: two or more crossings give
 *               FDAS_ERR_CAND_STORE_FULL;
 *   "nan_input" fdas_search / fdas_threshold report FDAS_ERR_NONFINITE after
 *               the search, as for a series holding NaN or Inf;
 *   "bad_args"  fdas_plan_create and fdas_search return FDAS_ERR_ARG before
 *               doing anything;
 *   "canary"    (checked build) fdas_search / fdas_search_async write one
 *               byte of the canary guard that follows the plan's power plane,
 *               inside its allocation, after the first correlation: the
 *               call returns FDAS_ERR_BOUNDS naming the buffer;
 *   "bounds"    (checked build) every device bounds limit is one element
 *               lower during fdas_search / fdas_search_async, so that checks
 *               fail at real sites (the accesses they skip were in bounds):
 *               FDAS_ERR_BOUNDS naming the first site.
 * "canary" and "bounds" in an ordinary build: FDAS_ERR_UNSUPPORTED.
 * Unset or empty: no fault.  Any other value: the calls above return
 * FDAS_ERR_ARG naming the value.
 * --------------------------------------------------------------------- */

/* ---------------------------------------------------------------------
 * Checked build (no counterpart in the paper): the same sources compiled
 * with -DFDAS_CHECK_BOUNDS into libfdas_checked.so, the same entry points.
 *  - Device bounds checks at the data-dependent accesses of the harmonic
 *    sums (span copies, top-row loads, sums stores, the gathered rows of the
 *    fundamental-indexed sum), of the tensor-core correlation (template
 *    image and spectrum window copies, the MMA rows inside the window,
 *    plane / F / edge stores) and of the candidate ordering.  A failed check
 *    records itself and skips its access; nothing traps.
 *  - Every device buffer of a search plan lies between two 256-byte guards
 *    of canary bytes (fdas_plan_info.workspace_bytes counts the buffers
 *    only).
 *  - After each launch group (the spectrum, correlation and harmonic sum of
 *    each series, the candidate ordering, plan creation and each stage
 *    entry point) the call waits for the device and returns FDAS_ERR_BOUNDS
 *    on the first failed check or overwritten guard byte, with
 *    fdas_last_error() naming the launch group, the site (or buffer) and the
 *    range.  Every call is therefore blocking, fdas_search_async included,
 *    and graph replay is checked after the whole graph.
 * It is a debugging build: slower, and its logs are per process (two plans
 * used at once from two threads may see each other's failures).
 * --------------------------------------------------------------------- */

/* 1 when this library is the checked build, else 0. */
int32_t fdas_checked_build(void);

/* Thread-local message describing the last failed call ("" if none). */
const char *fdas_last_error(void);

/* Library version string. */
const char *fdas_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDAS_H */
