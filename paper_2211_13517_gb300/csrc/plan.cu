// C ABI of the FDAS library: plan construction, the search driver and the
// stage entry points (declared in include/fdas.h).
#include "fdas_internal.cuh"
#include "check.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

namespace fdas {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

fdas_status cuda_status(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? FDAS_ERR_OOM : FDAS_ERR_CUDA;
}

static fdas_status arg_error(const std::string &msg) {
    set_error(msg);
    return FDAS_ERR_ARG;
}

// ---------------------------------------------------------------------------
// host-side fault injection: FDAS_FAULT = alloc[:N] | capacity | nan_input |
// bad_args, and in checked builds canary | bounds, read at every call
// (semantics in include/fdas.h).  Nothing is injected on the device: each
// fault makes the host take the error path the real failure would take, or
// (canary, bounds) writes one byte inside a guard or lowers the device
// bounds limits, both inside the allocations.
// ---------------------------------------------------------------------------
enum {
    kFaultNone = 0,
    kFaultAlloc,
    kFaultCapacity,
    kFaultNan,
    kFaultArgs,
    kFaultCanary,
    kFaultBounds,
    kFaultUnknown
};

struct Fault {
    int kind = kFaultNone;
    int64_t n = 0;           // alloc: which allocation fails (1-based)
    std::string text;
};

static Fault injected_fault() {
    Fault f;
    const char *s = std::getenv("FDAS_FAULT");
    if (!s || !*s) return f;
    f.text = s;
    if (std::strncmp(s, "alloc", 5) == 0 && (s[5] == 0 || s[5] == ':')) {
        f.kind = kFaultAlloc;
        f.n = s[5] == ':' ? std::atoll(s + 6) : 1;
        if (f.n < 1) f.kind = kFaultUnknown;
    } else if (std::strcmp(s, "capacity") == 0) {
        f.kind = kFaultCapacity;
    } else if (std::strcmp(s, "nan_input") == 0) {
        f.kind = kFaultNan;
    } else if (std::strcmp(s, "bad_args") == 0) {
        f.kind = kFaultArgs;
    } else if (std::strcmp(s, "canary") == 0) {
        f.kind = kFaultCanary;
    } else if (std::strcmp(s, "bounds") == 0) {
        f.kind = kFaultBounds;
    } else {
        f.kind = kFaultUnknown;
    }
    return f;
}

// FDAS_ERR_ARG for the bad_args fault and for an unknown FDAS_FAULT value;
// FDAS_ERR_UNSUPPORTED for the faults of checked builds in an ordinary one
static fdas_status fault_args_check(const Fault &f) {
    if (f.kind == kFaultArgs) return arg_error("injected fault (FDAS_FAULT=bad_args)");
    if (f.kind == kFaultUnknown)
        return arg_error("FDAS_FAULT=" + f.text +
                         ": unknown fault (alloc[:N] with N >= 1, capacity, nan_input, bad_args, "
                         "canary, bounds)");
#ifndef FDAS_CHECK_BOUNDS
    if (f.kind == kFaultCanary || f.kind == kFaultBounds) {
        set_error("FDAS_FAULT=" + f.text + " needs the checked build (libfdas_checked.so)");
        return FDAS_ERR_UNSUPPORTED;
    }
#endif
    return FDAS_OK;
}

// ---------------------------------------------------------------------------
// threshold factors: G_h = Q^-1(h, Phibar(sigma)), Q the regularised upper
// incomplete gamma function of integer order h (Poisson form, log scale),
// solved by bisection in FP64 on the host at plan time.
// ---------------------------------------------------------------------------
static double log_q_int(int h, double x) {
    if (x <= 0.0) return 0.0;
    const double lx = std::log(x);
    std::vector<double> lt(h);
    double lf = 0.0, mx = -1e300;
    for (int k = 0; k < h; ++k) {
        if (k > 0) lf += std::log((double)k);
        lt[k] = k * lx - lf;
        mx = std::max(mx, lt[k]);
    }
    double s = 0.0;
    for (int k = 0; k < h; ++k) s += std::exp(lt[k] - mx);
    return -x + mx + std::log(s);
}

static double gamma_tail_factor(int h, double sigma) {
    const double lp = std::log(0.5 * std::erfc(sigma / std::sqrt(2.0)));
    double lo = 0.0, hi = 1.0;
    while (log_q_int(h, hi) > lp) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (log_q_int(h, mid) > lp) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// ---------------------------------------------------------------------------
// checked builds (-DFDAS_CHECK_BOUNDS): every device buffer of a plan is
// allocated with kGuardBytes of canary bytes on each side.  After each launch
// group the library waits for the device and reads the device bounds logs of
// the checked kernels (check.cuh) and every guard; the first failure is
// reported as FDAS_ERR_BOUNDS, naming the launch group, and the logs and
// guards are reset.
// ---------------------------------------------------------------------------
#ifdef FDAS_CHECK_BOUNDS
constexpr size_t kGuardBytes = 256;   // each side: the buffer keeps 256-byte alignment
constexpr unsigned char kCanary = 0xA5;

cudaError_t bounds_take_harmonic(BoundsLog *out);
cudaError_t bounds_arm_harmonic(int64_t shrink);
cudaError_t bounds_take_correlate_tc(BoundsLog *out);
cudaError_t bounds_arm_correlate_tc(int64_t shrink);

struct GuardDesc {
    const unsigned char *lo, *hi;   // the kGuardBytes before and after a buffer
};

// one CTA per buffer: the smallest (buffer, guard byte) whose byte is not
// the canary, guard bytes counted from the start of the one before the buffer
__global__ void canary_check_kernel(const GuardDesc *g, int n, unsigned long long *first) {
    const int b = blockIdx.x;
    if (b >= n) return;
    for (int i = threadIdx.x; i < 2 * (int)kGuardBytes; i += blockDim.x) {
        const unsigned char v = i < (int)kGuardBytes ? g[b].lo[i] : g[b].hi[i - (int)kGuardBytes];
        if (v != kCanary) atomicMin(first, ((unsigned long long)b << 32) | (unsigned)i);
    }
}
#endif

// cudaFree of a buffer that dalloc made (its guards included)
static void dfree(Plan &p, void *ptr) {
    if (ptr == nullptr) return;
#ifdef FDAS_CHECK_BOUNDS
    for (size_t i = 0; i < p.pools->guards.size(); ++i) {
        if (p.pools->guards[i].base + kGuardBytes == (char *)ptr) {
            cudaFree(p.pools->guards[i].base);
            p.pools->guards.erase(p.pools->guards.begin() + (std::ptrdiff_t)i);
            return;
        }
    }
#else
    (void)p;
#endif
    cudaFree(ptr);
}

static void free_plan_memory(Plan *p) {
    dfree(*p, p->bank);
    dfree(*p, p->taps);
    dfree(*p, p->energy);
    dfree(*p, p->tap_off);
    dfree(*p, p->tap_m);
    dfree(*p, p->fft_a);
    dfree(*p, p->fft_b);
    dfree(*p, p->spec_pad);
    dfree(*p, p->corr);
    dfree(*p, p->tc_chunks);
    dfree(*p, p->tc_bank);
    dfree(*p, p->tc_inv_energy);
    dfree(*p, p->tc_edges);
    dfree(*p, p->spec_hi);
    dfree(*p, p->spec_lo);
    for (int b = 0; b < 2; ++b) {
        dfree(*p, p->plane[b]);
        dfree(*p, p->partials[b]);
        if (p->ev_conv[b]) cudaEventDestroy(p->ev_conv[b]);
        if (p->ev_hsum[b]) cudaEventDestroy(p->ev_hsum[b]);
    }
    dfree(*p, p->stats);
    dfree(*p, p->rank_ids);
    dfree(*p, p->cand);
    dfree(*p, p->cand_count);
    dfree(*p, p->flags);
    dfree(*p, p->out_stage);
    dfree(*p, p->async_res);
    dfree(*p, p->stage);
    dfree(*p, p->stage2);
    for (int b = 0; b < 2; ++b) {
        if (p->ev_copied[b]) cudaEventDestroy(p->ev_copied[b]);
        if (p->ev_consumed[b]) cudaEventDestroy(p->ev_consumed[b]);
    }
    if (p->cpy) cudaStreamDestroy(p->cpy);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    dfree(*p, p->gl_nodes);
    dfree(*p, p->ref_seeds);
    dfree(*p, p->ref_out);
    if (p->host_small) cudaFreeHost(p->host_small);
    for (cudaEvent_t e : p->pools->events) cudaEventDestroy(e);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->hi) cudaStreamDestroy(p->hi);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
}

// a device buffer of the plan, named for the checked build's reports
template <class T>
static fdas_status dalloc(Plan &p, T **ptr, size_t bytes, const char *name) {
    ++p.n_allocs;
    const Fault f = injected_fault();
    if (f.kind == kFaultAlloc && p.n_allocs == f.n) {
        *ptr = nullptr;
        set_error("cudaMalloc(" + std::to_string(bytes) + " bytes): injected fault (FDAS_FAULT=" +
                  f.text + ")");
        return FDAS_ERR_OOM;
    }
#ifdef FDAS_CHECK_BOUNDS
    char *base = nullptr;
    cudaError_t e = cudaMalloc((void **)&base, bytes + 2 * kGuardBytes);
    if (e == cudaSuccess) {
        e = cudaMemset(base, kCanary, kGuardBytes);
        if (e == cudaSuccess) e = cudaMemset(base + kGuardBytes + bytes, kCanary, kGuardBytes);
        if (e == cudaSuccess) {
            *ptr = reinterpret_cast<T *>(base + kGuardBytes);
            p.pools->guards.push_back({base, bytes, name});
        } else {
            cudaFree(base);
        }
    }
#else
    (void)name;
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
#endif
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(" + std::to_string(bytes) + " bytes) failed: " +
                  cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FDAS_ERR_OOM : FDAS_ERR_CUDA;
    }
    p.ws_bytes += (int64_t)bytes;
    return FDAS_OK;
}

// Checked builds: wait for the device, then report the first failed device
// bounds check and the first overwritten canary byte since the last check as
// FDAS_ERR_BOUNDS (message: `after`, the launch group just queued, and what
// failed), resetting logs and guards.  While the stream is being captured
// into a graph nothing can be read; the check after the graph's launch covers
// its kernels.  Ordinary builds never call it (FDAS_DEBUG_CHECK is empty).
#ifdef FDAS_CHECK_BOUNDS
static fdas_status debug_check(Plan &p, cudaStream_t s, const std::string &after) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    FDAS_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return FDAS_OK;
    FDAS_CUDA_TRY(cudaDeviceSynchronize());
    std::string msg;
    const struct {
        const char *unit;
        cudaError_t (*take)(BoundsLog *);
    } logs[] = {{"harmonic sum", bounds_take_harmonic},
                {"tensor-core correlation", bounds_take_correlate_tc}};
    for (const auto &l : logs) {
        BoundsLog lg{};
        FDAS_CUDA_TRY(l.take(&lg));
        if (lg.failures > 0 && msg.empty())
            msg = "after " + after + ": " + std::to_string(lg.failures) +
                  " failed device bounds check(s) in the " + l.unit + "; the first: " +
                  bounds_site_name(lg.site) + ", elements [" + std::to_string(lg.begin) + ", " +
                  std::to_string(lg.begin + lg.count) + ") against a limit of " +
                  std::to_string(lg.limit);
    }
    const int n = (int)p.pools->guards.size();
    if (n > 0) {
        std::vector<GuardDesc> g(n);
        for (int i = 0; i < n; ++i) {
            const Plan::GuardedBuf &b = p.pools->guards[i];
            g[i].lo = (const unsigned char *)b.base;
            g[i].hi = (const unsigned char *)b.base + kGuardBytes + b.bytes;
        }
        void *dev = nullptr;
        const size_t tb = sizeof(GuardDesc) * (size_t)n;
        FDAS_CUDA_TRY(cudaMalloc(&dev, tb + sizeof(unsigned long long)));
        unsigned long long first = ~0ull;
        auto *dfirst = (unsigned long long *)((char *)dev + tb);
        cudaError_t e = cudaMemcpy(dev, g.data(), tb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dfirst, &first, sizeof(first), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            canary_check_kernel<<<n, 256>>>((const GuardDesc *)dev, n, dfirst);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(&first, dfirst, sizeof(first), cudaMemcpyDeviceToHost);
        cudaFree(dev);
        FDAS_CUDA_TRY(e);
        if (first != ~0ull) {
            const Plan::GuardedBuf &b = p.pools->guards[first >> 32];
            const int64_t i = (int64_t)(first & 0xffffffffu);
            const int64_t off = i < (int64_t)kGuardBytes ? i - (int64_t)kGuardBytes
                                                         : (int64_t)b.bytes + i - (int64_t)kGuardBytes;
            if (msg.empty())
                msg = "after " + after + ": canary of workspace buffer " + b.name + " (" +
                      std::to_string(b.bytes) + " bytes) overwritten at byte offset " +
                      std::to_string(off);
            for (const Plan::GuardedBuf &r : p.pools->guards) {
                FDAS_CUDA_TRY(cudaMemset(r.base, kCanary, kGuardBytes));
                FDAS_CUDA_TRY(cudaMemset(r.base + kGuardBytes + r.bytes, kCanary, kGuardBytes));
            }
            FDAS_CUDA_TRY(cudaDeviceSynchronize());
        }
    }
    if (msg.empty()) return FDAS_OK;
    set_error(msg);
    return FDAS_ERR_BOUNDS;
}
#define FDAS_DEBUG_CHECK(p, s, after) FDAS_TRY(debug_check((p), (s), (after)))
#else
#define FDAS_DEBUG_CHECK(p, s, after) \
    do {                              \
    } while (0)
#endif

// FDAS_FAULT=bounds (checked builds): every device bounds limit is one
// element lower for the duration of one call
struct BoundsShrink {
    bool on = false;
    explicit BoundsShrink(bool want) {
#ifdef FDAS_CHECK_BOUNDS
        if (want) {
            bounds_arm_harmonic(1);
            bounds_arm_correlate_tc(1);
            on = true;
        }
#else
        (void)want;
#endif
    }
    ~BoundsShrink() {
#ifdef FDAS_CHECK_BOUNDS
        if (on) {
            cudaDeviceSynchronize();
            bounds_arm_harmonic(0);
            bounds_arm_correlate_tc(0);
        }
#endif
    }
};

static fdas_status grow_stats(Plan &p, int64_t need) {
    if (need <= p.stats_cap) return FDAS_OK;
    int64_t cap = std::max<int64_t>(need, 2 * p.stats_cap);
    FDAS_CUDA_TRY(cudaDeviceSynchronize());
    dfree(p, p.stats);
    dfree(p, p.rank_ids);
    p.stats = nullptr;
    p.rank_ids = nullptr;
    p.ws_bytes -= p.stats_cap * (int64_t)(sizeof(TrialStats) + sizeof(uint32_t));
    p.stats_cap = 0;
    FDAS_TRY(dalloc(p, &p.stats, sizeof(TrialStats) * (size_t)cap, "stats"));
    FDAS_TRY(dalloc(p, &p.rank_ids, sizeof(uint32_t) * (size_t)cap, "rank_ids"));
    p.stats_cap = cap;
    return FDAS_OK;
}

static int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// correlation grid: z chunks per segment chosen to fill the GPU evenly,
// counting one extra forward FFT per CTA
static int choose_zchunks(const Plan &p, int slots) {
    int best = 1;
    double best_eff = 0.0;
    for (int c = 1; c <= std::min(32, p.n_z); ++c) {
        const int zper = (p.n_z + c - 1) / c;
        const int64_t ctas = (int64_t)p.n_seg * c;
        const int64_t waves = (ctas + slots - 1) / slots;
        const double eff = (double)p.n_seg * p.n_z / ((double)slots * waves * (zper + 1));
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = c;
        }
    }
    return best;
}

// geometry of a series of n samples (the plan's length or a power-of-two
// fraction of it) on the plan's z grid and segment length
static void set_length(Plan &p, int64_t n) {
    p.n_samples = n;
    p.n_r = n / 2;
    p.n_seg = (int)((p.n_r + p.V - 1) / p.V);
    const int lm = ilog2(p.n_r);
    if (p.n_r <= 8192) {
        p.fft_m1 = 1;
        p.fft_m2 = (int)p.n_r;
    } else {
        p.fft_m1 = 1 << (lm / 2);
        p.fft_m2 = 1 << (lm - lm / 2);
    }
}

// the plan's buffers with the geometry of a shorter series
// the correlation (and interbinning) of one series into `plane`, leaving
// plane_partials(v) FP64 partials in `partials`
static fdas_status launch_plane(Plan &v, const void *spec_pad, void *plane, double2 *partials,
                                cudaStream_t s) {
    if (!v.interbin) return launch_correlate(v, spec_pad, plane, partials, s);
    if (v.correlator == FDAS_CORR_TENSOR) return launch_interbin_tc(v, spec_pad, plane, partials, s);
    FDAS_TRY(launch_correlate(v, spec_pad, v.corr, partials, s, true));
    return launch_interbin(v, v.corr, plane, partials, s);
}

static int plane_partials(const Plan &v) {
    if (!v.interbin) return correlate_ctas(v);
    return v.correlator == FDAS_CORR_TENSOR ? interbin_tc_partials(v) : interbin_ctas(v);
}

// the plan as the statistics and harmonic kernels see it: the plane's
// columns (half bins with interbinning) in place of the spectral bins
static Plan harm_view(const Plan &v) {
    Plan h = v;
    h.n_r = plane_cols(v);
    h.interbin = false;
    return h;
}

static Plan plan_view(const Plan &p, int64_t n) {
    Plan v = p;
    set_length(v, n);
    v.n_zchunk = choose_zchunks(v, v.n_sms);
    while (v.n_zchunk > 1 && (int64_t)v.n_seg * v.n_zchunk > p.partials_cap) --v.n_zchunk;
    return v;
}

static fdas_status create(Plan *&out, int64_t n_samples, double tsamp, double z_max, double z_step,
                          int32_t seg_len, int32_t n_harm, const fdas_opts *o) {
    FDAS_TRY(fault_args_check(injected_fault()));
    if (!is_pow2(n_samples) || n_samples < (1 << 10) || n_samples > (1 << 24))
        return arg_error("n_samples must be a power of two in [2^10, 2^24]");
    if (!(tsamp > 0.0) || !std::isfinite(tsamp)) return arg_error("tsamp must be > 0");
    if (!(z_step > 0.0) || !std::isfinite(z_step) || !(z_max >= 0.0) || !std::isfinite(z_max))
        return arg_error("need z_step > 0 and z_max >= 0");
    const double ratio = z_max / z_step;
    const double K = std::round(ratio);
    if (std::fabs(ratio - K) > 1e-9 * std::max(1.0, ratio))
        return arg_error("z_max / z_step must be an integer");
    if (2 * K + 1 > 65535) return arg_error("too many z trials (n_z > 65535)");
    if (!(n_harm == 1 || n_harm == 2 || n_harm == 4 || n_harm == 8 || n_harm == 16 || n_harm == 32))
        return arg_error("n_harm must be one of 1, 2, 4, 8, 16, 32");
    if (!is_pow2(seg_len) || seg_len < 1024 || seg_len > 16384)
        return arg_error("seg_len must be a power of two in [1024, 16384]");
    if (o->precision != FDAS_FP32 && o->precision != FDAS_BF16 && o->precision != FDAS_FP16)
        return arg_error("unknown precision");
    if (o->threshold_mode != FDAS_THRESH_GAMMA_TAIL && o->threshold_mode != FDAS_THRESH_MEAN_PLUS_KSIGMA)
        return arg_error("unknown threshold_mode");
    if (o->norm_mode != FDAS_NORM_MEDIAN && o->norm_mode != FDAS_NORM_NONE)
        return arg_error("unknown norm_mode");
    if (!is_pow2(o->norm_block) || o->norm_block < 16 || o->norm_block > 8192)
        return arg_error("norm_block must be a power of two in [16, 8192]");
    if (!(o->threshold_sigma > 0.0) || o->threshold_sigma > 37.0)
        return arg_error("threshold_sigma must be in (0, 37]");
    if (o->max_candidates < 1 || o->max_candidates > (int64_t(1) << 26))
        return arg_error("max_candidates must be in [1, 2^26]");
    if (o->autotune != 0 && o->autotune != 1) return arg_error("autotune must be 0 or 1");
    if (o->use_graph != 0 && o->use_graph != 1) return arg_error("use_graph must be 0 or 1");
    if (o->correlator != FDAS_CORR_AUTO && o->correlator != FDAS_CORR_FFT &&
        o->correlator != FDAS_CORR_TENSOR && o->correlator != FDAS_CORR_TENSOR_SPLIT)
        return arg_error("unknown correlator");
    if (o->correlator == FDAS_CORR_TENSOR_SPLIT && o->precision != FDAS_FP32)
        return arg_error("correlator FDAS_CORR_TENSOR_SPLIT: FDAS_FP32 storage only");
    if (o->correlator == FDAS_CORR_TENSOR_SPLIT && o->interbin)
        return arg_error("correlator FDAS_CORR_TENSOR_SPLIT: no interbinning (use the FFT correlator)");
    if (o->harmonic_mode != FDAS_HARM_TOP && o->harmonic_mode != FDAS_HARM_FUNDAMENTAL)
        return arg_error("unknown harmonic_mode");
    if (o->interbin != 0 && o->interbin != 1) return arg_error("interbin must be 0 or 1");
    if (o->template_order < FDAS_TORDER_DEFAULT || o->template_order > FDAS_TORDER_PAIRED)
        return arg_error("template_order must be FDAS_TORDER_DEFAULT, _Z or _PAIRED");
    // candidate records keep the plane column in 23 bits
    if (o->interbin && n_samples > (1 << 23))
        return arg_error("interbinning takes n_samples <= 2^23");

    Plan *pp = new (std::nothrow) Plan();
    if (!pp) return arg_error("out of host memory");
    Plan &p = *pp;
    p.n_samples = n_samples;
    p.n_r = n_samples / 2;
    p.tsamp = tsamp;
    p.z_max = z_max;
    p.z_step = z_step;
    p.iz0 = (int)K;
    p.n_z = 2 * (int)K + 1;
    p.H = n_harm;
    p.n_stages = ilog2(n_harm) + 1;
    p.prec = o->precision;
    p.norm_mode = o->norm_mode;
    p.norm_block = o->norm_block;
    p.thr_mode = o->threshold_mode;
    p.sigma = o->threshold_sigma;
    p.max_cands = o->max_candidates;
    p.store_cap = p.max_cands;
    p.harm_mode = o->harmonic_mode;
    p.interbin = o->interbin != 0;
    for (int s = 0; s < 6; ++s) p.G[s] = s < p.n_stages ? gamma_tail_factor(1 << s, p.sigma) : 0.0;

    // template half-widths m(z) = 8 + ceil(|z|/2) on the exact grid
    std::vector<int32_t> m(p.n_z);
    std::vector<int64_t> off(p.n_z);
    int64_t acc = 0;
    p.m_max = 0;
    for (int i = 0; i < p.n_z; ++i) {
        const double az = std::fabs((double)(i - p.iz0)) * z_step;
        m[i] = 8 + (int32_t)std::ceil(az / 2.0 - 1e-9);
        p.m_max = std::max(p.m_max, (int)m[i]);
        off[i] = acc;
        acc += 2 * m[i] + 1;
    }
    p.n_taps = acc;
    p.m_ov = (p.m_max + 7) / 8 * 8;
    p.L = seg_len;
    if (seg_len <= 2 * p.m_ov + 64) {
        delete pp;
        return arg_error("seg_len must exceed 2*m_overlap + 64 (m_overlap = " +
                         std::to_string(p.m_ov) + ")");
    }
    p.V = p.L - 2 * p.m_ov;
    set_length(p, n_samples);
    p.use_graph = o->use_graph != 0;

    cudaError_t ce = cudaGetDevice(&p.device);
    if (ce != cudaSuccess) {
        delete pp;
        return cuda_status(ce, "cudaGetDevice");
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    p.n_sms = std::max(1, sms);
    p.n_zchunk = choose_zchunks(p, p.n_sms);
    // partials serve every length the plan accepts (N, N/2, ..., 2^10) and
    // any template chunking up to 32
    p.partials_cap = std::max<int64_t>((int64_t)p.n_seg * 32, 5 * (int64_t)p.n_sms);
    for (int64_t n = n_samples; n >= (1 << 10); n /= 2) {
        Plan v = p;
        set_length(v, n);
        p.partials_cap = std::max<int64_t>(p.partials_cap, (int64_t)v.n_seg * 32);
    }
    // the correlator: the tensor-core GEMM where it applies (16-bit storage,
    // template chunks that fit in shared memory), else overlap-save FFTs
    std::vector<TcChunk> tc_table;
    p.tc_split = o->correlator == FDAS_CORR_TENSOR_SPLIT;
    p.tc_order = o->template_order == FDAS_TORDER_Z ? 0 : 1;
    if (o->correlator != FDAS_CORR_FFT && (p.prec != FDAS_FP32 || p.tc_split)) {
        tc_table = tc_chunk_table(p, m, &p.tc_win, &p.tc_max_ks);
        p.tc_n_ch = (int)tc_table.size();
    }
    {
        std::string why = "the tensor-core correlation takes 16-bit storage (FDAS_BF16/FDAS_FP16)";
        const bool tc_ok = !tc_table.empty() && tc_applicable(p, &why);
        if ((o->correlator == FDAS_CORR_TENSOR || p.tc_split) && !tc_ok) {
            delete pp;
            return arg_error(std::string(p.tc_split ? "correlator FDAS_CORR_TENSOR_SPLIT: "
                                                    : "correlator FDAS_CORR_TENSOR: ") + why);
        }
        p.correlator = (o->correlator != FDAS_CORR_FFT && tc_ok) ? FDAS_CORR_TENSOR : FDAS_CORR_FFT;
        // the overlap-save kernels go up to 8192-point segments; the
        // tensor-core correlation has no segments (seg_len only sizes the
        // frequency-domain template bank), so it takes 16384 as well
        if (seg_len > 8192 && p.correlator != FDAS_CORR_TENSOR) {
            delete pp;
            set_error("seg_len 16384 needs the tensor-core correlation (FDAS_BF16 or FDAS_FP16 "
                      "storage); the overlap-save correlator goes up to 8192");
            return FDAS_ERR_UNSUPPORTED;
        }
        if (p.correlator != FDAS_CORR_TENSOR) {
            tc_table.clear();
            p.tc_n_ch = 0;
        } else {
            p.tc_nbuf = tc_image_buffers(p);
        }
    }

    fdas_status st = FDAS_OK;
    auto fail = [&](fdas_status s) {
        cudaDeviceSynchronize();
        free_plan_memory(pp);
        delete pp;
        return s;
    };
#define PLAN_TRY(expr)                  \
    do {                                \
        st = (expr);                    \
        if (st != FDAS_OK) return fail(st); \
    } while (0)
#define PLAN_CUDA(expr)                                   \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return fail(cuda_status(_e, #expr)); \
    } while (0)

    const size_t cb = cpx_bytes(p.prec), rb = real_bytes(p.prec);
    PLAN_TRY(dalloc(p, &p.bank, cb * (size_t)p.n_z * p.L, "bank"));
    PLAN_TRY(dalloc(p, &p.taps, sizeof(double) * 2 * (size_t)p.n_taps, "taps"));
    PLAN_TRY(dalloc(p, &p.energy, sizeof(double) * p.n_z, "energy"));
    PLAN_TRY(dalloc(p, &p.tap_off, sizeof(int64_t) * p.n_z, "tap_off"));
    PLAN_TRY(dalloc(p, &p.tap_m, sizeof(int32_t) * p.n_z, "tap_m"));
    if (p.fft_m1 > 1) PLAN_TRY(dalloc(p, &p.fft_a, sizeof(float2) * (size_t)p.n_r, "fft_a"));
    PLAN_TRY(dalloc(p, &p.fft_b, sizeof(float2) * (size_t)p.n_r, "fft_b"));
    // 64 elements past the last segment: the tensor-core windows of the last
    // tile read up to 16 elements beyond the zero tail
    const size_t pad_elems = (size_t)p.n_seg * p.V + 2 * (size_t)p.m_ov + 64;
    PLAN_TRY(dalloc(p, &p.spec_pad, cb * pad_elems, "spec_pad"));
    p.spec_pad_elems = (int64_t)pad_elems;
    for (int b = 0; b < 2; ++b) {
        PLAN_TRY(dalloc(p, &p.plane[b], rb * (size_t)p.n_z * (size_t)plane_cols(p),
                        b == 0 ? "plane[0]" : "plane[1]"));
        PLAN_TRY(dalloc(p, &p.partials[b], sizeof(double2) * (size_t)p.partials_cap,
                        b == 0 ? "partials[0]" : "partials[1]"));
        PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_conv[b], cudaEventDisableTiming));
        PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_hsum[b], cudaEventDisableTiming));
    }
    // interbinning: the FFT correlators write the complex plane for the
    // interbinning kernel; the tensor-core epilogue writes the half-bin plane
    // itself and needs only its edge table (allocated below)
    if (p.interbin && p.correlator != FDAS_CORR_TENSOR)
        PLAN_TRY(dalloc(p, &p.corr, cb * (size_t)p.n_z * (size_t)p.n_r, "corr"));
    PLAN_TRY(grow_stats(p, 64));
    const int64_t rec_cap = next_pow2(p.max_cands);
    PLAN_TRY(dalloc(p, &p.cand, sizeof(CandRec) * (size_t)rec_cap, "cand"));
    PLAN_TRY(dalloc(p, &p.cand_count, sizeof(unsigned long long), "cand_count"));
    PLAN_TRY(dalloc(p, &p.flags, sizeof(unsigned int), "flags"));
    PLAN_TRY(dalloc(p, &p.out_stage, sizeof(fdas_candidate) * (size_t)p.max_cands, "out_stage"));
    PLAN_TRY(dalloc(p, &p.async_res, sizeof(AsyncResult), "async_res"));
    PLAN_TRY(dalloc(p, &p.stage, sizeof(float) * (size_t)p.n_samples, "stage"));
    PLAN_TRY(dalloc(p, &p.stage2, sizeof(float) * (size_t)p.n_samples, "stage2"));
    {
        // the copy stream at the highest priority: the copy kernel's CTAs
        // take the next free slots ahead of the running search's
        int least = 0, greatest = 0;
        PLAN_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        PLAN_CUDA(cudaStreamCreateWithPriority(&p.cpy, cudaStreamNonBlocking, greatest));
    }
    PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_start, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_copied[b], cudaEventDisableTiming));
        PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_consumed[b], cudaEventDisableTiming));
    }
    PLAN_CUDA(cudaMallocHost((void **)&p.host_small, 4 * sizeof(unsigned long long)));
    // the harmonic sum of one series runs on the lowest-priority stream
    // beside the spectrum and correlation of the next on the highest: as the
    // harmonic sum's CTAs retire, the block scheduler places the correlation's
    // persistent CTAs first, and the harmonic CTAs fill what they leave of
    // each SM, so the two kernels share the SMs instead of running in turn
    {
        int least = 0, greatest = 0;
        PLAN_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        PLAN_CUDA(cudaStreamCreateWithPriority(&p.aux, cudaStreamNonBlocking, least));
        PLAN_CUDA(cudaStreamCreateWithPriority(&p.hi, cudaStreamNonBlocking, greatest));
        PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_fork, cudaEventDisableTiming));
        PLAN_CUDA(cudaEventCreateWithFlags(&p.ev_join, cudaEventDisableTiming));
    }

    {
        const std::vector<float2> gl = gauss_legendre_01(refine_nodes());
        PLAN_TRY(dalloc(p, &p.gl_nodes, sizeof(float2) * gl.size(), "gl_nodes"));
        PLAN_CUDA(cudaMemcpy(p.gl_nodes, gl.data(), sizeof(float2) * gl.size(),
                             cudaMemcpyHostToDevice));
    }
    PLAN_CUDA(cudaMemset(p.spec_pad, 0, cb * pad_elems));
    PLAN_CUDA(cudaMemcpy(p.tap_off, off.data(), sizeof(int64_t) * p.n_z, cudaMemcpyHostToDevice));
    PLAN_CUDA(cudaMemcpy(p.tap_m, m.data(), sizeof(int32_t) * p.n_z, cudaMemcpyHostToDevice));
    PLAN_TRY(launch_template_bank(p, p.aux));
    if (p.correlator == FDAS_CORR_TENSOR) {
        const int64_t img = tc_bank_bytes(tc_table);
        PLAN_TRY(dalloc(p, &p.tc_chunks, sizeof(TcChunk) * tc_table.size(), "tc_chunks"));
        if (p.tc_split) {
            p.tc_bank_lo = img;
            p.tc_split_elems = (int64_t)pad_elems;
            PLAN_TRY(dalloc(p, &p.spec_hi, 4 * pad_elems, "spec_hi"));
            PLAN_TRY(dalloc(p, &p.spec_lo, 4 * pad_elems, "spec_lo"));
        }
        PLAN_TRY(dalloc(p, &p.tc_bank, (size_t)img * (p.tc_split ? 2 : 1), "tc_bank"));
        p.tc_img_bytes = img * (p.tc_split ? 2 : 1);
        PLAN_TRY(dalloc(p, &p.tc_inv_energy, sizeof(float) * (size_t)p.n_z, "tc_inv_energy"));
        if (p.interbin) PLAN_TRY(dalloc(p, &p.tc_edges, (size_t)tc_edge_bytes(p), "tc_edges"));
        PLAN_CUDA(cudaMemcpyAsync(p.tc_chunks, tc_table.data(), sizeof(TcChunk) * tc_table.size(),
                                  cudaMemcpyHostToDevice, p.aux));
        PLAN_TRY(launch_tc_bank(p, p.aux));
    }
    PLAN_CUDA(cudaStreamSynchronize(p.aux));
    PLAN_CUDA(cudaDeviceSynchronize());
#ifdef FDAS_CHECK_BOUNDS
    PLAN_TRY(debug_check(p, p.aux, "plan creation"));
#endif
#undef PLAN_TRY
#undef PLAN_CUDA
    out = pp;
    return FDAS_OK;
}

// pointer kinds
// the address a kernel reads or writes `ptr` through: device (or managed) memory as
// it is, page-locked host memory by its mapped device address; NULL for
// memory the device cannot reach
static void *device_view(void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ptr;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

static bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// sort/convert the stored candidates and copy them out; blocking
static fdas_status collect(Plan &p, fdas_candidate *cands, int64_t capacity, int64_t *n_found,
                           cudaStream_t s) {
    FDAS_CUDA_TRY(cudaMemcpyAsync(p.host_small, p.cand_count, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, s));
    FDAS_CUDA_TRY(cudaMemcpyAsync(p.host_small + 1, p.flags, sizeof(unsigned int),
                                  cudaMemcpyDeviceToHost, s));
    FDAS_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t total = (int64_t)p.host_small[0];
    unsigned int flags = (unsigned int)(p.host_small[1] & 0xffffffffu);
    if (injected_fault().kind == kFaultNan) flags |= 1u;
    if (flags & 2u) {
        *n_found = 0;
        set_error("a bounded wait for an asynchronous copy gave up");
        return FDAS_ERR_TIMEOUT;
    }
    if (flags & 1u) {
        *n_found = 0;
        set_error("non-finite values in an input series");
        return FDAS_ERR_NONFINITE;
    }
    if (total > p.store_cap) {
        // the store kept the first store_cap crossings to arrive, which
        // depend on scheduling: no subset of them is the ordered prefix
        *n_found = total;
        set_error("device candidate store full: " + std::to_string(total) +
                  " crossings, store of " + std::to_string(p.store_cap) +
                  " (raise max_candidates or the threshold)");
        return FDAS_ERR_CAND_STORE_FULL;
    }
    const int64_t stored = total;
    FDAS_TRY(launch_candidates_finish(p, stored, p.out_stage, s));
    const int64_t n_copy = std::min(stored, capacity);
    if (n_copy > 0)
        FDAS_CUDA_TRY(cudaMemcpyAsync(cands, p.out_stage, sizeof(fdas_candidate) * (size_t)n_copy,
                                      cudaMemcpyDefault, s));
    FDAS_CUDA_TRY(cudaStreamSynchronize(s));
    *n_found = total;
    if (total > capacity) {
        set_error("candidate buffer too small: " + std::to_string(total) + " found, capacity " +
                  std::to_string(capacity));
        return FDAS_ERR_CAND_OVERFLOW;
    }
    return FDAS_OK;
}

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&old_);
        if (old_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != old_) cudaSetDevice(old_);
    }

   private:
    int old_ = 0;
};

// event pool for the tracing intervals
static fdas_status events_reserve(Plan &p, size_t n) {
    while (p.pools->events.size() < n) {
        cudaEvent_t e;
        FDAS_CUDA_TRY(cudaEventCreate(&e));
        p.pools->events.push_back(e);
    }
    return FDAS_OK;
}

struct Interval {
    int group;
    cudaEvent_t a, b;
};

static void accumulate(Plan &p, const std::vector<Interval> &iv) {
    for (const Interval &x : iv) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, x.a, x.b) == cudaSuccess) {
            p.prof_ms[x.group] += ms;
            p.timed[x.group] += 1;
        } else {
            cudaGetLastError();
        }
    }
}

static bool is_pinned_or_device(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
           a.type == cudaMemoryTypeHost;
}

// A series in page-locked host memory is copied to its staging buffer by
// this kernel, which reads the host memory directly through its mapped
// address (16-byte loads, four in flight per thread), on the plan's copy
// stream.  The copy engine's transfers of the same memory were measured
// to stall intermittently (a search of 64 series from 100 to 135-145 ms)
// once other processes had churned the host's memory, while these loads
// kept their rate (100.5 ms, against 99.6 ms for device-resident series);
// pageable memory still goes through cudaMemcpyAsync.  Eight CTAs keep the
// copy ahead of the kernels while taking the fewest SM slots from them (32
// and 152 CTAs measured 101.5 and 106.8 ms).
constexpr int kH2dCtas = 8, kH2dThreads = 512;
__global__ void __launch_bounds__(kH2dThreads) h2d_copy_kernel(float4 *__restrict__ dst,
                                                               const float4 *__restrict__ src,
                                                               int64_t n4) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        const float4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n4; i += stride) dst[i] = src[i];
}

// the per-series work of a batch, queued on s (and the plan's second
// stream); returns the intervals to time when tracing
static fdas_status enqueue_batch(Plan &p, const fdas_series *batch, int32_t n_series,
                                 const std::vector<int32_t> &rank, cudaStream_t s,
                                 std::vector<Interval> &iv, size_t &ev) {
    const size_t cb = cpx_bytes(p.prec);
    void *spec = (char *)p.spec_pad + cb * (size_t)p.m_ov;
    auto mark = [&](cudaStream_t st) -> cudaEvent_t {
        cudaEvent_t e = p.pools->events[ev++];
        cudaEventRecord(e, st);
        return e;
    };
    // while tracing, every group runs on the caller's stream, so that each
    // event interval holds the kernels of one group and nothing else;
    // otherwise the spectrum and correlation run on the plan's
    // high-priority stream (after the work already queued on the caller's)
    // and the harmonic sums on its low-priority one
    cudaStream_t hs = p.profiling ? s : p.aux;
    cudaStream_t caller = s;
    if (!p.profiling) {
        FDAS_CUDA_TRY(cudaEventRecord(p.ev_fork, caller));
        FDAS_CUDA_TRY(cudaStreamWaitEvent(p.hi, p.ev_fork, 0));
        s = p.hi;
    }
    // series in host memory are copied on their own stream into two
    // alternating staging buffers, so that the copy of the next series
    // overlaps the work on this one
    std::vector<char> on_host(n_series);
    std::vector<const float *> mapped(n_series, nullptr);   // device address of page-locked series
    int n_host = 0;
    for (int32_t t = 0; t < n_series; ++t) {
        n_host += on_host[t] = !is_device_ptr(batch[t].data);
        if (on_host[t]) mapped[t] = (const float *)device_view((void *)batch[t].data);
    }
    float *stages[2] = {p.stage, p.stage2};
    int copied = 0;   // host series queued for copy so far
    auto queue_copy = [&](int32_t t, int slot) -> fdas_status {
        // the slot is free once the spectrum of the series two copies back read it
        if (copied >= 2) FDAS_CUDA_TRY(cudaStreamWaitEvent(p.cpy, p.ev_consumed[slot], 0));
        if (mapped[t] != nullptr) {
            h2d_copy_kernel<<<kH2dCtas, kH2dThreads, 0, p.cpy>>>(
                (float4 *)stages[slot], (const float4 *)mapped[t], batch[t].n_samples / 4);
            FDAS_CUDA_TRY(cudaGetLastError());
        } else {
            FDAS_CUDA_TRY(cudaMemcpyAsync(stages[slot], batch[t].data,
                                          sizeof(float) * (size_t)batch[t].n_samples,
                                          cudaMemcpyHostToDevice, p.cpy));
        }
        FDAS_CUDA_TRY(cudaEventRecord(p.ev_copied[slot], p.cpy));
        ++copied;
        return FDAS_OK;
    };
    if (n_host > 0) {
        // the copy stream starts after the work already queued on the
        // caller's stream (and joins a graph capture of it)
        FDAS_CUDA_TRY(cudaEventRecord(p.ev_start, s));
        FDAS_CUDA_TRY(cudaStreamWaitEvent(p.cpy, p.ev_start, 0));
    }
    int host_seen = 0;
    int32_t next_host = 0;   // next host series whose copy is not queued yet
    auto queue_next = [&]() -> fdas_status {
        while (next_host < n_series && !on_host[next_host]) ++next_host;
        if (next_host < n_series) {
            FDAS_TRY(queue_copy(next_host, copied & 1));
            ++next_host;
        }
        return FDAS_OK;
    };
    if (n_host > 0) {
        FDAS_TRY(queue_next());
        FDAS_TRY(queue_next());
    }
    for (int32_t t = 0; t < n_series; ++t) {
        const int b = t & 1;
        Plan v = batch[t].n_samples == p.n_samples ? p : plan_view(p, batch[t].n_samples);
        const float *x = batch[t].data;
        int slot = -1;
        if (on_host[t]) {
            slot = host_seen & 1;
            ++host_seen;
            FDAS_CUDA_TRY(cudaStreamWaitEvent(s, p.ev_copied[slot], 0));
            x = stages[slot];
        }
        if (v.n_r < p.n_r) {
            // a shorter series: the bins past its end must read as 0 again
            const size_t tail = (size_t)v.n_seg * v.V + 2 * (size_t)v.m_ov - ((size_t)v.m_ov + v.n_r);
            FDAS_CUDA_TRY(cudaMemsetAsync((char *)spec + cb * (size_t)v.n_r, 0, cb * tail, s));
        }
        cudaEvent_t e0 = p.profiling ? mark(s) : nullptr;
        FDAS_TRY(launch_spectrum(v, x, spec, nullptr, s));
        FDAS_DEBUG_CHECK(p, s, "the spectrum of series " + std::to_string(t));
        cudaEvent_t e1 = p.profiling ? mark(s) : nullptr;
        if (slot >= 0) {
            FDAS_CUDA_TRY(cudaEventRecord(p.ev_consumed[slot], s));
            FDAS_TRY(queue_next());
        }
        // plane[b] and partials[b] are free once the harmonic sum of series t-2
        // is done; only the correlation writes them
        if (t >= 2) {
            FDAS_CUDA_TRY(cudaStreamWaitEvent(s, p.ev_hsum[b], 0));
            if (p.profiling) e1 = mark(s);
        }
        FDAS_TRY(launch_plane(v, p.spec_pad, p.plane[b], p.partials[b], s));
#ifdef FDAS_CHECK_BOUNDS
        if (p.plant_canary && t == 0) {
            // FDAS_FAULT=canary: one byte of the guard after the plane
            for (const Plan::GuardedBuf &g : p.pools->guards)
                if (g.base + kGuardBytes == (char *)p.plane[b])
                    FDAS_CUDA_TRY(cudaMemsetAsync(g.base + kGuardBytes + g.bytes, 0, 1, s));
        }
#endif
        FDAS_DEBUG_CHECK(p, s, "the correlation of series " + std::to_string(t));
        cudaEvent_t e2 = p.profiling ? mark(s) : nullptr;
        FDAS_CUDA_TRY(cudaEventRecord(p.ev_conv[b], s));
        FDAS_CUDA_TRY(cudaStreamWaitEvent(hs, p.ev_conv[b], 0));
        cudaEvent_t e3 = p.profiling ? mark(hs) : nullptr;
        TrialStats *ts = p.stats + rank[t];
        Plan hv = harm_view(v);
        FDAS_TRY(launch_finalize_stats(hv, p.partials[b], plane_partials(v), nullptr, ts, hs));
        FDAS_TRY(launch_harmonic_threshold(hv, p.plane[b], ts, (uint32_t)rank[t], hs));
        FDAS_DEBUG_CHECK(p, hs, "the harmonic sum of series " + std::to_string(t));
        cudaEvent_t e4 = p.profiling ? mark(hs) : nullptr;
        FDAS_CUDA_TRY(cudaEventRecord(p.ev_hsum[b], hs));
        p.launches[FDAS_PROF_SPECTRUM] += (v.fft_m1 == 1 ? 1 : 2) + 1;
        p.launches[FDAS_PROF_CORRELATE] += p.interbin ? 2 : 1;   // + fix-up or interbinning
        p.launches[FDAS_PROF_HARMONIC] += 2;
        if (p.profiling) {
            iv.push_back({FDAS_PROF_SPECTRUM, e0, e1});
            iv.push_back({FDAS_PROF_CORRELATE, e1, e2});
            iv.push_back({FDAS_PROF_HARMONIC, e3, e4});
        }
    }
    if (s != caller) {
        FDAS_CUDA_TRY(cudaEventRecord(p.ev_join, s));
        FDAS_CUDA_TRY(cudaStreamWaitEvent(caller, p.ev_join, 0));
    }
    for (int b = 0; b < 2 && b < n_series; ++b)
        FDAS_CUDA_TRY(cudaStreamWaitEvent(caller, p.ev_hsum[(n_series - 1 - b) & 1], 0));
    return FDAS_OK;
}

// capture the batch into one CUDA graph (updating the previous executable
// when the launch sequence has the same shape) and launch it
static fdas_status run_as_graph(Plan &p, const fdas_series *batch, int32_t n_series,
                                const std::vector<int32_t> &rank, cudaStream_t s) {
    std::vector<Interval> iv;
    size_t ev = 0;
    FDAS_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    fdas_status st = enqueue_batch(p, batch, n_series, rank, s, iv, ev);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != FDAS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    FDAS_CUDA_TRY(ce);
    bool updated = false;
    if (p.graph_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(p.graph_exec, g, &info) == cudaSuccess) updated = true;
        else {
            cudaGetLastError();
            cudaGraphExecDestroy(p.graph_exec);
            p.graph_exec = nullptr;
        }
    }
    if (!updated) {
        ce = cudaGraphInstantiate(&p.graph_exec, g, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(g);
            p.graph_exec = nullptr;
            return cuda_status(ce, "cudaGraphInstantiate");
        }
    }
    cudaGraphDestroy(g);
    FDAS_CUDA_TRY(cudaGraphLaunch(p.graph_exec, s));
    return FDAS_OK;
}

// the series checks shared by both searches; graphable is cleared when a
// series is in pageable host memory
static fdas_status check_batch(const Plan &p, const fdas_series *batch, int32_t n_series,
                               bool &graphable) {
    if (n_series < 0) return arg_error("n_series < 0");
    if (n_series > (1 << 22)) return arg_error("n_series > 2^22");
    if (n_series > 0 && batch == nullptr) return arg_error("batch is NULL");
    for (int32_t i = 0; i < n_series; ++i) {
        const int64_t n = batch[i].n_samples;
        if (batch[i].data == nullptr) return arg_error("series " + std::to_string(i) + " has NULL data");
        if (!is_pow2(n) || n > p.n_samples || n < (1 << 10))
            return arg_error("series " + std::to_string(i) +
                             " must hold the plan's n_samples / 2^d samples, at least 2^10");
        if (((uintptr_t)batch[i].data & 15u) != 0)
            return arg_error("series " + std::to_string(i) + " is not 16-byte aligned");
        if (graphable && !is_pinned_or_device(batch[i].data)) graphable = false;
    }
    return FDAS_OK;
}

// everything of a search up to the candidate collection, queued on s: trial
// ranks, counters reset, and the batch (as a graph, or forked to the plan's
// streams and joined back to s)
static fdas_status enqueue_search(Plan &p, const Fault &fault, const fdas_series *batch,
                                  int32_t n_series, bool graphable, cudaStream_t s,
                                  std::vector<Interval> &iv, size_t &ev) {
    p.store_cap = fault.kind == kFaultCapacity ? 1 : p.max_cands;
    FDAS_TRY(grow_stats(p, std::max<int64_t>(1, n_series)));
    // rank = position in trial_id order (stable), so the output order is
    // (trial_id, stage, iz, ir)
    std::vector<int32_t> order(n_series), rank(n_series);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return batch[a].trial_id < batch[b].trial_id; });
    std::vector<uint32_t> ids(std::max(1, (int)n_series));
    for (int32_t i = 0; i < n_series; ++i) {
        rank[order[i]] = i;
        ids[i] = batch[order[i]].trial_id;
    }
    // (a copy from pageable memory returns once the source has been read)
    if (n_series > 0)
        FDAS_CUDA_TRY(cudaMemcpyAsync(p.rank_ids, ids.data(), sizeof(uint32_t) * n_series,
                                      cudaMemcpyHostToDevice, s));
    FDAS_CUDA_TRY(cudaMemsetAsync(p.cand_count, 0, sizeof(unsigned long long), s));
    FDAS_CUDA_TRY(cudaMemsetAsync(p.flags, 0, sizeof(unsigned int), s));
    if (p.profiling) {
        FDAS_TRY(events_reserve(p, 7 * (size_t)n_series + 2));
        iv.reserve(3 * (size_t)n_series + 1);
    }
    p.plant_canary = fault.kind == kFaultCanary;
    fdas_status st = graphable && n_series > 0
                         ? run_as_graph(p, batch, n_series, rank, s)
                         : enqueue_batch(p, batch, n_series, rank, s, iv, ev);
    p.plant_canary = false;
    return st;
}

static fdas_status search(Plan &p, const fdas_series *batch, int32_t n_series,
                          fdas_candidate *cands, int64_t capacity, int64_t *n_found,
                          cudaStream_t s) {
    const Fault fault = injected_fault();
    FDAS_TRY(fault_args_check(fault));
    if (n_found == nullptr) return arg_error("n_found is NULL");
    if (capacity < 0 || (capacity > 0 && cands == nullptr)) return arg_error("bad cands/capacity");
    bool graphable = p.use_graph && !p.profiling && s != nullptr && s != cudaStreamLegacy &&
                     s != cudaStreamPerThread;
    FDAS_TRY(check_batch(p, batch, n_series, graphable));
    *n_found = 0;
    DeviceGuard guard(p.device);
    BoundsShrink shrink(fault.kind == kFaultBounds);
    std::vector<Interval> iv;
    size_t ev = 0;
    FDAS_TRY(enqueue_search(p, fault, batch, n_series, graphable, s, iv, ev));
    p.prof_trials += n_series;
    cudaEvent_t f0 = nullptr;
    if (p.profiling) {
        f0 = p.pools->events[ev++];
        cudaEventRecord(f0, s);
    }
    fdas_status st = collect(p, cands, capacity, n_found, s);
    if (p.profiling) {
        cudaEvent_t f1 = p.pools->events[ev++];
        cudaEventRecord(f1, s);
        cudaEventSynchronize(f1);
        iv.push_back({FDAS_PROF_FINISH, f0, f1});
        accumulate(p, iv);
    }
    FDAS_DEBUG_CHECK(p, s, "the candidate ordering");
    return st;
}


static fdas_status search_async(Plan &p, const fdas_series *batch, int32_t n_series,
                                fdas_candidate *cands, int64_t capacity, int64_t *n_found,
                                int32_t *status, cudaStream_t s) {
    const Fault fault = injected_fault();
    FDAS_TRY(fault_args_check(fault));
    if (n_found == nullptr || status == nullptr) return arg_error("n_found or status is NULL");
    if (capacity < 0 || (capacity > 0 && cands == nullptr)) return arg_error("bad cands/capacity");
    if (p.profiling)
        return arg_error("tracing is on: the stream-ordered search is not traced (use fdas_search)");
    // nothing below may wait for the device: the results go to memory the
    // stream can write without the host
    if (!is_pinned_or_device(n_found) || !is_pinned_or_device(status))
        return arg_error("n_found and status must be device or page-locked host memory");
    fdas_candidate *out_dev = nullptr;
    if (capacity > 0) {
        out_dev = (fdas_candidate *)device_view(cands);
        if (out_dev == nullptr) return arg_error("cands must be device or page-locked host memory");
    }
    bool graphable = p.use_graph && s != nullptr && s != cudaStreamLegacy &&
                     s != cudaStreamPerThread;
    FDAS_TRY(check_batch(p, batch, n_series, graphable));
    DeviceGuard guard(p.device);
    BoundsShrink shrink(fault.kind == kFaultBounds);
    std::vector<Interval> iv;
    size_t ev = 0;
    FDAS_TRY(enqueue_search(p, fault, batch, n_series, graphable, s, iv, ev));
    const unsigned int extra = fault.kind == kFaultNan ? 1u : 0u;
    FDAS_TRY(launch_candidates_finish_async(p, capacity, extra, out_dev, s));
    FDAS_CUDA_TRY(cudaMemcpyAsync(n_found, &p.async_res->n_found, sizeof(int64_t),
                                  cudaMemcpyDefault, s));
    FDAS_CUDA_TRY(cudaMemcpyAsync(status, &p.async_res->status, sizeof(int32_t),
                                  cudaMemcpyDefault, s));
    FDAS_DEBUG_CHECK(p, s, "the candidate ordering");
    return FDAS_OK;
}

// time the correlation of one full-length series on a plan (synthetic unit
// spectrum), median of a few runs, in ms
static fdas_status time_correlation(Plan &p, double &ms) {
    const size_t cb = cpx_bytes(p.prec);
    cudaStream_t s = p.aux;
    // any finite spectrum will do for timing: the plan's own zero-padded
    // buffer with its interior set to a constant pattern
    FDAS_CUDA_TRY(cudaMemsetAsync((char *)p.spec_pad + cb * (size_t)p.m_ov, 0x3c, cb * (size_t)p.n_r, s));
    cudaEvent_t a, b;
    FDAS_CUDA_TRY(cudaEventCreate(&a));
    FDAS_CUDA_TRY(cudaEventCreate(&b));
    std::vector<float> t;
    fdas_status st = FDAS_OK;
    for (int rep = 0; rep < 4 && st == FDAS_OK; ++rep) {
        cudaEventRecord(a, s);
        st = launch_correlate(p, p.spec_pad, p.plane[0], p.partials[0], s);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) st = cuda_status(cudaGetLastError(), "autotune");
        float x = 0.f;
        cudaEventElapsedTime(&x, a, b);
        if (rep > 0) t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != FDAS_OK) return st;
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return FDAS_OK;
}

// rebuild the tensor-core template chunks of a plan in another template
// order (chunk table, template images, shared-memory layout)
static fdas_status retable_tc(Plan &p, int order) {
    if (p.correlator != FDAS_CORR_TENSOR || p.tc_order == order) return FDAS_OK;
    std::vector<int32_t> m(p.n_z);
    FDAS_CUDA_TRY(cudaMemcpy(m.data(), p.tap_m, sizeof(int32_t) * p.n_z, cudaMemcpyDeviceToHost));
    const int old_order = p.tc_order, old_win = p.tc_win, old_ks = p.tc_max_ks, old_n = p.tc_n_ch;
    p.tc_order = order;
    std::vector<TcChunk> table = tc_chunk_table(p, m, &p.tc_win, &p.tc_max_ks);
    if (!tc_applicable(p, nullptr)) {
        p.tc_order = old_order;
        p.tc_win = old_win;
        p.tc_max_ks = old_ks;
        p.tc_n_ch = old_n;
        set_error("template order does not fit in shared memory");
        return FDAS_ERR_UNSUPPORTED;
    }
    FDAS_CUDA_TRY(cudaDeviceSynchronize());
    const int64_t img = tc_bank_bytes(table);
    p.ws_bytes -= p.tc_img_bytes + (int64_t)sizeof(TcChunk) * old_n;
    dfree(p, p.tc_chunks);
    dfree(p, p.tc_bank);
    p.tc_chunks = nullptr;
    p.tc_bank = nullptr;
    FDAS_TRY(dalloc(p, &p.tc_chunks, sizeof(TcChunk) * table.size(), "tc_chunks"));
    if (p.tc_split) p.tc_bank_lo = img;
    FDAS_TRY(dalloc(p, &p.tc_bank, (size_t)img * (p.tc_split ? 2 : 1), "tc_bank"));
    p.tc_img_bytes = img * (p.tc_split ? 2 : 1);
    p.tc_n_ch = (int)table.size();
    p.tc_nbuf = tc_image_buffers(p);
    FDAS_CUDA_TRY(cudaMemcpy(p.tc_chunks, table.data(), sizeof(TcChunk) * table.size(),
                             cudaMemcpyHostToDevice));
    FDAS_TRY(launch_tc_bank(p, p.aux));
    FDAS_CUDA_TRY(cudaStreamSynchronize(p.aux));
    return FDAS_OK;
}

// autotune: the correlator (the tensor-core GEMM, where it applies and was
// not excluded, against overlap-save FFTs), the segment length among {2048,
// 4096, 8192} and the one asked for, then the template chunking of the
// fastest FFT plan or the template order of the tensor-core chunks, by
// timing the correlation
static fdas_status create_tuned(Plan *&out, int64_t n_samples, double tsamp, double z_max,
                                double z_step, int32_t seg_len, int32_t n_harm, fdas_opts o) {
    o.autotune = 0;
    std::vector<std::pair<int32_t, int32_t>> cand;   // (seg_len, correlator)
    if (o.correlator == FDAS_CORR_TENSOR_SPLIT)
        cand.push_back({seg_len, FDAS_CORR_TENSOR_SPLIT});   // asked for explicitly
    else if (o.correlator != FDAS_CORR_TENSOR) {
        std::vector<int32_t> lens = {2048, 4096, 8192};
        if (std::find(lens.begin(), lens.end(), seg_len) == lens.end()) lens.push_back(seg_len);
        for (int32_t L : lens) cand.push_back({L, FDAS_CORR_FFT});
    }
    if (o.correlator != FDAS_CORR_FFT && o.precision != FDAS_FP32)
        cand.push_back({seg_len, FDAS_CORR_TENSOR});
    Plan *best = nullptr;
    double best_ms = 1e300;
    std::string first_error;
    fdas_status first_status = FDAS_OK;
    for (const auto &lc : cand) {
        const int32_t L = lc.first;
        Plan *p = nullptr;
        fdas_opts oc = o;
        oc.correlator = lc.second;
        fdas_status s = create(p, n_samples, tsamp, z_max, z_step, L, n_harm, &oc);
        if (s != FDAS_OK) {
            if (first_status == FDAS_OK) {
                first_status = s;
                first_error = g_last_error;
            }
            continue;
        }
        double ms = 0.0;
        s = time_correlation(*p, ms);
        if (s == FDAS_OK && ms < best_ms) {
            if (best) {
                free_plan_memory(best);
                delete best;
            }
            best = p;
            best_ms = ms;
        } else {
            free_plan_memory(p);
            delete p;
        }
    }
    if (!best) {
        set_error(first_error.empty() ? "autotune: no segment length fits" : first_error);
        return first_status == FDAS_OK ? FDAS_ERR_ARG : first_status;
    }
    // template chunking of the chosen length
    const int base = best->n_zchunk;
    int best_c = base;
    for (int c : {1, 2, 3, 4, 6, 8, 12, 16}) {
        if (best->correlator != FDAS_CORR_FFT) break;
        if (c == base || c > best->n_z || (int64_t)best->n_seg * c > best->partials_cap) continue;
        best->n_zchunk = c;
        double ms = 0.0;
        if (time_correlation(*best, ms) == FDAS_OK && ms < best_ms) {
            best_ms = ms;
            best_c = c;
        }
    }
    best->n_zchunk = best_c;
    // template order of the tensor-core chunks, unless asked for
    if (best->correlator == FDAS_CORR_TENSOR && o.template_order == FDAS_TORDER_DEFAULT) {
        const int first = best->tc_order;
        if (retable_tc(*best, 1 - first) == FDAS_OK) {
            double ms = 0.0;
            if (time_correlation(*best, ms) == FDAS_OK && ms < best_ms) {
                best_ms = ms;
            } else {
                FDAS_TRY(retable_tc(*best, first));
            }
        }
    }
    best->tuned_ms = best_ms;
    out = best;
    return FDAS_OK;
}

}  // namespace fdas

using namespace fdas;

extern "C" {

void fdas_opts_default(fdas_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FDAS_FP32;
    o->threshold_sigma = 6.0;
    o->threshold_mode = FDAS_THRESH_GAMMA_TAIL;
    o->norm_mode = FDAS_NORM_MEDIAN;
    o->norm_block = 2048;
    o->max_candidates = int64_t(1) << 20;
    o->autotune = 0;
    o->use_graph = 0;
}

fdas_status fdas_plan_create(fdas_plan **out, int64_t n_samples, double tsamp, double z_max,
                             double z_step, int32_t seg_len, int32_t n_harm, const fdas_opts *opts) {
    try {
        if (!out) return arg_error("out is NULL");
        *out = nullptr;
        fdas_opts o;
        fdas_opts_default(&o);
        if (opts) o = *opts;
        Plan *p = nullptr;
        fdas_status s = o.autotune ? create_tuned(p, n_samples, tsamp, z_max, z_step, seg_len,
                                                  n_harm, o)
                                   : create(p, n_samples, tsamp, z_max, z_step, seg_len, n_harm, &o);
        if (s == FDAS_OK) *out = reinterpret_cast<fdas_plan *>(p);
        return s;
    } catch (...) {
        set_error("unexpected C++ exception in fdas_plan_create");
        return FDAS_ERR_CUDA;
    }
}

void fdas_plan_destroy(fdas_plan *plan) {
    if (!plan) return;
    Plan *p = reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    free_plan_memory(p);
    delete p;
}

fdas_status fdas_plan_get_info(const fdas_plan *plan, fdas_plan_info *info) {
    if (!plan || !info) return arg_error("NULL argument");
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    std::memset(info, 0, sizeof(*info));
    info->n_samples = p.n_samples;
    info->n_r = p.n_r;
    info->n_z = p.n_z;
    info->iz0 = p.iz0;
    info->m_max = p.m_max;
    info->m_overlap = p.m_ov;
    info->seg_len = p.L;
    info->valid_per_seg = p.V;
    info->n_seg = p.n_seg;
    info->n_harm = p.H;
    info->n_stages = p.n_stages;
    info->precision = p.prec;
    info->norm_block = p.norm_block;
    info->threshold_mode = p.thr_mode;
    info->tsamp = p.tsamp;
    info->z_max = p.z_max;
    info->z_step = p.z_step;
    info->threshold_sigma = p.sigma;
    for (int s = 0; s < 6; ++s) info->stage_factor[s] = p.G[s];
    info->workspace_bytes = p.ws_bytes;
    info->z_chunks = p.n_zchunk;
    info->use_graph = p.use_graph ? 1 : 0;
    info->tuned_ms = p.tuned_ms;
    info->correlator = p.tc_split ? FDAS_CORR_TENSOR_SPLIT : p.correlator;
    info->harmonic_mode = p.harm_mode;
    info->interbin = p.interbin ? 1 : 0;
    info->template_order = p.correlator != FDAS_CORR_TENSOR ? 0
                           : p.tc_order == 0                  ? FDAS_TORDER_Z
                                                              : FDAS_TORDER_PAIRED;
    info->plane_cols = plane_cols(p);
    return FDAS_OK;
}

fdas_status fdas_search(fdas_plan *plan, const fdas_series *batch, int32_t n_series,
                        fdas_candidate *cands, int64_t capacity, int64_t *n_found, void *stream) {
    try {
        if (!plan) return arg_error("plan is NULL");
        return search(*reinterpret_cast<Plan *>(plan), batch, n_series, cands, capacity, n_found,
                      (cudaStream_t)stream);
    } catch (...) {
        set_error("unexpected C++ exception in fdas_search");
        return FDAS_ERR_CUDA;
    }
}

fdas_status fdas_search_async(fdas_plan *plan, const fdas_series *batch, int32_t n_series,
                              fdas_candidate *cands, int64_t capacity, int64_t *n_found,
                              int32_t *status, void *stream) {
    try {
        if (!plan) return arg_error("plan is NULL");
        return search_async(*reinterpret_cast<Plan *>(plan), batch, n_series, cands, capacity,
                            n_found, status, (cudaStream_t)stream);
    } catch (...) {
        set_error("unexpected C++ exception in fdas_search_async");
        return FDAS_ERR_CUDA;
    }
}

fdas_status fdas_spectrum(fdas_plan *plan, const float *series, void *spectrum_out,
                          float *medians_out, void *stream) {
    if (!plan || !series || !spectrum_out) return arg_error("NULL argument");
    if (((uintptr_t)series & 15u) != 0) return arg_error("series is not 16-byte aligned");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    FDAS_TRY(launch_spectrum(p, series, spectrum_out, medians_out, (cudaStream_t)stream));
    FDAS_DEBUG_CHECK(p, (cudaStream_t)stream, "fdas_spectrum");
    return FDAS_OK;
}

fdas_status fdas_power_plane(fdas_plan *plan, const void *spectrum, void *plane_out,
                             double *stats_out, void *stream) {
    if (!plan || !spectrum || !plane_out) return arg_error("NULL argument");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cb = cpx_bytes(p.prec);
    FDAS_CUDA_TRY(cudaMemcpyAsync((char *)p.spec_pad + cb * (size_t)p.m_ov, spectrum,
                                  cb * (size_t)p.n_r, cudaMemcpyDeviceToDevice, s));
    FDAS_TRY(launch_plane(p, p.spec_pad, plane_out, p.partials[0], s));
    if (stats_out) {
        Plan hv = harm_view(p);
        FDAS_TRY(launch_finalize_stats(hv, p.partials[0], plane_partials(p), nullptr, p.stats, s));
        FDAS_CUDA_TRY(cudaMemcpyAsync(stats_out, p.stats, 2 * sizeof(double),
                                      cudaMemcpyDeviceToDevice, s));
    }
    FDAS_DEBUG_CHECK(p, s, "fdas_power_plane");
    return FDAS_OK;
}

fdas_status fdas_correlation_plane(fdas_plan *plan, const void *spectrum, void *corr_out,
                                   void *stream) {
    if (!plan || !spectrum || !corr_out) return arg_error("NULL argument");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cb = cpx_bytes(p.prec);
    FDAS_CUDA_TRY(cudaMemcpyAsync((char *)p.spec_pad + cb * (size_t)p.m_ov, spectrum,
                                  cb * (size_t)p.n_r, cudaMemcpyDeviceToDevice, s));
    FDAS_TRY(launch_correlate(p, p.spec_pad, corr_out, p.partials[0], s, true));
    FDAS_DEBUG_CHECK(p, s, "fdas_correlation_plane");
    return FDAS_OK;
}

fdas_status fdas_harmonic_sums(fdas_plan *plan, const void *plane, float *sums_out, void *stream) {
    if (!plan || !plane || !sums_out) return arg_error("NULL argument");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    Plan hv = harm_view(p);
    FDAS_TRY(launch_harmonic_sums(hv, plane, sums_out, (cudaStream_t)stream));
    FDAS_DEBUG_CHECK(p, (cudaStream_t)stream, "fdas_harmonic_sums");
    return FDAS_OK;
}

fdas_status fdas_threshold(fdas_plan *plan, const void *plane, const double *stats,
                           uint32_t trial_id, fdas_candidate *cands, int64_t capacity,
                           int64_t *n_found, void *stream) {
    if (!plan || !plane || !stats || !n_found) return arg_error("NULL argument");
    if (capacity < 0 || (capacity > 0 && !cands)) return arg_error("bad cands/capacity");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    cudaStream_t s = (cudaStream_t)stream;
    *n_found = 0;
    const Fault fault = injected_fault();
    if (fault.kind == kFaultUnknown) return fault_args_check(fault);
    p.store_cap = fault.kind == kFaultCapacity ? 1 : p.max_cands;
    FDAS_CUDA_TRY(cudaMemcpyAsync(p.rank_ids, &trial_id, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    FDAS_CUDA_TRY(cudaMemsetAsync(p.cand_count, 0, sizeof(unsigned long long), s));
    FDAS_CUDA_TRY(cudaMemsetAsync(p.flags, 0, sizeof(unsigned int), s));
    Plan hv = harm_view(p);
    FDAS_TRY(launch_finalize_stats(hv, nullptr, 0, stats, p.stats, s));
    FDAS_TRY(launch_harmonic_threshold(hv, plane, p.stats, 0, s));
    const fdas_status st = collect(p, cands, capacity, n_found, s);
    FDAS_DEBUG_CHECK(p, s, "fdas_threshold");
    return st;
}

fdas_status fdas_selftest_wait_timeout(fdas_plan *plan, int64_t limit_cycles, void *stream) {
    if (!plan) return arg_error("plan is NULL");
    if (limit_cycles < 1 || limit_cycles > 2000000000LL) return arg_error("limit_cycles out of range");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    cudaStream_t s = (cudaStream_t)stream;
    FDAS_CUDA_TRY(cudaMemsetAsync(p.cand_count, 0, sizeof(unsigned long long), s));
    FDAS_CUDA_TRY(cudaMemsetAsync(p.flags, 0, sizeof(unsigned int), s));
    FDAS_TRY(launch_stuck_wait(p.flags, (long long)limit_cycles, s));
    int64_t n_found = 0;
    return collect(p, nullptr, 0, &n_found, s);
}

fdas_status fdas_template_bank(fdas_plan *plan, double *taps_out, double *energy_out,
                               void *bank_out, void *stream) {
    if (!plan) return arg_error("plan is NULL");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    cudaStream_t s = (cudaStream_t)stream;
    if (taps_out)
        FDAS_CUDA_TRY(cudaMemcpyAsync(taps_out, p.taps, sizeof(double) * 2 * (size_t)p.n_taps,
                                      cudaMemcpyDeviceToHost, s));
    if (energy_out)
        FDAS_CUDA_TRY(cudaMemcpyAsync(energy_out, p.energy, sizeof(double) * p.n_z,
                                      cudaMemcpyDeviceToHost, s));
    if (bank_out)
        FDAS_CUDA_TRY(cudaMemcpyAsync(bank_out, p.bank, cpx_bytes(p.prec) * (size_t)p.n_z * p.L,
                                      cudaMemcpyDeviceToDevice, s));
    FDAS_CUDA_TRY(cudaStreamSynchronize(s));
    return FDAS_OK;
}

fdas_status fdas_fourier_power(fdas_plan *plan, const float *spectrum, const double *rz, int32_t n,
                               float *power, float *grad_rz, void *stream) {
    if (!plan || !spectrum || (n > 0 && (!rz || !power))) return arg_error("NULL argument");
    if (n < 0) return arg_error("n < 0");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    return launch_fourier_power(p, (const float2 *)spectrum, (const double2 *)rz, n, power,
                                (float2 *)grad_rz, (cudaStream_t)stream);
}

fdas_status fdas_fourier_power_backward(fdas_plan *plan, const float *spectrum, const double *rz,
                                        int32_t n, const float *grad_power, float *grad_spectrum,
                                        double *grad_rz, void *stream) {
    if (!plan || !spectrum || (n > 0 && (!rz || !grad_power))) return arg_error("NULL argument");
    if (n < 0) return arg_error("n < 0");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    return launch_fourier_power_backward(p, (const float2 *)spectrum, (const double2 *)rz, n,
                                         grad_power, (float2 *)grad_spectrum, (double2 *)grad_rz,
                                         (cudaStream_t)stream);
}

fdas_status fdas_refine(fdas_plan *plan, const float *spectrum, const fdas_seed *seeds, int32_t n,
                        int32_t n_steps, fdas_refined *out, void *stream) {
    if (!plan || !spectrum || (n > 0 && (!seeds || !out))) return arg_error("NULL argument");
    if (n < 0 || n_steps < 0) return arg_error("n and n_steps must be >= 0");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    DeviceGuard guard(p.device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return FDAS_OK;
    if (n > p.ref_cap) {
        FDAS_CUDA_TRY(cudaStreamSynchronize(s));
        p.ws_bytes -= (int64_t)(sizeof(fdas_seed) + sizeof(fdas_refined)) * p.ref_cap;
        dfree(p, p.ref_seeds);
        dfree(p, p.ref_out);
        p.ref_seeds = nullptr;
        p.ref_out = nullptr;
        p.ref_cap = 0;
        FDAS_TRY(dalloc(p, &p.ref_seeds, sizeof(fdas_seed) * (size_t)n, "ref_seeds"));
        FDAS_TRY(dalloc(p, &p.ref_out, sizeof(fdas_refined) * (size_t)n, "ref_out"));
        p.ref_cap = n;
    }
    FDAS_CUDA_TRY(cudaMemcpyAsync(p.ref_seeds, seeds, sizeof(fdas_seed) * (size_t)n,
                                  cudaMemcpyDefault, s));
    FDAS_TRY(launch_refine(p, (const float2 *)spectrum, p.ref_seeds, n, n_steps, p.ref_out, s));
    FDAS_DEBUG_CHECK(p, s, "fdas_refine");
    FDAS_CUDA_TRY(cudaMemcpyAsync(out, p.ref_out, sizeof(fdas_refined) * (size_t)n,
                                  cudaMemcpyDefault, s));
    FDAS_CUDA_TRY(cudaStreamSynchronize(s));
    return FDAS_OK;
}

fdas_status fdas_profile_enable(fdas_plan *plan, int32_t on) {
    if (!plan) return arg_error("plan is NULL");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    p.profiling = on != 0;
    p.prof_trials = 0;
    for (int g = 0; g < 4; ++g) {
        p.launches[g] = 0;
        p.timed[g] = 0;
        p.prof_ms[g] = 0.0;
    }
    return FDAS_OK;
}

fdas_status fdas_profile_read(const fdas_plan *plan, fdas_profile *out) {
    if (!plan || !out) return arg_error("NULL argument");
    const Plan &p = *reinterpret_cast<const Plan *>(plan);
    out->trials = p.prof_trials;
    for (int g = 0; g < 4; ++g) {
        out->launches[g] = p.launches[g];
        out->timed[g] = p.timed[g];
        out->ms[g] = p.prof_ms[g];
    }
    return FDAS_OK;
}

const char *fdas_last_error(void) { return g_last_error.c_str(); }

#ifdef FDAS_CHECK_BOUNDS
const char *fdas_version(void) { return "fdas-gb300 0.1 (sm_103a, checked)"; }
int32_t fdas_checked_build(void) { return 1; }
#else
const char *fdas_version(void) { return "fdas-gb300 0.1 (sm_103a)"; }
int32_t fdas_checked_build(void) { return 0; }
#endif

}  // extern "C"
