// Incoherent dedispersion: the stage that turns a filterbank into the
// DM-trial series the search runs on (the paper's workload is 5925 DM trials,
// §3; the paper does not describe this stage, so the textbook definition is
// used).
//
// Channel c has centre frequency f_c = f_top - c df (MHz, descending).  At
// DM_d = dm_lo + d dm_step the cold-plasma delay of channel c relative to the
// top of the band, in samples, is
//
//     Delta(c, d) = floor(K_DM DM_d (f_c^-2 - f_top^-2) / tsamp + 1/2),
//     K_DM = 4.148808e3 MHz^2 pc^-1 cm^3 s,
//
// and the dedispersed series is out[d][t] = sum_c in[c][t + Delta(c, d)],
// samples at or past n_t counted as 0.  The delays are computed once per plan
// in FP64 with every operation rounded separately (no contraction), so they
// are exactly those of the same formula evaluated in IEEE FP64 elsewhere.
//
// Kernel: a CTA owns 32 DM trials x 512 output samples.  Per batch of
// channels it stages, for each channel, the window of input samples its 32
// DMs read (512 + the spread of their delays) in shared memory by
// asynchronous 4-byte copies (cp.async, zero-filled past n_t), double
// buffered so that the copies of the next batch run during the sums of this
// one.  Warp w accumulates DMs 4w..4w+3, lane l the samples l + 32k (k < 16),
// reading shared memory with consecutive lanes on consecutive words; where
// two DMs of a pair have the same delay for a channel (common at high
// frequency and small DM steps) one load feeds both.  FP32 sums over the
// channels in channel order; the bound is shared-memory bandwidth (one 4-byte
// word per lane per addition, less with shared delays).
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kDdT = 512;        // output samples per tile
constexpr int kDdD = 32;         // DM trials per tile
constexpr int kDdThreads = 256;  // 8 warps x 4 DM trials
constexpr int kDdPer = kDdT / 32;
constexpr double kDm = 4.148808e3;
constexpr size_t kDdSmemCap = 200 * 1024;   // both buffers

__global__ void dm_delay_kernel(int32_t *__restrict__ out, int n_chan, int n_dm, double f_top,
                                double df, double tsamp, double dm_lo, double dm_step) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_chan * n_dm) return;
    const int d = (int)(i / n_chan), c = (int)(i % n_chan);
    const double f = __dsub_rn(f_top, __dmul_rn((double)c, df));
    const double a = __ddiv_rn(1.0, __dmul_rn(f, f));
    const double b = __ddiv_rn(1.0, __dmul_rn(f_top, f_top));
    const double dm = __dadd_rn(dm_lo, __dmul_rn((double)d, dm_step));
    const double x = __ddiv_rn(__dmul_rn(__dmul_rn(kDm, dm), __dsub_rn(a, b)), tsamp);
    out[i] = (int32_t)floor(__dadd_rn(x, 0.5));
}

// 4-byte global -> shared copy, zero-filled when `valid` is false
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 16-byte global -> shared copy of the first `valid` bytes (the rest zero)
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid)
                 : "memory");
}

// acc_a += w[oa + 32k], acc_b += w[ob + 32k]; one load when oa == ob
template <class T, class A>
__device__ __forceinline__ void add_pair(const T *w, int oa, int ob, A (&acc_a)[kDdPer],
                                         A (&acc_b)[kDdPer]) {
    if (oa == ob) {
#pragma unroll
        for (int k = 0; k < kDdPer; ++k) {
            const A v = (A)w[oa + 32 * k];
            acc_a[k] += v;
            acc_b[k] += v;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kDdPer; ++k) {
            acc_a[k] += (A)w[oa + 32 * k];
            acc_b[k] += (A)w[ob + 32 * k];
        }
    }
}

// Input sample type T: FP32 samples sum in FP32 (4-byte asynchronous copies
// of each window, `pitch` = win elements per channel); 8-bit samples sum in
// int32, exactly (16-byte copies of the window rounded out to 16-byte
// boundaries, `pitch` = win + 16 bytes per channel, rows 16-byte aligned).
template <class T>
struct DdIn;
template <>
struct DdIn<float> {
    using Acc = float;
    static constexpr int kPad = 0;
};
template <>
struct DdIn<uint8_t> {
    using Acc = int;
    static constexpr int kPad = 16;
};

template <class T>
__global__ void __launch_bounds__(kDdThreads, 2)
    dedisperse_kernel(const T *__restrict__ fb, const int32_t *__restrict__ delays,
                      float *__restrict__ out, int n_chan, int64_t n_t, int n_dm, int64_t n_out,
                      int win, int chan_batch) {
    using Acc = typename DdIn<T>::Acc;
    extern __shared__ __align__(16) unsigned char dd_smem[];   // [2][chan_batch][pitch] of T
    T *sw = reinterpret_cast<T *>(dd_smem);
    const int pitch = win + DdIn<T>::kPad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = (int64_t)blockIdx.x * kDdT;
    const int d_lo = blockIdx.y * kDdD;
    const int32_t *dl = delays + (int64_t)d_lo * n_chan;
    // this warp's four DM trials (clamped: rows past n_dm are not stored)
    const int32_t *dw[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) dw[q] = delays + (int64_t)min(d_lo + 4 * warp + q, n_dm - 1) * n_chan;
    Acc acc[4][kDdPer];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < kDdPer; ++k) acc[q][k] = 0;

    const size_t buf_elems = (size_t)chan_batch * pitch;
    auto stage = [&](int cb, int slot) {
        const int nc = min(chan_batch, n_chan - cb);
        T *dst0 = sw + slot * buf_elems;
        for (int j = 0; j < nc; ++j) {
            const int64_t base = t0 + __ldg(dl + cb + j);
            const T *src = fb + (int64_t)(cb + j) * n_t;
            T *dst = dst0 + (size_t)j * pitch;
            if constexpr (sizeof(T) == 4) {
                for (int i = threadIdx.x; i < win; i += kDdThreads) {
                    const int64_t s = base + i;
                    const bool ok = s < n_t;
                    cp_async4(dst + i, src + (ok ? s : 0), ok);
                }
            } else {
                const int64_t b16 = base & ~(int64_t)15;
                for (int i = threadIdx.x; i < pitch / 16; i += kDdThreads) {
                    const int64_t s = b16 + 16 * (int64_t)i;
                    const int64_t left = n_t - s;
                    const int valid = left <= 0 ? 0 : (left >= 16 ? 16 : (int)left);
                    cp_async16(dst + 16 * i, src + (valid > 0 ? s : 0), valid);
                }
            }
        }
        cp_async_commit();
    };

    stage(0, 0);
    int slot = 0;
    for (int cb = 0; cb < n_chan; cb += chan_batch, slot ^= 1) {
        const int nc = min(chan_batch, n_chan - cb);
        if (cb + chan_batch < n_chan) {
            stage(cb + chan_batch, slot ^ 1);
            cp_async_wait<1>();   // this batch has landed (the next may be in flight)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T *buf = sw + slot * buf_elems + lane;
        for (int j = 0; j < nc; ++j) {
            const int c = cb + j;
            const int lo = __ldg(dl + c);
            // 8-bit windows start at the 16-byte boundary below the first sample
            const int shift = sizeof(T) == 1 ? (int)((t0 + lo) & 15) : 0;
            const T *w = buf + (size_t)j * pitch + shift;
            add_pair(w, __ldg(dw[0] + c) - lo, __ldg(dw[1] + c) - lo, acc[0], acc[1]);
            add_pair(w, __ldg(dw[2] + c) - lo, __ldg(dw[3] + c) - lo, acc[2], acc[3]);
        }
        __syncthreads();   // every warp is done with this slot before it is refilled
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int d = d_lo + 4 * warp + q;
        if (d >= n_dm) continue;
        float *row = out + (int64_t)d * n_out;
#pragma unroll
        for (int k = 0; k < kDdPer; ++k) {
            const int64_t t = t0 + lane + 32 * k;
            if (t < n_out) row[t] = (float)acc[q][k];
        }
    }
}

}  // namespace

struct DedispPlan {
    int32_t n_chan = 0, n_dm = 0;
    int64_t n_t = 0, n_out = 0;
    double f_top = 0, df = 0, tsamp = 0, dm_lo = 0, dm_step = 0;
    int32_t *delays = nullptr;   // device [n_dm][n_chan]
    std::vector<int32_t> host_delays;
    int32_t max_delay = 0, span = 0, win = 0, chan_batch = 0, chan_batch_u8 = 0;
    int device = 0;
};

template <class T>
fdas_status launch_dedisperse(DedispPlan &p, const T *filterbank, float *out, cudaStream_t s) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p.device) cudaSetDevice(p.device);
    const int pitch = p.win + DdIn<T>::kPad;
    const int cb = sizeof(T) == 4 ? p.chan_batch : p.chan_batch_u8;
    const size_t smem = 2 * sizeof(T) * (size_t)pitch * cb;
    cudaError_t e = cudaFuncSetAttribute(dedisperse_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)((p.n_out + kDdT - 1) / kDdT), (unsigned)((p.n_dm + kDdD - 1) / kDdD));
        dedisperse_kernel<T><<<grid, kDdThreads, smem, s>>>(filterbank, p.delays, out, p.n_chan,
                                                            p.n_t, p.n_dm, p.n_out, p.win, cb);
        e = cudaGetLastError();
    }
    if (cur != p.device) cudaSetDevice(cur);
    return e == cudaSuccess ? FDAS_OK : cuda_status(e, "dedisperse_kernel");
}

}  // namespace fdas

using fdas::DedispPlan;

namespace {

fdas_status dd_arg(const std::string &m) {
    fdas::set_error(m);
    return FDAS_ERR_ARG;
}

}  // namespace

extern "C" {

fdas_status fdas_dedisp_plan_create(fdas_dedisp_plan **out, int32_t n_chan, int64_t n_t,
                                    double f_top_mhz, double df_mhz, double tsamp, double dm_lo,
                                    double dm_step, int32_t n_dm, int64_t n_out) {
    try {
        if (!out) return dd_arg("out is NULL");
        *out = nullptr;
        if (n_chan < 1 || n_chan > 65536) return dd_arg("n_chan must be in [1, 65536]");
        if (n_dm < 1 || n_dm > 65536) return dd_arg("n_dm must be in [1, 65536]");
        if (n_t < 1 || n_t > (int64_t(1) << 34)) return dd_arg("n_t must be in [1, 2^34]");
        if (n_out < 1 || n_out > n_t) return dd_arg("n_out must be in [1, n_t]");
        if ((int64_t)n_chan * n_t > (int64_t(1) << 36)) return dd_arg("filterbank larger than 2^36 samples");
        if (!(tsamp > 0.0) || !std::isfinite(tsamp)) return dd_arg("tsamp must be > 0");
        if (!(f_top_mhz > 0.0) || !(df_mhz > 0.0) || !std::isfinite(f_top_mhz) || !std::isfinite(df_mhz))
            return dd_arg("need f_top_mhz > 0 and df_mhz > 0");
        const double f_bot = f_top_mhz - (double)(n_chan - 1) * df_mhz;
        if (!(f_bot > 0.0)) return dd_arg("the lowest channel frequency must be > 0");
        if (!(dm_lo >= 0.0) || !(dm_step >= 0.0) || !std::isfinite(dm_lo) || !std::isfinite(dm_step))
            return dd_arg("need dm_lo >= 0 and dm_step >= 0");
        const double dm_hi = dm_lo + (double)(n_dm - 1) * dm_step;
        const double x_max = fdas::kDm * dm_hi * (1.0 / (f_bot * f_bot) - 1.0 / (f_top_mhz * f_top_mhz)) / tsamp;
        if (!(x_max < 1.0e9)) return dd_arg("delays beyond 1e9 samples");

        DedispPlan *p = new (std::nothrow) DedispPlan();
        if (!p) return dd_arg("out of host memory");
        p->n_chan = n_chan;
        p->n_dm = n_dm;
        p->n_t = n_t;
        p->n_out = n_out;
        p->f_top = f_top_mhz;
        p->df = df_mhz;
        p->tsamp = tsamp;
        p->dm_lo = dm_lo;
        p->dm_step = dm_step;
        auto fail = [&](fdas_status s) {
            cudaFree(p->delays);
            delete p;
            return s;
        };
        cudaError_t e = cudaGetDevice(&p->device);
        if (e != cudaSuccess) return fail(fdas::cuda_status(e, "cudaGetDevice"));
        const size_t n = (size_t)n_chan * n_dm;
        e = cudaMalloc(&p->delays, sizeof(int32_t) * n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fdas::set_error("dedispersion: out of device memory for the delay table");
            return fail(FDAS_ERR_OOM);
        }
        fdas::dm_delay_kernel<<<(unsigned)((n + 255) / 256), 256>>>(p->delays, n_chan, n_dm, f_top_mhz,
                                                                    df_mhz, tsamp, dm_lo, dm_step);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(fdas::cuda_status(e, "dm_delay_kernel"));
        p->host_delays.resize(n);
        e = cudaMemcpy(p->host_delays.data(), p->delays, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(fdas::cuda_status(e, "cudaMemcpy"));
        // the widest window a 16-DM tile reads (per channel) and the largest delay
        int32_t span = 0, mx = 0;
        for (int d0 = 0; d0 < n_dm; d0 += fdas::kDdD) {
            const int d1 = std::min(n_dm - 1, d0 + fdas::kDdD - 1);
            for (int c = 0; c < n_chan; ++c) {
                const int32_t lo = p->host_delays[(size_t)d0 * n_chan + c];
                const int32_t hi = p->host_delays[(size_t)d1 * n_chan + c];
                span = std::max(span, hi - lo);
                mx = std::max(mx, hi);
            }
        }
        p->span = span;
        p->max_delay = mx;
        p->win = (fdas::kDdT + span + 31) / 32 * 32;
        const size_t per_chan = 2 * sizeof(float) * (size_t)p->win;   // double buffered
        if (per_chan > fdas::kDdSmemCap) {
            fdas::set_error("dedispersion: the delays of 32 consecutive DM trials spread over more "
                            "than " + std::to_string(fdas::kDdSmemCap / 8 - fdas::kDdT) +
                            " samples; use a smaller dm_step");
            return fail(FDAS_ERR_UNSUPPORTED);
        }
        p->chan_batch = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_chan));
        // 8-bit windows: a quarter of the bytes, so more channels per batch
        const size_t per_chan_u8 = 2 * (size_t)(p->win + 16);
        p->chan_batch_u8 = (int)std::max<size_t>(1, std::min<size_t>(16, (96 * 1024) / per_chan_u8));
        *out = reinterpret_cast<fdas_dedisp_plan *>(p);
        return FDAS_OK;
    } catch (...) {
        fdas::set_error("unexpected C++ exception in fdas_dedisp_plan_create");
        return FDAS_ERR_CUDA;
    }
}

void fdas_dedisp_plan_destroy(fdas_dedisp_plan *plan) {
    if (!plan) return;
    DedispPlan *p = reinterpret_cast<DedispPlan *>(plan);
    cudaFree(p->delays);
    delete p;
}

fdas_status fdas_dedisp_get_info(const fdas_dedisp_plan *plan, fdas_dedisp_info *info) {
    if (!plan || !info) return dd_arg("NULL argument");
    const DedispPlan &p = *reinterpret_cast<const DedispPlan *>(plan);
    info->n_chan = p.n_chan;
    info->n_dm = p.n_dm;
    info->n_t = p.n_t;
    info->n_out = p.n_out;
    info->f_top_mhz = p.f_top;
    info->df_mhz = p.df;
    info->tsamp = p.tsamp;
    info->dm_lo = p.dm_lo;
    info->dm_step = p.dm_step;
    info->max_delay = p.max_delay;
    info->tile_span = p.span;
    info->workspace_bytes = (int64_t)sizeof(int32_t) * p.n_chan * p.n_dm;
    return FDAS_OK;
}

fdas_status fdas_dedisp_delays(const fdas_dedisp_plan *plan, int32_t *delays_out) {
    if (!plan || !delays_out) return dd_arg("NULL argument");
    const DedispPlan &p = *reinterpret_cast<const DedispPlan *>(plan);
    std::copy(p.host_delays.begin(), p.host_delays.end(), delays_out);
    return FDAS_OK;
}

fdas_status fdas_dedisperse(fdas_dedisp_plan *plan, const float *filterbank, float *out,
                            void *stream) {
    if (!plan || !filterbank || !out) return dd_arg("NULL argument");
    return fdas::launch_dedisperse(*reinterpret_cast<DedispPlan *>(plan), filterbank, out,
                                   (cudaStream_t)stream);
}

fdas_status fdas_dedisperse_u8(fdas_dedisp_plan *plan, const uint8_t *filterbank, float *out,
                               void *stream) {
    if (!plan || !filterbank || !out) return dd_arg("NULL argument");
    DedispPlan &p = *reinterpret_cast<DedispPlan *>(plan);
    if (p.n_t % 16 != 0 || ((uintptr_t)filterbank & 15u) != 0)
        return dd_arg("8-bit filterbanks need n_t a multiple of 16 and a 16-byte aligned pointer");
    return fdas::launch_dedisperse(p, filterbank, out, (cudaStream_t)stream);
}

}  // extern "C"
