// R2C FFT of one series and median normalisation (the input of the
// convolution stage of paper §2.2).
//
// The N real samples are read as M = N/2 complex values z_n = x_{2n} +
// i x_{2n+1}.  Their M-point FFT Z_k (one CTA when M <= 8192, otherwise the
// four-step split M = M1 * M2: M1 column FFTs of length M2 with the twiddle
// W_M^{n1 k2}, then M2 FFTs of length M1) gives the real-input spectrum
//
//     X_k = (Z_k + conj(Z_{M-k}))/2 - (i/2) W_N^k (Z_k - conj(Z_{M-k})),
//
// k in [0, M) (Z_M = Z_0), with X_0 set to 0.  The normalisation kernel then
// takes blocks of B bins, selects the middle order statistics of |X_k|^2
// (radix selection on their bit patterns, shared memory), takes the median
// mu_b (block 0 without k = 0; the mean of the two middle values for an even
// count) and stores X'_k = X_k sqrt(ln 2 / mu_b) at the plan's
// precision: exponential noise has median ln 2 times its mean, so white noise
// leaves with unit mean power.  Non-finite spectrum values raise a flag.
#include "fdas_internal.cuh"
#include "fft_cta.cuh"

#include <algorithm>

namespace fdas {
namespace {

// Strided FFTs of length L, W per CTA: input element n of transform c at
// in[c*in_cs + n*in_es], output element k to out[c*out_cs + k*out_es],
// multiplied by W_tw^{c k} when tw_m > 0.  Thread i of the CTA works on
// transform W blockIdx + i % W as its thread i / W, so that with in_cs = 1
// (or out_cs = 1) a warp's strided accesses touch W consecutive elements of
// each of 32 / W rows instead of one element per 32-byte sector.
template <int L, int W>
__global__ void __launch_bounds__(W * (L / 16)) fft_strided_kernel(const float2 *__restrict__ in,
                                                                   float2 *__restrict__ out,
                                                                   int64_t in_cs, int64_t in_es,
                                                                   int64_t out_cs, int64_t out_es,
                                                                   int64_t tw_m) {
    using F = CtaFft<L, -1>;
    extern __shared__ float2 smem_fft[];
    const int g = threadIdx.x % W;
    const int tid = threadIdx.x / W;
    const int64_t c = (int64_t)blockIdx.x * W + g;
    float2 *buf = smem_fft + g * F::SMEM_ELEMS;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = in[c * in_cs + (int64_t)(tid + r * (L / 16)) * in_es];
    float2 tw[F::NPASS];
    F::make_twiddles(tid, tw);
    float2 o[16];
    F::to_regs(v, buf, tid, tw, o);
    constexpr int K = F::NPASS - 1;
    constexpr int R = F::template Pass<K>::R, NB = F::template Pass<K>::NB;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = F::last_index(tid, b, r);
            float2 y = o[b * R + r];
            if (tw_m > 0) {
                const int64_t e = (c * k) % tw_m;
                float s, co;
                sincospif(-2.0f * (float)e / (float)tw_m, &s, &co);
                y = cmul(y, make_float2(co, s));
            }
            out[c * out_cs + (int64_t)k * out_es] = y;
        }
}

template <int L, int W>
fdas_status launch_fft_w(const float2 *in, float2 *out, int n_cta, int64_t in_cs, int64_t in_es,
                         int64_t out_cs, int64_t out_es, int64_t tw_m, cudaStream_t s) {
    const size_t smem = sizeof(float2) * W * CtaFft<L, -1>::SMEM_ELEMS;
    FDAS_CUDA_TRY(cudaFuncSetAttribute(fft_strided_kernel<L, W>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fft_strided_kernel<L, W><<<n_cta / W, W * (L / 16), smem, s>>>(in, out, in_cs, in_es, out_cs,
                                                                     out_es, tw_m);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

// two transforms per CTA where the count allows (the strided passes of the
// four-step split come in powers of two; two measured faster than four,
// which limits the SM to one 512-thread CTA)
template <int L>
fdas_status launch_fft(const float2 *in, float2 *out, int n_cta, int64_t in_cs, int64_t in_es,
                       int64_t out_cs, int64_t out_es, int64_t tw_m, cudaStream_t s) {
    if constexpr (L <= 4096) {
        if (n_cta % 2 == 0)
            return launch_fft_w<L, 2>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
    }
    return launch_fft_w<L, 1>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
}

fdas_status fft_any(int L, const float2 *in, float2 *out, int n_cta, int64_t in_cs, int64_t in_es,
                    int64_t out_cs, int64_t out_es, int64_t tw_m, cudaStream_t s) {
    switch (L) {
        case 128: return launch_fft<128>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        case 256: return launch_fft<256>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        case 512: return launch_fft<512>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        case 1024: return launch_fft<1024>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        case 2048: return launch_fft<2048>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        case 4096: return launch_fft<4096>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        case 8192: return launch_fft<8192>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
        default:
            set_error("internal: unsupported FFT length " + std::to_string(L));
            return FDAS_ERR_UNSUPPORTED;
    }
}

constexpr int kNormThreads = 512;
constexpr int kSelBins = 2048;   // radix-select digit of up to 11 bits

// Rank `r` (0-based, ascending) among the n keys key[0..n) (non-negative
// float bit patterns, so their order as unsigned integers is their order as
// floats), by radix selection on digits of 11, 11 and 10 bits: each pass
// counts the keys that share the prefix found so far per digit value,
// scans the counts and keeps the digit whose range holds the rank.  All
// threads of the CTA call it; returns the key (every thread gets it).
__device__ uint32_t radix_select(const uint32_t *key, int n, int r, uint32_t *hist,
                                 uint32_t *wsum, uint32_t *res) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t prefix = 0u, mask = 0u;
    int rr = r;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
        const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
        const int nb = pass == 2 ? 1024 : 2048;
        for (int i = tid; i < kSelBins; i += kNormThreads) hist[i] = 0u;
        __syncthreads();
        for (int i = tid; i < n; i += kNormThreads) {
            const uint32_t k = key[i];
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & (uint32_t)(nb - 1)], 1u);
        }
        __syncthreads();
        // thread t owns the 4 consecutive bins 4t .. 4t+3
        uint32_t c[4], local = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            c[q] = hist[4 * tid + q];
            local += c[q];
        }
        uint32_t incl = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t base = incl - local;
        for (int w = 0; w < warp; ++w) base += wsum[w];
        if ((uint32_t)rr >= base && (uint32_t)rr < base + local) {
            uint32_t before = base;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((uint32_t)rr >= before && (uint32_t)rr < before + c[q]) {
                    res[0] = (uint32_t)(4 * tid + q);
                    res[1] = before;
                }
                before += c[q];
            }
        }
        __syncthreads();
        const uint32_t digit = res[0], below = res[1];
        prefix |= digit << shift;
        mask |= (uint32_t)(nb - 1) << shift;
        rr -= (int)below;
        __syncthreads();   // res is rewritten by the next pass
    }
    return prefix;
}

// One CTA per normalisation block of B bins (B a power of two <= 8192).
template <class P>
__global__ void __launch_bounds__(kNormThreads) normalise_kernel(
    const float2 *__restrict__ Z, typename P::cpx *__restrict__ out, float *__restrict__ medians,
    unsigned int *__restrict__ flags, int64_t M, int B, int median_mode) {
    extern __shared__ float smem[];
    float *key = smem;                       // [B]
    float2 *xs = (float2 *)(smem + B);       // [B]
    __shared__ uint32_t hist[kSelBins];
    __shared__ uint32_t wsum[kNormThreads / 32], res[2];
    __shared__ uint32_t red_cnt[kNormThreads / 32], red_min[kNormThreads / 32];
    const int tid = threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.x * B;
    const int64_t N = 2 * M;
    bool bad = false;
    for (int i = tid; i < B; i += kNormThreads) {
        const int64_t k = k0 + i;
        float2 X = make_float2(0.f, 0.f);
        float p = __int_as_float(0x7f800000);   // +inf: k = 0 sorts last
        if (k != 0) {
            const float2 zk = Z[k];
            const float2 zm = Z[(M - k) % M];
            const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            // (Z_k - conj(Z_{M-k})) / (2i)
            const float2 d = make_float2(zk.x - zm.x, zk.y + zm.y);
            const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
            float sn, cs;
            sincospif(-2.0f * (float)k / (float)N, &sn, &cs);
            X = cadd(e, cmul(make_float2(cs, sn), o));
            p = X.x * X.x + X.y * X.y;
            if (!isfinite(p)) bad = true;
        }
        key[i] = p;
        xs[i] = X;
    }
    if (bad) atomicOr(flags, 1u);
    __syncthreads();
    float f = 1.0f;
    if (median_mode == FDAS_NORM_MEDIAN) {
        // the middle order statistics of |X_k|^2 by radix selection (the +inf
        // key of k = 0 is the largest and never selected)
        const uint32_t *ukey = reinterpret_cast<const uint32_t *>(key);
        const int cnt = (k0 == 0) ? B - 1 : B;
        const int r_lo = (cnt & 1) ? cnt / 2 : cnt / 2 - 1;
        const uint32_t lo = radix_select(ukey, B, r_lo, hist, wsum, res);
        float med = __uint_as_float(lo);
        if (!(cnt & 1)) {
            // the next order statistic: lo again if it occurs at rank r_lo + 1,
            // else the smallest key above lo
            uint32_t n_le = 0u, m_gt = 0xffffffffu;
            for (int i = tid; i < B; i += kNormThreads) {
                const uint32_t k = ukey[i];
                if (k <= lo) ++n_le;
                else m_gt = min(m_gt, k);
            }
            n_le = __reduce_add_sync(0xffffffffu, n_le);
            m_gt = __reduce_min_sync(0xffffffffu, m_gt);
            if ((tid & 31) == 0) {
                red_cnt[tid >> 5] = n_le;
                red_min[tid >> 5] = m_gt;
            }
            __syncthreads();
            uint32_t tot = 0u, mn = 0xffffffffu;
            for (int w = 0; w < kNormThreads / 32; ++w) {
                tot += red_cnt[w];
                mn = min(mn, red_min[w]);
            }
            const uint32_t hi = tot >= (uint32_t)(r_lo + 2) ? lo : mn;
            med = 0.5f * (__uint_as_float(lo) + __uint_as_float(hi));
        }
        f = med > 0.f ? (float)sqrt(0.69314718055994530942 / (double)med) : 0.f;
        if (medians != nullptr && tid == 0) medians[blockIdx.x] = med;
    }
    for (int i = tid; i < B; i += kNormThreads) out[k0 + i] = P::st(cscale(xs[i], f));
}

}  // namespace

fdas_status launch_spectrum(Plan &p, const float *x, void *spec_out, float *medians,
                            cudaStream_t s) {
    const int64_t M = p.n_r;
    const float2 *z = (const float2 *)x;
    if (p.fft_m1 == 1) {
        FDAS_TRY(fft_any((int)M, z, p.fft_b, 1, 0, 1, 0, 1, 0, s));
    } else {
        const int64_t m1 = p.fft_m1, m2 = p.fft_m2;
        // columns: n1 = CTA, length m2 over z[n1 + m1 n2]; twiddle W_M^{n1 k2}
        FDAS_TRY(fft_any((int)m2, z, p.fft_a, (int)m1, 1, m1, m2, 1, M, s));
        // rows: k2 = CTA, length m1 over a[n1 m2 + k2]; out[k2 + m2 k1]
        FDAS_TRY(fft_any((int)m1, p.fft_a, p.fft_b, (int)m2, 1, m2, 1, m2, 0, s));
    }
    const int B = (int)std::min<int64_t>(p.norm_block, M);
    const int nb = (int)(M / B);
    const size_t smem = (size_t)B * (sizeof(float) + sizeof(float2));
    switch (p.prec) {
        case FDAS_FP32: {
            auto k = normalise_kernel<PrecF32>;
            FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k<<<nb, kNormThreads, smem, s>>>(p.fft_b, (float2 *)spec_out, medians, p.flags, M, B, p.norm_mode);
            break;
        }
        case FDAS_BF16: {
            auto k = normalise_kernel<PrecBF16>;
            FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k<<<nb, kNormThreads, smem, s>>>(p.fft_b, (__nv_bfloat162 *)spec_out, medians, p.flags, M, B,
                                             p.norm_mode);
            break;
        }
        default: {
            auto k = normalise_kernel<PrecF16>;
            FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k<<<nb, kNormThreads, smem, s>>>(p.fft_b, (__half2 *)spec_out, medians, p.flags, M, B,
                                             p.norm_mode);
            break;
        }
    }
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

}  // namespace fdas
