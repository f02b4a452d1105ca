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
// multiplied by W_tw^{c k} when TW (tw_m > 0).  Thread i of the CTA works on
// transform W blockIdx + i % W as its thread i / W, so that with in_cs = 1
// (or out_cs = 1) a warp's strided accesses touch W consecutive elements of
// each of 32 / W rows instead of one element per 32-byte sector.
// Elements between the W transforms' buffers: the padded length rounded up
// so that buffer g starts g * 32/W banks further on.  The W lanes that share
// a thread index then hit disjoint banks, also within the half-warp in which
// 8-byte accesses are served.
template <int L, int W>
__host__ __device__ constexpr int fft_buf_stride() {
    constexpr int E = CtaFft<L, -1>::SMEM_ELEMS;
    return W == 1 ? E : E + ((16 / W - E % 16) % 16 + 16) % 16;
}

template <int L, int W, bool TW>
__global__ void __launch_bounds__(W * (L / 16), 1024 / (W * (L / 16))) fft_strided_kernel(const float2 *__restrict__ in,
                                                                   float2 *__restrict__ out,
                                                                   int64_t in_cs, int64_t in_es,
                                                                   int64_t out_cs, int64_t out_es,
                                                                   int64_t tw_m) {
    using F = CtaFft<L, -1>;
    extern __shared__ float2 smem_fft[];
    const int g = threadIdx.x % W;
    const int tid = threadIdx.x / W;
    const int64_t c = (int64_t)blockIdx.x * W + g;
    float2 *buf = smem_fft + g * fft_buf_stride<L, W>();
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = in[c * in_cs + (int64_t)(tid + r * (L / 16)) * in_es];
    float2 tw[F::NPASS];
    F::make_twiddles(tid, tw);
    float2 o[16];
    F::to_regs(v, buf, tid, tw, o);
    constexpr int K = F::NPASS - 1;
    constexpr int R = F::template Pass<K>::R, NB = F::template Pass<K>::NB;
    constexpr int Ns = F::template Pass<K>::Ns;
    // output k = tid + b T + r Ns (last_index) takes W_tw^{c k} = W^{c tid}
    // W^{c b T} (W^{c Ns})^r: one sincospi per butterfly and one for the
    // stride, the powers of the stride by a product tree (depth <= 4)
    float2 wb[NB], pw[R];
    if constexpr (TW) {
        const int64_t msk = tw_m - 1;                 // tw_m is a power of two
        const float sc = -2.0f / (float)tw_m;         // exact: the arguments are exact
        auto w_of = [&](int64_t e) {
            float s, co;
            sincospif((float)(e & msk) * sc, &s, &co);
            return make_float2(co, s);
        };
#pragma unroll
        for (int b = 0; b < NB; ++b) wb[b] = w_of(c * (int64_t)(tid + b * F::T));
        pw[0] = make_float2(1.f, 0.f);
        pw[1] = w_of(c * (int64_t)Ns);
#pragma unroll
        for (int r = 2; r < R; ++r) pw[r] = cmul(pw[r / 2], pw[r - r / 2]);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = F::last_index(tid, b, r);
            float2 y = o[b * R + r];
            if constexpr (TW) y = cmul(y, r == 0 ? wb[b] : cmul(wb[b], pw[r]));
            out[c * out_cs + (int64_t)k * out_es] = y;
        }
}

template <int L, int W>
fdas_status launch_fft_w(const float2 *in, float2 *out, int n_cta, int64_t in_cs, int64_t in_es,
                         int64_t out_cs, int64_t out_es, int64_t tw_m, cudaStream_t s) {
    const size_t smem = sizeof(float2) * W * fft_buf_stride<L, W>();
    auto k = tw_m > 0 ? fft_strided_kernel<L, W, true> : fft_strided_kernel<L, W, false>;
    FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<n_cta / W, W * (L / 16), smem, s>>>(in, out, in_cs, in_es, out_cs, out_es, tw_m);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

// several transforms per CTA where the count allows (the strided passes of
// the four-step split come in powers of two), so that each strided access
// of a warp covers W consecutive elements
constexpr int kFftWideMax = 4;
template <int L>
fdas_status launch_fft(const float2 *in, float2 *out, int n_cta, int64_t in_cs, int64_t in_es,
                       int64_t out_cs, int64_t out_es, int64_t tw_m, cudaStream_t s) {
    if constexpr (L <= 2048 && kFftWideMax >= 4) {
        if (n_cta % 4 == 0)
            return launch_fft_w<L, 4>(in, out, n_cta, in_cs, in_es, out_cs, out_es, tw_m, s);
    }
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

constexpr int kNormThreads = 256;
constexpr int kNormWarps = kNormThreads / 32;
constexpr int kTopShift = 19;                    // first digit: bits 31..19 of the key
constexpr int kTopBins = 1 << (32 - kTopShift);  // 8192 (two 16-bit counters per word)
constexpr int kListCap = 2 * kNormThreads;       // keys of the median's bin ranked directly
static_assert(kTopBins % (16 * kNormThreads) == 0, "whole 16-byte groups of packed counters");
static_assert(((kTopBins / (16 * kNormThreads)) & (kTopBins / (16 * kNormThreads) - 1)) == 0,
              "a power-of-two number of 16-byte loads per thread");

// CTA-wide exclusive position of rank `r` in a histogram of `nb` counters
// (16-bit halves of `words` when `packed`, else one counter per word): the
// counter c holding rank r, the number of keys below it and its count.
// Thread t scans the nb / T consecutive counters it owns; every thread
// returns with res[0..2] set.
__device__ __forceinline__ void hist_locate(const uint32_t *words, int nb, bool packed, uint32_t r,
                                            uint32_t *wsum, uint32_t *res) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = nb / kNormThreads;   // counters per thread
    uint32_t local = 0u;
    if (packed) {
        // per counters = per / 2 words, in 16-byte loads; thread t starts at
        // its (t / 2)-th load (mod the count), so the 8 lanes of a
        // quarter-warp read distinct banks (the sum does not depend on order)
        const int nq = per / 8;
        const uint4 *w4 = reinterpret_cast<const uint4 *>(words) + tid * nq;
        for (int q = 0; q < nq; ++q) {
            const uint4 a = w4[(q + (tid >> 1)) & (nq - 1)];
            local += (a.x & 0xffffu) + (a.x >> 16) + (a.y & 0xffffu) + (a.y >> 16) +
                     (a.z & 0xffffu) + (a.z >> 16) + (a.w & 0xffffu) + (a.w >> 16);
        }
    } else {
        for (int q = 0; q < per; ++q) local += words[tid * per + q];
    }
    uint32_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    // exclusive prefix of the warp totals, by a shuffle scan in every warp
    uint32_t ws = lane < kNormWarps ? wsum[lane] : 0u;
#pragma unroll
    for (int off = 1; off < kNormWarps; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, ws, off);
        if (lane >= off) ws += v;
    }
    const uint32_t wbase = __shfl_sync(0xffffffffu, ws, (warp + 31) & 31);
    const uint32_t base = incl - local + (warp > 0 ? wbase : 0u);
    if (r >= base && r < base + local) {
        uint32_t before = base;
        for (int q = 0; q < per; ++q) {
            const int c = tid * per + q;
            const uint32_t n = packed ? (words[c >> 1] >> ((c & 1) * 16)) & 0xffffu : words[c];
            if (r >= before && r < before + n) {
                res[0] = (uint32_t)c;
                res[1] = before;
                res[2] = n;
            }
            before += n;
        }
    }
    __syncthreads();
}

// Rank `r` among the keys key[0..n) whose bits under `mask` equal `prefix`
// (r counted within them), by radix selection on the remaining low bits
// 18..0 in digits of 11 and 8 bits: each pass counts the keys that share the
// prefix found so far per digit value and keeps the digit whose range holds
// the rank.  All threads of the CTA call it; every thread gets the key.
__device__ __forceinline__ uint32_t radix_select_low(const uint32_t *key, int n, uint32_t r, uint32_t prefix,
                                     uint32_t mask, uint32_t *hist, uint32_t *wsum,
                                     uint32_t *res) {
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const int shift = pass == 0 ? 8 : 0;
        const int nb = pass == 0 ? 2048 : 512;   // 11- and 9-bit counters (bit 8 is 0 by then)
        for (int i = tid; i < nb; i += kNormThreads) hist[i] = 0u;
        __syncthreads();
        for (int i = tid; i < n; i += kNormThreads) {
            const uint32_t k = key[i];
            if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & (uint32_t)(nb - 1)], 1u);
        }
        __syncthreads();
        hist_locate(hist, nb, false, r, wsum, res);
        prefix |= res[0] << shift;
        mask |= (uint32_t)(nb - 1) << shift;
        r -= res[1];
        __syncthreads();   // res and hist are rewritten by the next pass
    }
    return prefix;
}

// One CTA per normalisation block of B bins (B a power of two <= 8192).
// The median's first digit (bits 31..19 of the power's bit pattern: sign,
// exponent and 4 mantissa bits) comes from a histogram built while the
// powers are computed; the keys in that digit's bin (typically a few dozen)
// are gathered and ranked by direct counting, and the rank above the lower
// middle (even counts) is either in the bin too or the smallest key of the
// bins above it.  A bin of more than kListCap keys (e.g. many equal powers)
// is resolved by radix passes over the low 19 bits instead.
template <class P>
__global__ void __launch_bounds__(kNormThreads) normalise_kernel(
    const float2 *__restrict__ Z, typename P::cpx *__restrict__ out, float *__restrict__ medians,
    unsigned int *__restrict__ flags, int64_t M, int B, int median_mode) {
    extern __shared__ float smem[];
    float *key = smem;                       // [B]
    float2 *xs = (float2 *)(smem + B);       // [B]
    __shared__ __align__(16) uint32_t hist[kTopBins / 2];
    __shared__ uint32_t list[kListCap];
    __shared__ uint32_t wsum[kNormWarps], res[4], n_list, red[kNormWarps];
    const int tid = threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.x * B;
    const int64_t N = 2 * M;
    const bool med_on = median_mode == FDAS_NORM_MEDIAN;
    if (med_on) {
        for (int i = tid; i < kTopBins / 8; i += kNormThreads)
            reinterpret_cast<uint4 *>(hist)[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) n_list = 0u;
        __syncthreads();
    }
    bool bad = false;
    // W_N^k for this thread's k = k0 + tid + m T: sincospi at every fourth m
    // (k and 2/N are exact in FP32, N a power of two <= 2^24, so the
    // argument -2k/N is exact), times W_N^T in between
    const float sc = -2.0f / (float)N;
    float2 step;
    sincospif((float)kNormThreads * sc, &step.y, &step.x);
    float2 w = make_float2(1.f, 0.f);
    // up to four bins per thread at a time: their loads are all issued
    // before the first is used
    constexpr int U = 4;
    for (int i0 = 0, m = 0; i0 < B; i0 += U * kNormThreads) {
        float2 zk[U], zm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t k = k0 + i0 + tid + u * kNormThreads;
            const bool in = i0 + tid + u * kNormThreads < B && k != 0;
            zk[u] = in ? Z[k] : make_float2(0.f, 0.f);
            zm[u] = in ? Z[M - k] : make_float2(0.f, 0.f);   // 0 < k < M
        }
#pragma unroll
        for (int u = 0; u < U; ++u, ++m) {
            const int i = i0 + tid + u * kNormThreads;
            if (i >= B) break;
            const int64_t k = k0 + i;
            if ((m & 3) == 0) sincospif((float)k * sc, &w.y, &w.x);
            else w = cmul(w, step);
            float2 X = make_float2(0.f, 0.f);
            float p = __int_as_float(0x7f800000);   // +inf: k = 0 sorts last
            if (k != 0) {
                const float2 e = make_float2(0.5f * (zk[u].x + zm[u].x), 0.5f * (zk[u].y - zm[u].y));
                // (Z_k - conj(Z_{M-k})) / (2i)
                const float2 d = make_float2(zk[u].x - zm[u].x, zk[u].y + zm[u].y);
                const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);
                X = cadd(e, cmul(w, o));
                p = X.x * X.x + X.y * X.y;
                if (!isfinite(p)) bad = true;
            }
            key[i] = p;
            xs[i] = X;
            if (med_on) {
                const uint32_t u32 = __float_as_uint(p);
                atomicAdd(&hist[u32 >> (kTopShift + 1)], 1u << (((u32 >> kTopShift) & 1u) * 16u));
            }
        }
    }
    if (bad) atomicOr(flags, 1u);
    __syncthreads();
    float f = 1.0f;
    if (med_on) {
        // the middle order statistics of |X_k|^2 (the +inf key of k = 0 is
        // the largest and never selected)
        const uint32_t *ukey = reinterpret_cast<const uint32_t *>(key);
        const int cnt = (k0 == 0) ? B - 1 : B;
        const uint32_t r_lo = (uint32_t)((cnt & 1) ? cnt / 2 : cnt / 2 - 1);
        const bool two = !(cnt & 1);   // even count: also rank r_lo + 1
        hist_locate(hist, kTopBins, true, r_lo, wsum, res);
        const uint32_t dig = res[0], below = res[1], n_dig = res[2];
        const uint32_t rl = r_lo - below;   // rank within the bin
        const bool hi_in_bin = rl + 1 < n_dig;
        // the bin's keys into the list (if they fit) and the smallest key of
        // the bins above it
        uint32_t m_gt = 0xffffffffu;
        for (int i = tid; i < B; i += kNormThreads) {
            const uint32_t u = ukey[i];
            const uint32_t du = u >> kTopShift;
            if (du == dig) {
                if (n_dig <= (uint32_t)kListCap) list[atomicAdd(&n_list, 1u)] = u;
            } else if (du > dig) {
                m_gt = min(m_gt, u);
            }
        }
        if (two && !hi_in_bin) {
            m_gt = __reduce_min_sync(0xffffffffu, m_gt);
            if ((tid & 31) == 0) red[tid >> 5] = m_gt;
        }
        __syncthreads();
        uint32_t lo, hi = 0u;
        if (n_dig <= (uint32_t)kListCap) {
            // rank of each listed key by counting: G threads per key (a
            // power of two <= 32 with G * n_dig <= T where possible), the
            // partial counts reduced within the warp
            int lg = 5;
            while (lg > 0 && (n_dig << lg) > (uint32_t)kNormThreads) --lg;
            const int G = 1 << lg, sub = tid & (G - 1);
            const uint32_t per_it = (uint32_t)(kNormThreads >> lg);   // keys per round
            const uint32_t n_it = (n_dig + per_it - 1) / per_it;
            for (uint32_t it = 0; it < n_it; ++it) {
                const uint32_t e = (uint32_t)(tid >> lg) + it * per_it;
                const bool valid = e < n_dig;
                const uint32_t v = valid ? list[e] : 0u;
                uint32_t less = 0u, eq = 0u;
                if (valid)
                    for (uint32_t j = (uint32_t)sub; j < n_dig; j += (uint32_t)G) {
                        const uint32_t w = list[j];
                        less += w < v;
                        eq += w == v;
                    }
                for (int off = G >> 1; off > 0; off >>= 1) {
                    less += __shfl_xor_sync(0xffffffffu, less, off);
                    eq += __shfl_xor_sync(0xffffffffu, eq, off);
                }
                if (sub == 0 && valid) {
                    if (rl >= less && rl < less + eq) res[0] = v;
                    if (two && hi_in_bin && rl + 1 >= less && rl + 1 < less + eq) res[1] = v;
                }
            }
            __syncthreads();
            lo = res[0];
            if (two && hi_in_bin) hi = res[1];
        } else {
            lo = radix_select_low(ukey, B, rl, dig << kTopShift, ~0u << kTopShift, hist, wsum,
                                  res);
            if (two && hi_in_bin) {
                // lo again if it also has rank rl + 1, else the smallest key
                // of the bin above lo
                uint32_t n_le = 0u, m_bin = 0xffffffffu;
                for (int i = tid; i < B; i += kNormThreads) {
                    const uint32_t u = ukey[i];
                    if ((u >> kTopShift) != dig) continue;
                    if (u <= lo) ++n_le;
                    else m_bin = min(m_bin, u);
                }
                n_le = __reduce_add_sync(0xffffffffu, n_le);
                m_bin = __reduce_min_sync(0xffffffffu, m_bin);
                if ((tid & 31) == 0) {
                    wsum[tid >> 5] = n_le;
                    list[tid >> 5] = m_bin;
                }
                __syncthreads();
                uint32_t tot = 0u, mn = 0xffffffffu;
                for (int w = 0; w < kNormWarps; ++w) {
                    tot += wsum[w];
                    mn = min(mn, list[w]);
                }
                hi = tot >= rl + 2 ? lo : mn;
            }
        }
        if (two && !hi_in_bin) {
            uint32_t mn = 0xffffffffu;
            for (int w = 0; w < kNormWarps; ++w) mn = min(mn, red[w]);
            hi = mn;
        }
        float med = __uint_as_float(lo);
        if (two) med = 0.5f * (__uint_as_float(lo) + __uint_as_float(hi));
        // FP32 division and square root, each correctly rounded (FP64 is a
        // small fraction of the FP32 rate on this GPU, and the factor is
        // applied in FP32)
        f = med > 0.f ? sqrtf(0.69314718055994530942f / med) : 0.f;
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
