// Fused overlap-save correlation -> |.|^2 power plane (the "convolution
// stage" of paper §2.2; the matched filter of §2.1), plus FP64 statistics.
//
// The normalised spectrum lives in a zero-padded buffer: element m_ov + k
// holds X'_k and everything outside k in [0, N_r) is 0, so segment s is the
// contiguous window [s V, s V + L) of the buffer (local index j <-> bin
// s V - m_ov + j).  One CTA takes one segment and a chunk of templates:
//
//   1. load the window and FFT it forward (CTA FFT, shared memory) -> S_s;
//   2. keep, in registers, the 16 values of S_s this thread feeds into the
//      first inverse pass;
//   3. for each template z of the chunk: Y = S_s * bank_z (bank_z already
//      holds FFT_L(g_z)/L), inverse FFT, and for the outputs j in
//      [m_ov, m_ov + V) the power |y_j|^2 = P(s V + j - m_ov, z) goes to the
//      plane (one coalesced store per output register).
//
// Since |e| <= m(z) <= m_ov the circular correlation equals the linear one on
// the kept outputs, so P is exactly sum_e X'_{r-e} g_z[e] squared.  Every
// thread sums P and P^2 of its 16 outputs per template in FP32 and adds those
// partial sums across templates with compensated (Kahan) FP32 sums; the CTA
// adds them in FP64 in a fixed order and writes one partial per CTA, which the
// statistics kernel reduces in a fixed order (deterministic mean and std).
//
// With kCplx the kernels write the complex F itself (plane of complex values
// at the plan's precision, no statistics): the input of interbinning.
#include "fdas_internal.cuh"
#include "fft_cta.cuh"
#include "fft8k.cuh"
#include "tma.cuh"

namespace fdas {
namespace {

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <int L, class P, bool kCplx>
__global__ void __launch_bounds__(L / 16, 1)
    correlate_kernel(const typename P::cpx *__restrict__ spec_pad,
                     const typename P::cpx *__restrict__ bank, void *__restrict__ out,
                     double2 *__restrict__ partials, int64_t n_r, int n_z, int V, int m_ov,
                     int z_per_cta, float bank_scale) {
    using Fw = CtaFft<L, -1>;
    using Iv = CtaFft<L, +1>;
    constexpr int T = L / 16;
    extern __shared__ float2 buf[];
    __shared__ double red[2][T / 32];
    const int tid = threadIdx.x;
    const int64_t seg0 = (int64_t)blockIdx.x * V;
    const int iz_begin = blockIdx.y * z_per_cta;
    const int iz_end = min(n_z, iz_begin + z_per_cta);

    float2 v[16], S[16], tw[Fw::NPASS];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = P::ld(spec_pad[seg0 + tid + r * T]);
    Fw::make_twiddles(tid, tw);
    Fw::to_smem(v, buf, tid, tw);
#pragma unroll
    for (int r = 0; r < 16; ++r) S[r] = cscale(buf[fft_pad(tid + r * T)], bank_scale);
    Iv::make_twiddles(tid, tw);

    Kahan sp, sq;
    constexpr int K = Iv::NPASS - 1;
    constexpr int R = Iv::template Pass<K>::R, NB = Iv::template Pass<K>::NB;
    for (int iz = iz_begin; iz < iz_end; ++iz) {
        __syncthreads();   // the previous last pass has read buf
        const typename P::cpx *h = bank + (int64_t)iz * L;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(S[r], P::ld(__ldg(h + tid + r * T)));
        float2 o[16];
        Iv::to_regs(v, buf, tid, tw, o);
        typename P::real *row = static_cast<typename P::real *>(out) + (int64_t)iz * n_r;
        typename P::cpx *crow = static_cast<typename P::cpx *>(out) + (int64_t)iz * n_r;
        float zs = 0.f, zq = 0.f;   // this template's 16 outputs, plain FP32
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int n = Iv::last_index(tid, b, r);
                const int64_t rr = seg0 + n - m_ov;
                if (n >= m_ov && n < m_ov + V && rr < n_r) {
                    const float2 y = o[b * R + r];
                    if constexpr (kCplx) {
                        crow[rr] = P::st(y);
                        continue;
                    }
                    const float pw = fmaf(y.x, y.x, y.y * y.y);
                    row[rr] = P::str(pw * P::plane_scale);
                    zs += pw;
                    zq = fmaf(pw, pw, zq);
                }
            }
        sp.add(zs);   // compensated across templates
        sq.add(zq);
    }
    // fixed-order FP64 reduction of the CTA's sums
    double a = (double)sp.s - (double)sp.c, b2 = (double)sq.s - (double)sq.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b2 += __shfl_down_sync(0xffffffffu, b2, off);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = a;
        red[1][tid >> 5] = b2;
    }
    __syncthreads();
    if (tid == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < T / 32; ++w) {
            ta += red[0][w];
            tb += red[1][w];
        }
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(ta, tb);
    }
}

// The same correlation for L = 8192 with 256 threads x 32 points (fft8k.cuh):
// two shared-memory exchanges per inverse transform instead of three.  The
// segment window and the template spectra reach shared memory by bulk
// asynchronous copies (cp.async.bulk + mbarrier): the spectrum of template
// z + 1 is in flight while the inverse FFT of template z runs.  A bounded
// wait that gives up sets bit 1 of `flags` and the CTA returns.
template <class P, bool kCplx>
__global__ void __launch_bounds__(256, 1)
    correlate8k_kernel(const typename P::cpx *__restrict__ spec_pad,
                       const typename P::cpx *__restrict__ bank, void *__restrict__ out,
                       double2 *__restrict__ partials, int64_t n_r, int n_z, int V, int m_ov,
                       int z_per_cta, float bank_scale, unsigned int *__restrict__ flags) {
    using Fw = Fft8k<-1>;
    using Iv = Fft8k<+1>;
    using cpx = typename P::cpx;
    constexpr int L = 8192;
    constexpr unsigned kBytes = L * sizeof(cpx);
    extern __shared__ __align__(16) float2 buf[];
    cpx *const hb0 = reinterpret_cast<cpx *>(buf + Fw::SMEM_ELEMS);   // two template slots
    cpx *const hb1 = hb0 + L;
    __shared__ __align__(8) uint64_t bars[3];   // segment, template slot 0, slot 1
    __shared__ double red[2][8];
    const int t = threadIdx.x;
    const int64_t seg0 = (int64_t)blockIdx.x * V;
    const int iz_begin = blockIdx.y * z_per_cta;
    const int iz_end = min(n_z, iz_begin + z_per_cta);

    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (t == 0) {
        mbar_arrive_expect_tx(&bars[0], kBytes);
        bulk_copy_g2s(hb1, spec_pad + seg0, kBytes, &bars[0]);
        if (iz_begin < iz_end) {
            mbar_arrive_expect_tx(&bars[1], kBytes);
            bulk_copy_g2s(hb0, bank + (int64_t)iz_begin * L, kBytes, &bars[1]);
        }
    }
    bool ok = mbar_wait(&bars[0], 0);
    if (__syncthreads_or(!ok)) {
        if (t == 0) atomicOr(flags, 2u);
        return;
    }

    float2 v[32], S[32], o[32], w1, w2;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int r = 0; r < 16; ++r) v[16 * b + r] = P::ld(hb1[t + 256 * b + 512 * r]);
    Fw::make_twiddles(t, w1, w2);
    Fw::pass0(v, buf, t);
    __syncthreads();
    Fw::pass1(buf, t, w1);
    Fw::pass2(buf, t, w2, o);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; ++r) buf[fft_pad(t + 256 * r)] = o[r];
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int r = 0; r < 16; ++r)
            S[16 * b + r] = cscale(buf[fft_pad(t + 256 * b + 512 * r)], bank_scale);
    Iv::make_twiddles(t, w1, w2);
    // the segment copy in slot 1 has been read by every thread: refill it with
    // the second template
    if (t == 0 && iz_begin + 1 < iz_end) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[2], kBytes);
        bulk_copy_g2s(hb1, bank + (int64_t)(iz_begin + 1) * L, kBytes, &bars[2]);
    }
    // CTA-uniform: every output but r = 0 and r = 31 is kept, and those two
    // by a per-thread test, unless the overlap is wide or this is the last
    // segment (then every output is tested)
    const bool interior = m_ov <= 256 && seg0 + L - m_ov <= n_r;
    const bool keep0 = t >= m_ov;
    const bool keep31 = t + 256 * 31 < m_ov + V;

    Kahan sp, sq;
    unsigned phase0 = 0u, phase1 = 0u;   // next phase of each template slot
    for (int iz = iz_begin, k = 0; iz < iz_end; ++iz, ++k) {
        const int slot = k & 1;
        __syncthreads();   // the previous pass 2 has read buf
        ok = mbar_wait(&bars[1 + slot], slot ? phase1 : phase0);
        if (__syncthreads_or(!ok)) {
            if (t == 0) atomicOr(flags, 2u);
            return;
        }
        if (slot) phase1 ^= 1u;
        else phase0 ^= 1u;
        const cpx *h = hb0 + slot * L;
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int r = 0; r < 16; ++r)
                v[16 * b + r] = cmul(S[16 * b + r], P::ld(h[t + 256 * b + 512 * r]));
        Iv::pass0(v, buf, t);
        __syncthreads();
        // every thread has read template iz: its slot takes template iz + 2
        if (t == 0 && iz + 2 < iz_end) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[1 + slot], kBytes);
            bulk_copy_g2s(hb0 + slot * L, bank + (int64_t)(iz + 2) * L, kBytes, &bars[1 + slot]);
        }
        Iv::pass1(buf, t, w1);
        Iv::pass2(buf, t, w2, o);
        typename P::real *row = static_cast<typename P::real *>(out) + (seg0 - m_ov) + (int64_t)iz * n_r + t;
        typename P::cpx *crow = static_cast<typename P::cpx *>(out) + (seg0 - m_ov) + (int64_t)iz * n_r + t;
        float zs = 0.f, zq = 0.f;
        if constexpr (kCplx) {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int n = t + 256 * r;
                const int64_t rr = seg0 + n - m_ov;
                if (n >= m_ov && n < m_ov + V && rr < n_r) crow[256 * r] = P::st(o[r]);
            }
        } else if (interior) {
            // outputs r = 1..30 lie inside [m_ov, L - m_ov) when m_ov <= 256,
            // and inside the plane row when the segment is not the last
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                if ((r == 0 && !keep0) || (r == 31 && !keep31)) continue;
                const float pw = fmaf(o[r].x, o[r].x, o[r].y * o[r].y);
                row[256 * r] = P::str(pw * P::plane_scale);
                zs += pw;
                zq = fmaf(pw, pw, zq);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int n = t + 256 * r;
                const int64_t rr = seg0 + n - m_ov;
                if (n >= m_ov && n < m_ov + V && rr < n_r) {
                    const float pw = fmaf(o[r].x, o[r].x, o[r].y * o[r].y);
                    row[256 * r] = P::str(pw * P::plane_scale);
                    zs += pw;
                    zq = fmaf(pw, pw, zq);
                }
            }
        }
        sp.add(zs);
        sq.add(zq);
    }
    double a = (double)sp.s - (double)sp.c, b2 = (double)sq.s - (double)sq.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b2 += __shfl_down_sync(0xffffffffu, b2, off);
    }
    if ((t & 31) == 0) {
        red[0][t >> 5] = a;
        red[1][t >> 5] = b2;
    }
    __syncthreads();
    if (t == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 8; ++w) {
            ta += red[0][w];
            tb += red[1][w];
        }
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(ta, tb);
    }
}

template <class P, bool kCplx>
fdas_status launch_8k(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                      cudaStream_t s) {
    const size_t smem = sizeof(float2) * Fft8k<1>::SMEM_ELEMS + 2 * 8192 * sizeof(typename P::cpx);
    auto k = correlate8k_kernel<P, kCplx>;
    FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int zper = (p.n_z + p.n_zchunk - 1) / p.n_zchunk;
    dim3 grid(p.n_seg, p.n_zchunk);
    const float bank_scale = P::id == FDAS_FP16 ? 1.0f / (float)p.L : 1.0f;
    k<<<grid, 256, smem, s>>>((const typename P::cpx *)spec_padded, (const typename P::cpx *)p.bank,
                              plane, partials, p.n_r, p.n_z, p.V, p.m_ov, zper,
                              bank_scale, p.flags);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

template <int L, class P, bool kCplx>
fdas_status launch_L(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                     cudaStream_t s) {
    const size_t smem = sizeof(float2) * CtaFft<L, 1>::SMEM_ELEMS;
    auto k = correlate_kernel<L, P, kCplx>;
    FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int zper = (p.n_z + p.n_zchunk - 1) / p.n_zchunk;
    dim3 grid(p.n_seg, p.n_zchunk);
    const float bank_scale = P::id == FDAS_FP16 ? 1.0f / (float)p.L : 1.0f;
    k<<<grid, L / 16, smem, s>>>((const typename P::cpx *)spec_padded,
                                 (const typename P::cpx *)p.bank, plane,
                                 partials, p.n_r, p.n_z, p.V, p.m_ov, zper, bank_scale);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

template <class P, bool kCplx>
fdas_status launch_P(Plan &p, const void *spec, void *plane, double2 *partials, cudaStream_t s) {
    switch (p.L) {
        case 1024: return launch_L<1024, P, kCplx>(p, spec, plane, partials, s);
        case 2048: return launch_L<2048, P, kCplx>(p, spec, plane, partials, s);
        case 4096: return launch_L<4096, P, kCplx>(p, spec, plane, partials, s);
        case 8192: return launch_8k<P, kCplx>(p, spec, plane, partials, s);
        default:
            set_error("seg_len " + std::to_string(p.L) + " is not built");
            return FDAS_ERR_UNSUPPORTED;
    }
}

}  // namespace

int correlate_ctas(const Plan &p) {
    return p.correlator == FDAS_CORR_TENSOR ? correlate_tc_ctas(p) : p.n_seg * p.n_zchunk;
}

template <bool kCplx>
fdas_status launch_prec(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                        cudaStream_t s) {
    switch (p.prec) {
        case FDAS_FP32: return launch_P<PrecF32, kCplx>(p, spec_padded, plane, partials, s);
        case FDAS_BF16: return launch_P<PrecBF16, kCplx>(p, spec_padded, plane, partials, s);
        default: return launch_P<PrecF16, kCplx>(p, spec_padded, plane, partials, s);
    }
}

fdas_status launch_correlate(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                             cudaStream_t s, bool cplx) {
    if (p.correlator == FDAS_CORR_TENSOR)
        return launch_correlate_tc(p, spec_padded, plane, partials, s, cplx);
    return cplx ? launch_prec<true>(p, spec_padded, plane, partials, s)
                : launch_prec<false>(p, spec_padded, plane, partials, s);
}

}  // namespace fdas
