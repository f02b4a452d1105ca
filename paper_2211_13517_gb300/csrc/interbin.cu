// Interbinning: the power plane on a half-bin grid (r step 1/2) from the
// complex correlation F(r, z) of the matched filter (paper §2.1).
//
// Column 2r of a row holds |F(r)|^2 and column 2r + 1 the power half-way to
// the next bin, estimated from the two complex neighbours:
//
//     P(r + 1/2) = (pi/4)^2 |F(r) - F(r + 1)|^2,   F(N_r) = 0.
//
// (A sinusoid exactly between bins k and k + 1 has F(k) - F(k+1) equal to 4/pi
// times its full response, hence the factor.)  The plane is then
// n_z x 2 N_r and the statistics, harmonic sums and thresholds run on it as on
// the integer grid.
//
// One thread takes 4 consecutive bins of a row: one vector load of 4 complex
// values, F(r + 4) from the next lane (the last lane of a warp loads it, or
// uses 0 at the end of the row: rows are multiples of 128 bins, so a warp
// never straddles two), one vector store of the 8 plane values, and P and P^2
// summed in FP32 per thread, compensated across its groups, FP64 per CTA.  A
// fixed grid with a fixed stride makes the statistics deterministic.
#include <algorithm>

#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kIbThreads = 256;
constexpr int kIbCtasPerSm = 4;
constexpr float kIbPower = 0.61685027506808491f;   // (pi/4)^2

struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// 4 complex values <-> one 16- or 32-byte vector
template <class P>
struct Quad;
template <>
struct Quad<PrecF32> {
    __device__ __forceinline__ static void load(const float2 *p, float2 (&f)[4]) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        const float4 b = *reinterpret_cast<const float4 *>(p + 2);
        f[0] = make_float2(a.x, a.y);
        f[1] = make_float2(a.z, a.w);
        f[2] = make_float2(b.x, b.y);
        f[3] = make_float2(b.z, b.w);
    }
    __device__ __forceinline__ static void store8(float *p, const float (&v)[8]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
};
template <class P>
struct Quad16 {
    using cpx = typename P::cpx;
    __device__ __forceinline__ static void load(const cpx *p, float2 (&f)[4]) {
        const uint4 w = *reinterpret_cast<const uint4 *>(p);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cpx c;
            memcpy(&c, &ws[q], 4);
            f[q] = P::ld(c);
        }
    }
    __device__ __forceinline__ static void store8(typename P::real *p, const float (&v)[8]) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const cpx c = P::st(make_float2(v[2 * q] * P::plane_scale, v[2 * q + 1] * P::plane_scale));
            memcpy(&w[q], &c, 4);
        }
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <>
struct Quad<PrecBF16> : Quad16<PrecBF16> {};
template <>
struct Quad<PrecF16> : Quad16<PrecF16> {};

__device__ __forceinline__ float norm2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

template <class P>
__global__ void __launch_bounds__(kIbThreads)
    interbin_kernel(const typename P::cpx *__restrict__ F, typename P::real *__restrict__ plane,
                    double2 *__restrict__ partials, int64_t n_r, int64_t n_groups) {
    __shared__ double red[2][kIbThreads / 32];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kIbThreads;
    KahanF k1, k2;
    // every lane runs the same number of iterations (n_groups is a multiple
    // of 32 and so is the stride), so the shuffles see full warps
    for (int64_t g = (int64_t)blockIdx.x * kIbThreads + threadIdx.x; g < n_groups; g += stride) {
        const int64_t i = 4 * g;   // flat index of the first bin (row-major)
        float2 f[4];
        Quad<P>::load(F + i, f);
        float2 nx;
        nx.x = __shfl_down_sync(0xffffffffu, f[0].x, 1);
        nx.y = __shfl_down_sync(0xffffffffu, f[0].y, 1);
        if (lane == 31) {
            nx = make_float2(0.f, 0.f);
            if ((i + 4) % n_r != 0) nx = P::ld(F[i + 4]);
        }
        float v[8];
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 b = q < 3 ? f[q + 1] : nx;
            const float pe = norm2(f[q]);
            const float po = kIbPower * norm2(make_float2(f[q].x - b.x, f[q].y - b.y));
            v[2 * q] = pe;
            v[2 * q + 1] = po;
            s1 += pe + po;
            s2 = fmaf(pe, pe, fmaf(po, po, s2));
        }
        Quad<P>::store8(plane + 2 * i, v);
        k1.add(s1);
        k2.add(s2);
    }
    double a = (double)k1.s - (double)k1.c, b = (double)k2.s - (double)k2.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kIbThreads / 32; ++w) {
            ta += red[0][w];
            tb += red[1][w];
        }
        partials[blockIdx.x] = make_double2(ta, tb);
    }
}

template <class P>
fdas_status launch_ib(Plan &p, const void *F, void *plane, double2 *partials, cudaStream_t s) {
    const int64_t n_groups = (int64_t)p.n_z * p.n_r / 4;
    interbin_kernel<P><<<interbin_ctas(p), kIbThreads, 0, s>>>(
        (const typename P::cpx *)F, (typename P::real *)plane, partials, p.n_r, n_groups);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

}  // namespace

int interbin_ctas(const Plan &p) {
    const int64_t groups = (int64_t)p.n_z * p.n_r / 4;
    const int64_t need = (groups + kIbThreads - 1) / kIbThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)kIbCtasPerSm * p.n_sms, need));
}

fdas_status launch_interbin(Plan &p, const void *F, void *plane, double2 *partials,
                            cudaStream_t s) {
    if (p.n_r % 128 != 0) {
        set_error("interbinning needs rows of a multiple of 128 bins");
        return FDAS_ERR_UNSUPPORTED;
    }
    switch (p.prec) {
        case FDAS_FP32: return launch_ib<PrecF32>(p, F, plane, partials, s);
        case FDAS_BF16: return launch_ib<PrecBF16>(p, F, plane, partials, s);
        default: return launch_ib<PrecF16>(p, F, plane, partials, s);
    }
}

}  // namespace fdas
