// Template bank (plan time, FP64 on the GPU).
//
// The matched filter of paper §2.1 correlates the spectrum with the response
// of a sinusoid whose frequency drifts linearly by z bins over the
// observation.  Its response at offset q from the mid-observation frequency is
//
//     rho(q, z) = int_0^1 exp(2 pi i [(q - z/2) u + z u^2 / 2]) du .
//
// For z > 0, with a = z/2 and b = q - a, completing the square turns the
// phase into a Fresnel argument:
//
//     rho = exp(-i pi b^2 / z) / (2 sqrt(a)) * [E(t1) - E(t0)],
//     t0 = b / sqrt(a),  t1 = (q + a) / sqrt(a),
//     E(t) = int_0^t exp(i pi s^2 / 2) ds = C(t) + i S(t),
//
// and rho(q, -z) = conj(rho(-q, z)); rho(e, 0) = 1 if e = 0 else 0 at integer
// e.  E(t) is evaluated (Abramowitz & Stegun 7.3.22 and 7.1.14) by its power
// series sum_n (i pi/2)^n t^(2n+1) / (n! (2n+1)) for |t| <= 2 and otherwise as
// E(t) = (1+i)/2 [1 - erfc(w)], w = sqrt(pi)(1-i)|t|/2, with erfc from its
// Laplace continued fraction evaluated backwards from a fixed depth; when both
// ends of the interval are beyond 2 on the same side the two erfc terms are
// subtracted directly, so nothing cancels.
//
// The taps are g_z[e] = conj(rho(e, z)) / sqrt(E_z), |e| <= m(z), E_z =
// sum_e |rho(e, z)|^2 (unit energy, so noise cells stay Exp(1)); the bank entry
// is the seg_len-point DFT of g_z placed circularly, divided by seg_len.
#include "fdas_internal.cuh"

namespace fdas {
namespace {

struct cd {
    double x, y;
};
__device__ __forceinline__ cd mk(double x, double y) { return {x, y}; }
__device__ __forceinline__ cd add(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd sub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd mul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd scl(cd a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ cd dvd(cd a, cd b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return {(a.x + a.y * r) / d, (a.y - a.x * r) / d};
    }
    double r = b.x / b.y, d = b.y + b.x * r;
    return {(a.x * r + a.y) / d, (a.y * r - a.x) / d};
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;

// erfc(w) for w = sqrt(pi)(1 - i) a / 2, a > 2 (continued fraction, A&S 7.1.14)
__device__ cd erfc_diag(double a) {
    const double c = 0.5 * kSqrtPi * a;
    const cd w = mk(c, -c);
    cd f = w;
    for (int k = 80; k >= 1; --k) f = add(w, dvd(mk(0.5 * k, 0.0), f));
    // exp(-w^2) = exp(i pi a^2 / 2)
    double s, co;
    sincospi(0.5 * a * a, &s, &co);
    return dvd(mk(co, s), scl(f, kSqrtPi));
}

// E(t) for |t| <= 2 (power series)
__device__ cd fresnel_series(double t) {
    cd term = mk(t, 0.0), sum = term;
    const cd q = mk(0.0, 0.5 * kPi * t * t);
    for (int n = 1; n < 60; ++n) {
        term = scl(mul(term, q), 1.0 / n);
        cd add_t = scl(term, 1.0 / (2 * n + 1));
        sum = add(sum, add_t);
        if (n > 3 && fabs(term.x) + fabs(term.y) < 1e-18 * (fabs(sum.x) + fabs(sum.y))) break;
    }
    return sum;
}

// E(t) for any t
__device__ cd fresnel_E(double t) {
    const double a = fabs(t);
    cd r;
    if (a <= 2.0) {
        r = fresnel_series(a);
    } else {
        cd e = erfc_diag(a);
        // (1+i)/2 (1 - e)
        cd one_m = mk(1.0 - e.x, -e.y);
        r = mul(mk(0.5, 0.5), one_m);
    }
    return t < 0 ? mk(-r.x, -r.y) : r;
}

// E(t1) - E(t0)
__device__ cd fresnel_diff(double t0, double t1) {
    if (t0 > 2.0 && t1 > 2.0) {
        cd d = sub(erfc_diag(t0), erfc_diag(t1));
        return mul(mk(0.5, 0.5), d);
    }
    if (t0 < -2.0 && t1 < -2.0) {
        cd d = sub(erfc_diag(-t1), erfc_diag(-t0));
        return mul(mk(0.5, 0.5), d);
    }
    return sub(fresnel_E(t1), fresnel_E(t0));
}

// rho(q, z) for z > 0
__device__ cd rho_pos(double q, double z) {
    const double a = 0.5 * z, sa = sqrt(a), b = q - a;
    cd d = fresnel_diff(b / sa, (q + a) / sa);
    double s, c;
    sincospi(-b * b / z, &s, &c);
    return scl(mul(mk(c, s), d), 0.5 / sa);
}

__device__ cd rho(double q, double z) {
    if (z == 0.0) return mk(q == 0.0 ? 1.0 : 0.0, 0.0);   // integer q only
    if (z < 0.0) {
        cd r = rho_pos(-q, -z);
        return mk(r.x, -r.y);
    }
    return rho_pos(q, z);
}

// one thread per tap: raw rho(e, z) into taps (complex double, interleaved)
__global__ void rho_kernel(double *taps, const int64_t *off, const int32_t *m, int n_z,
                           double z_step, int K) {
    const int iz = blockIdx.y;
    if (iz >= n_z) return;
    const int mz = m[iz];
    const int e = (int)(blockIdx.x * blockDim.x + threadIdx.x) - mz;
    if (e > mz) return;
    const double z = (double)(iz - K) * z_step;
    cd r = rho((double)e, z);
    const int64_t i = off[iz] + (e + mz);
    taps[2 * i] = r.x;
    taps[2 * i + 1] = r.y;
}

// one block per template: E_z (fixed order) and taps <- conj(rho)/sqrt(E_z)
__global__ void normalise_taps_kernel(double *taps, double *energy, const int64_t *off,
                                      const int32_t *m) {
    const int iz = blockIdx.x;
    const int n = 2 * m[iz] + 1;
    double *t = taps + 2 * off[iz];
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double E = 0.0;
        for (int i = 0; i < n; ++i) E += t[2 * i] * t[2 * i] + t[2 * i + 1] * t[2 * i + 1];
        energy[iz] = E;
        inv = 1.0 / sqrt(E);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        t[2 * i] *= inv;
        t[2 * i + 1] *= -inv;
    }
}

// exp(-2 pi i k / L) table, FP64
__global__ void dft_table_kernel(double2 *tab, int L) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    tab[k] = make_double2(c, s);
}

// bank[iz][f] = scale/L * sum_e g_z[e] exp(-2 pi i f e / L)
template <class P>
__global__ void bank_kernel(typename P::cpx *bank, const double *taps, const int64_t *off,
                            const int32_t *m, const double2 *tab, int L, double scale) {
    const int iz = blockIdx.y;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= L) return;
    const int mz = m[iz];
    const double *t = taps + 2 * off[iz];
    double ar = 0.0, ai = 0.0;
    for (int e = -mz; e <= mz; ++e) {
        const int k = (int)((((int64_t)f * e) % L + L) % L);
        const double2 w = tab[k];
        const double gr = t[2 * (e + mz)], gi = t[2 * (e + mz) + 1];
        ar += gr * w.x - gi * w.y;
        ai += gr * w.y + gi * w.x;
    }
    const double s = scale / (double)L;
    bank[(int64_t)iz * L + f] = P::st(make_float2((float)(ar * s), (float)(ai * s)));
}

}  // namespace

fdas_status launch_template_bank(Plan &p, cudaStream_t s) {
    int max_taps = 2 * p.m_max + 1;
    dim3 g1((max_taps + 127) / 128, p.n_z);
    rho_kernel<<<g1, 128, 0, s>>>(p.taps, p.tap_off, p.tap_m, p.n_z, p.z_step, p.iz0);
    FDAS_CUDA_TRY(cudaGetLastError());
    normalise_taps_kernel<<<p.n_z, 128, 0, s>>>(p.taps, p.energy, p.tap_off, p.tap_m);
    FDAS_CUDA_TRY(cudaGetLastError());
    double2 *tab = nullptr;
    FDAS_CUDA_TRY(cudaMallocAsync((void **)&tab, sizeof(double2) * p.L, s));
    dft_table_kernel<<<(p.L + 255) / 256, 256, 0, s>>>(tab, p.L);
    dim3 g2((p.L + 127) / 128, p.n_z);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        switch (p.prec) {
            case FDAS_FP32:
                bank_kernel<PrecF32><<<g2, 128, 0, s>>>((float2 *)p.bank, p.taps, p.tap_off,
                                                        p.tap_m, tab, p.L, 1.0);
                break;
            case FDAS_BF16:
                bank_kernel<PrecBF16><<<g2, 128, 0, s>>>((__nv_bfloat162 *)p.bank, p.taps,
                                                         p.tap_off, p.tap_m, tab, p.L, 1.0);
                break;
            default:  // FP16 holds L times the bank (range)
                bank_kernel<PrecF16><<<g2, 128, 0, s>>>((__half2 *)p.bank, p.taps, p.tap_off,
                                                        p.tap_m, tab, p.L, (double)p.L);
                break;
        }
        e = cudaGetLastError();
    }
    cudaFreeAsync(tab, s);
    FDAS_CUDA_TRY(e);
    return FDAS_OK;
}

}  // namespace fdas
