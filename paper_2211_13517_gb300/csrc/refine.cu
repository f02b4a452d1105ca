// Fourier-interpolated power P(r, z), its gradients, and candidate refinement.
//
// For a continuous frequency r (bins) and drift z, with k0 = floor(r + 1/2),
// delta = r - k0 and the window e in [-m, m], m = 32 + ceil(|z|/2):
//
//   F(r, z) = sum_e X_{k0+e} conj(rho(delta - e, z)),   P = |F|^2,
//
// rho the (unnormalised) response of the accelerated sinusoid of paper §2.1.
// Writing rho as its integral and exchanging sum and integral,
//
//   F = int_0^1 conj(A(u)) Y(u) du,  A(u) = exp(2 pi i [(delta - z/2) u + z u^2/2]),
//                                     Y(u) = sum_e X_{k0+e} exp(2 pi i e u),
//
// so dF/dr = int -2 pi i u conj(A) Y du and dF/dz = int -2 pi i (u^2 - u)/2
// conj(A) Y du (the window is held fixed), and dF/dX_{k0+e} = conj(rho(delta -
// e, z)) with rho(delta - e, z) = int A(u) exp(-2 pi i e u) du.  All integrals
// use one Gauss-Legendre rule of kRefNodes nodes on [0, 1] (exact for
// polynomials of degree 1023; the integrands turn through at most
// m + |z|/2 + 1 cycles).  One CTA evaluates one point; arithmetic is FP32.
#include "fdas_internal.cuh"

#include <cmath>
#include <vector>

namespace fdas {

constexpr int kRefNodes = 512;
constexpr int kRefThreads = 128;
constexpr int kRefMaxHalf = 255;   // window half-width limit (|z| <= 446)
constexpr float kTwoPi = 6.28318530717958647692f;

namespace {

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// exp(i pi x)
__device__ __forceinline__ float2 cispi(float x) {
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, s);
}

// CTA-wide sum of three complex values (kRefThreads threads)
__device__ void reduce3(float2 &a, float2 &b, float2 &c, float2 *red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, off);
        a.y += __shfl_down_sync(0xffffffffu, a.y, off);
        b.x += __shfl_down_sync(0xffffffffu, b.x, off);
        b.y += __shfl_down_sync(0xffffffffu, b.y, off);
        c.x += __shfl_down_sync(0xffffffffu, c.x, off);
        c.y += __shfl_down_sync(0xffffffffu, c.y, off);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red[3 * w] = a;
        red[3 * w + 1] = b;
        red[3 * w + 2] = c;
    }
    __syncthreads();
    a = red[0];
    b = red[1];
    c = red[2];
    for (int i = 1; i < kRefThreads / 32; ++i) {
        a = c_add(a, red[3 * i]);
        b = c_add(b, red[3 * i + 1]);
        c = c_add(c, red[3 * i + 2]);
    }
    __syncthreads();
}

struct Window {
    int64_t k0;
    float delta;
    int m;
};

__device__ Window make_window(double r, double z) {
    Window w;
    w.k0 = (int64_t)floor(r + 0.5);
    w.delta = (float)(r - (double)w.k0);
    w.m = 32 + (int)ceil(fabs(z) / 2.0 - 1e-12);
    if (w.m > kRefMaxHalf) w.m = kRefMaxHalf;
    return w;
}

// copy X_{k0+e}, e in [-m, m], into shared memory (0 outside [0, n_r))
__device__ void load_window(const float2 *__restrict__ X, int64_t n_r, const Window &w, float2 *sx) {
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * w.m + 1; i += kRefThreads) {
        const int64_t k = w.k0 - w.m + i;
        sx[i] = (k >= 0 && k < n_r) ? X[k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// F, dF/dr, dF/dz at (delta, z) for the window in sx.  Each thread takes the
// kRefNodes / kRefThreads nodes u_i, i = tid + kRefThreads q, together: their
// phase recurrences are independent, so each window value read from shared
// memory feeds all of them and the chains overlap.
constexpr int kRefPer = kRefNodes / kRefThreads;
static_assert(kRefNodes % kRefThreads == 0, "nodes per thread");

__device__ void eval_F(const float2 *sx, const Window &w, float z, const float2 *__restrict__ nodes,
                       float2 *red, float2 &F, float2 &Fr, float2 &Fz) {
    float u[kRefPer], Y[kRefPer][2];
    float2 step[kRefPer], ph[kRefPer];
#pragma unroll
    for (int q = 0; q < kRefPer; ++q) {
        u[q] = nodes[threadIdx.x + kRefThreads * q].x;
        step[q] = cispi(2.0f * u[q]);
        Y[q][0] = Y[q][1] = 0.f;
    }
    // Y(u) = sum_e x_e exp(2 pi i e u), e = -m..m; exact phase every 32 terms
    for (int e0 = -w.m; e0 <= w.m; e0 += 32) {
#pragma unroll
        for (int q = 0; q < kRefPer; ++q) ph[q] = cispi(2.0f * (float)e0 * u[q]);
        const int e1 = min(e0 + 32, w.m + 1);
        for (int e = e0; e < e1; ++e) {
            const float2 x = sx[e + w.m];
#pragma unroll
            for (int q = 0; q < kRefPer; ++q) {
                const float2 t = c_mul(x, ph[q]);
                Y[q][0] += t.x;
                Y[q][1] += t.y;
                ph[q] = c_mul(ph[q], step[q]);
            }
        }
    }
    float2 aF = make_float2(0.f, 0.f), aR = aF, aZ = aF;
#pragma unroll
    for (int q = 0; q < kRefPer; ++q) {
        const float wt = nodes[threadIdx.x + kRefThreads * q].y;
        // conj(A(u)) = exp(-2 pi i [(delta - z/2) u + z u^2 / 2])
        const float theta = fmaf(0.5f * z * u[q], u[q], (w.delta - 0.5f * z) * u[q]);
        const float2 ca = cispi(-2.0f * theta);
        const float2 G = c_mul(ca, make_float2(Y[q][0], Y[q][1]));
        const float2 Gw = make_float2(G.x * wt, G.y * wt);
        aF = c_add(aF, Gw);
        // -2 pi i u G and -2 pi i (u^2 - u)/2 G
        const float su = kTwoPi * u[q], sz = kTwoPi * 0.5f * (u[q] * u[q] - u[q]);
        aR = c_add(aR, make_float2(su * Gw.y, -su * Gw.x));
        aZ = c_add(aZ, make_float2(sz * Gw.y, -sz * Gw.x));
    }
    reduce3(aF, aR, aZ, red);
    F = aF;
    Fr = aR;
    Fz = aZ;
}

__device__ __forceinline__ void power_and_grad(float2 F, float2 Fr, float2 Fz, float &P, float &gr,
                                               float &gz) {
    P = F.x * F.x + F.y * F.y;
    gr = 2.0f * (F.x * Fr.x + F.y * Fr.y);   // 2 Re(conj(F) dF/dr)
    gz = 2.0f * (F.x * Fz.x + F.y * Fz.y);
}

__global__ void __launch_bounds__(kRefThreads)
    fourier_power_kernel(const float2 *__restrict__ X, int64_t n_r, const double2 *__restrict__ rz,
                         int n, const float2 *__restrict__ nodes, float *__restrict__ power,
                         float2 *__restrict__ grad) {
    __shared__ float2 sx[2 * kRefMaxHalf + 1];
    __shared__ float2 red[3 * (kRefThreads / 32)];
    const int s = blockIdx.x;
    if (s >= n) return;
    const double2 p = rz[s];
    const Window w = make_window(p.x, p.y);
    load_window(X, n_r, w, sx);
    float2 F, Fr, Fz;
    eval_F(sx, w, (float)p.y, nodes, red, F, Fr, Fz);
    if (threadIdx.x == 0) {
        float P, gr, gz;
        power_and_grad(F, Fr, Fz, P, gr, gz);
        power[s] = P;
        if (grad) grad[s] = make_float2(gr, gz);
    }
}

// grad_X[k0 + e] += g * 2 F rho(delta - e, z); grad_rz = g * (dP/dr, dP/dz)
__global__ void __launch_bounds__(kRefThreads)
    fourier_power_backward_kernel(const float2 *__restrict__ X, int64_t n_r,
                                  const double2 *__restrict__ rz, int n,
                                  const float2 *__restrict__ nodes, const float *__restrict__ gP,
                                  float2 *__restrict__ grad_X, double2 *__restrict__ grad_rz) {
    __shared__ float2 sx[2 * kRefMaxHalf + 1];
    __shared__ float2 red[3 * (kRefThreads / 32)];
    __shared__ float2 aw[kRefNodes];
    const int s = blockIdx.x;
    if (s >= n) return;
    const double2 p = rz[s];
    const float z = (float)p.y;
    const Window w = make_window(p.x, p.y);
    load_window(X, n_r, w, sx);
    float2 F, Fr, Fz;
    eval_F(sx, w, z, nodes, red, F, Fr, Fz);
    const float g = gP[s];
    if (threadIdx.x == 0 && grad_rz) {
        float P, gr, gz;
        power_and_grad(F, Fr, Fz, P, gr, gz);
        grad_rz[s] = make_double2((double)g * gr, (double)g * gz);
    }
    if (!grad_X) return;
    // A(u_i) w_i for every node
    for (int i = threadIdx.x; i < kRefNodes; i += kRefThreads) {
        const float u = nodes[i].x, wt = nodes[i].y;
        const float theta = fmaf(0.5f * z * u, u, (w.delta - 0.5f * z) * u);
        const float2 a = cispi(2.0f * theta);
        aw[i] = make_float2(a.x * wt, a.y * wt);
    }
    __syncthreads();
    const float2 c = make_float2(2.0f * g * F.x, 2.0f * g * F.y);
    for (int i = threadIdx.x; i < 2 * w.m + 1; i += kRefThreads) {
        const int e = i - w.m;
        const int64_t k = w.k0 + e;
        if (k < 0 || k >= n_r) continue;
        float2 rho = make_float2(0.f, 0.f);
        for (int j = 0; j < kRefNodes; ++j)
            rho = c_add(rho, c_mul(aw[j], cispi(-2.0f * (float)e * nodes[j].x)));
        const float2 d = c_mul(c, rho);
        atomicAdd(&grad_X[k].x, d.x);
        atomicAdd(&grad_X[k].y, d.y);
    }
}

// n_steps of gradient ascent with backtracking, one CTA per seed.  Steps are
// taken in the scaled coordinates (r, z / kZScale) along the gradient; a step
// that lowers P is retried four times shorter (up to kRetries times), an
// accepted step makes the next one 1.5 times longer.
constexpr float kZScale = 4.0f;
constexpr int kRetries = 8;

__global__ void __launch_bounds__(kRefThreads)
    refine_kernel(const float2 *__restrict__ X, int64_t n_r, const fdas_seed *__restrict__ seeds,
                  int n, int n_steps, const float2 *__restrict__ nodes,
                  fdas_refined *__restrict__ out) {
    __shared__ float2 sx[2 * kRefMaxHalf + 1];
    __shared__ float2 red[3 * (kRefThreads / 32)];
    const int s = blockIdx.x;
    if (s >= n) return;
    double r = seeds[s].r, z = seeds[s].z;
    Window w = make_window(r, z);
    load_window(X, n_r, w, sx);
    float2 F, Fr, Fz;
    eval_F(sx, w, (float)z, nodes, red, F, Fr, Fz);
    float P, gr, gz;
    power_and_grad(F, Fr, Fz, P, gr, gz);
    float len = 0.25f;
    int accepted = 0;
    for (int it = 0; it < n_steps && len > 1e-5f; ++it) {
        bool ok = false;
        for (int tr = 0; tr < kRetries && !ok; ++tr) {
            const float G = sqrtf(gr * gr + kZScale * kZScale * gz * gz);
            if (!(G > 0.f)) break;
            const double nr = r + (double)(len * gr / G);
            const double nz = z + (double)(len * kZScale * kZScale * gz / G);
            const Window nw = make_window(nr, nz);
            load_window(X, n_r, nw, sx);
            float2 nF, nFr, nFz;
            eval_F(sx, nw, (float)nz, nodes, red, nF, nFr, nFz);
            float nP, ngr, ngz;
            power_and_grad(nF, nFr, nFz, nP, ngr, ngz);
            if (nP > P) {
                r = nr;
                z = nz;
                w = nw;
                P = nP;
                gr = ngr;
                gz = ngz;
                len *= 1.5f;
                ok = true;
                ++accepted;
            } else {
                len *= 0.25f;
            }
        }
        if (!ok) break;
    }
    if (threadIdx.x == 0) {
        fdas_refined o;
        o.r = r;
        o.z = z;
        o.power = P;
        o.dpdr = gr;
        o.dpdz = gz;
        o.steps = accepted;
        o.trial_id = seeds[s].trial_id;
        out[s] = o;
    }
}

}  // namespace

// Gauss-Legendre nodes and weights on [0, 1] (Newton on the three-term
// recurrence of the Legendre polynomials, FP64 on the host)
std::vector<float2> gauss_legendre_01(int n) {
    std::vector<float2> out(n);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-15) break;
        }
        const double wgt = 2.0 / ((1.0 - x * x) * dp * dp);
        out[i] = make_float2((float)(0.5 * (1.0 - x)), (float)(0.5 * wgt));
    }
    return out;
}

int refine_nodes() { return kRefNodes; }

fdas_status launch_fourier_power(Plan &p, const float2 *X, const double2 *rz, int n, float *power,
                                 float2 *grad, cudaStream_t s) {
    if (n <= 0) return FDAS_OK;
    fourier_power_kernel<<<n, kRefThreads, 0, s>>>(X, p.n_r, rz, n, p.gl_nodes, power, grad);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

fdas_status launch_fourier_power_backward(Plan &p, const float2 *X, const double2 *rz, int n,
                                          const float *gP, float2 *grad_X, double2 *grad_rz,
                                          cudaStream_t s) {
    if (n <= 0) return FDAS_OK;
    fourier_power_backward_kernel<<<n, kRefThreads, 0, s>>>(X, p.n_r, rz, n, p.gl_nodes, gP, grad_X,
                                                            grad_rz);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

fdas_status launch_refine(Plan &p, const float2 *X, const fdas_seed *seeds, int n, int n_steps,
                          fdas_refined *out, cudaStream_t s) {
    if (n <= 0) return FDAS_OK;
    refine_kernel<<<n, kRefThreads, 0, s>>>(X, p.n_r, seeds, n, n_steps, p.gl_nodes, out);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

}  // namespace fdas
