// CTA-wide power-of-two complex FFT in registers + shared memory (FP32).
//
// One CTA of T = L/16 threads transforms L points.  The transform is a
// Stockham autosort decomposition L = 16 * 16 * ... * REM: pass k takes
// butterflies j = 0..L/R-1, reads the R inputs j + r L/R, multiplies input r
// by W_{Ns R}^{r (j mod Ns)} (Ns = product of the earlier radices), does an
// R-point DFT in registers and writes output r to (j/Ns) Ns R + (j mod Ns) +
// r Ns.  The last pass therefore leaves the natural order.  Every thread owns
// 16 inputs per pass (16/R butterflies).
//
// Shared memory holds one padded L-point buffer (one spare slot per 16, so
// that the stride-16 writes of the first pass do not collide in banks); each
// pass reads all of its inputs, synchronises and then writes in place.
//
// Direction D = -1 is the forward transform exp(-2 pi i k n / L), D = +1 the
// unnormalised inverse.
#pragma once

#include <cuda_runtime.h>

namespace fdas {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (D i)
template <int D>
__device__ __forceinline__ float2 mul_di(float2 a) {
    return D > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr int ipow16(int k) { return k == 0 ? 1 : 16 * ipow16(k - 1); }

__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }

// exp(D * 2 pi i * num / den) for integers, den a power of two
template <int D>
__device__ __forceinline__ float2 twiddle(int num, int den) {
    float s, c;
    sincospif(2.0f * (float)num / (float)den, &s, &c);
    return make_float2(c, D > 0 ? s : -s);
}

// W_16^b = exp(D 2 pi i b / 16); b is a compile-time constant after unrolling
template <int D>
__device__ __forceinline__ float2 w16(int b) {
    constexpr float C[16] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f,
                             0.38268343236508977173f, 0.0f, -0.38268343236508977173f,
                             -0.70710678118654752440f, -0.92387953251128675613f, -1.0f,
                             -0.92387953251128675613f, -0.70710678118654752440f,
                             -0.38268343236508977173f, 0.0f, 0.38268343236508977173f,
                             0.70710678118654752440f, 0.92387953251128675613f};
    return make_float2(C[b & 15], D * C[(b + 12) & 15]);   // sin(x) = cos(x - pi/2)
}

// ---- small DFTs in registers (natural order in and out) -------------------
template <int D>
__device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3) {
    float2 a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_di<D>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

template <int R, int D>
struct Dft;

template <int D>
struct Dft<2, D> {
    __device__ __forceinline__ static void run(float2 *v) {
        float2 t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    }
};

template <int D>
struct Dft<4, D> {
    __device__ __forceinline__ static void run(float2 *v) { dft4<D>(v[0], v[1], v[2], v[3]); }
};

// 8 = 2 x 4: Y[a][c] = DFT4 over b of x[a + 2b]; X[c + 4d] = sum_a W8^{ac} W2^{ad} Y[a][c]
template <int D>
struct Dft<8, D> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float h = 0.70710678118654752440f;
        dft4<D>(v[0], v[2], v[4], v[6]);
        dft4<D>(v[1], v[3], v[5], v[7]);
        // v[1 + 2c] *= W8^c
        v[3] = cmul(v[3], make_float2(h, D * h));
        v[5] = mul_di<D>(v[5]);
        v[7] = cmul(v[7], make_float2(-h, D * h));
        float2 o[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            o[c] = cadd(v[2 * c], v[2 * c + 1]);
            o[c + 4] = csub(v[2 * c], v[2 * c + 1]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = o[k];
    }
};

// 16 = 4 x 4: Y[a][c] = DFT4 over b of x[a + 4b]; times W16^{ac}; DFT4 over a
template <int D>
struct Dft<16, D> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float c1 = 0.92387953251128675613f;  // cos(pi/8)
        const float s1 = 0.38268343236508977173f;  // sin(pi/8)
        const float h = 0.70710678118654752440f;
#pragma unroll
        for (int a = 0; a < 4; ++a) dft4<D>(v[a], v[a + 4], v[a + 8], v[a + 12]);
        // v[a + 4c] *= W16^{ac}
        v[5] = cmul(v[5], make_float2(c1, D * s1));     // W^1
        v[9] = cmul(v[9], make_float2(h, D * h));       // W^2
        v[13] = cmul(v[13], make_float2(s1, D * c1));   // W^3
        v[6] = cmul(v[6], make_float2(h, D * h));       // W^2
        v[10] = mul_di<D>(v[10]);                       // W^4
        v[14] = cmul(v[14], make_float2(-h, D * h));    // W^6
        v[7] = cmul(v[7], make_float2(s1, D * c1));     // W^3
        v[11] = cmul(v[11], make_float2(-h, D * h));    // W^6
        v[15] = cmul(v[15], make_float2(-c1, -D * s1)); // W^9
#pragma unroll
        for (int c = 0; c < 4; ++c) dft4<D>(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        // now v[4c + d] = X[c + 4d]
        float2 o[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) o[k] = v[4 * (k & 3) + (k >> 2)];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = o[k];
    }
};

// v[r] *= w^r, r = 1..R-1 (powers by a balanced product tree)
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 *v, float2 w) {
    float2 p[R];
    p[1] = w;
#pragma unroll
    for (int r = 2; r < R; ++r) p[r] = cmul(p[r / 2], p[r - r / 2]);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], p[r]);
}

// ---------------------------------------------------------------------------
template <int L, int D>
struct CtaFft {
    static constexpr int T = L / 16;                  // threads
    static constexpr int LOG = ilog2c(L);
    static constexpr int NP16 = LOG / 4;
    static constexpr int REM = 1 << (LOG % 4);
    static constexpr int NPASS = NP16 + (REM > 1 ? 1 : 0);
    static constexpr int SMEM_ELEMS = L + L / 16;     // padded buffer
    static_assert(L >= 128 && (L & (L - 1)) == 0, "L must be a power of two >= 128");

    template <int K>
    struct Pass {
        static constexpr int R = K < NP16 ? 16 : REM;
        static constexpr int Ns = ipow16(K);
        static constexpr int NB = 16 / R;             // butterflies per thread
    };

    // base twiddle of pass K >= 1 for this thread's first butterfly
    template <int K>
    __device__ __forceinline__ static float2 base_twiddle(int tid) {
        constexpr int R = Pass<K>::R, Ns = Pass<K>::Ns;
        return twiddle<D>(tid % Ns, Ns * R);
    }

    // first pass (K = 0, radix 16, no twiddles): inputs already in v, the
    // 16 values at positions tid + r L/16; writes the outputs to smem.
    __device__ __forceinline__ static void first_pass(float2 *v, float2 *buf, int tid) {
        Dft<16, D>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[fft_pad(tid * 16 + r)] = v[r];
        __syncthreads();
    }

    // one in-place smem pass K (1 <= K < NPASS) with base twiddle w
    template <int K>
    __device__ __forceinline__ static void smem_pass(float2 *buf, int tid, float2 w) {
        constexpr int R = Pass<K>::R, Ns = Pass<K>::Ns, NB = Pass<K>::NB;
        float2 v[16];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = tid + b * T;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = buf[fft_pad(j + r * (L / R))];
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = tid + b * T;
            // twiddle base for butterfly b: W_{Ns R}^{j mod Ns}
            float2 wb = w;
            if (NB > 1) wb = twiddle_shift<K>(w, b);
            apply_twiddles<R>(v + b * R, wb);
            Dft<R, D>::run(v + b * R);
            const int jm = j % Ns;
            const int idxD = (j / Ns) * Ns * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[fft_pad(idxD + r * Ns)] = v[b * R + r];
        }
        __syncthreads();
    }

    // last pass into registers: out[b*R + r] is output element
    // n = tid + b*T + r*Ns (natural order index), b < NB.
    __device__ __forceinline__ static void last_pass_regs(const float2 *buf, int tid, float2 w,
                                                          float2 *out) {
        constexpr int K = NPASS - 1;
        constexpr int R = Pass<K>::R, NB = Pass<K>::NB;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = tid + b * T;
#pragma unroll
            for (int r = 0; r < R; ++r) out[b * R + r] = buf[fft_pad(j + r * (L / R))];
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float2 wb = w;
            if (NB > 1) wb = twiddle_shift<K>(w, b);
            apply_twiddles<R>(out + b * R, wb);
            Dft<R, D>::run(out + b * R);
        }
    }
    __device__ __forceinline__ static int last_index(int tid, int b, int r) {
        constexpr int K = NPASS - 1;
        return tid + b * T + r * Pass<K>::Ns;
    }

    // For passes with several butterflies per thread the j's differ by b*T
    // and (j mod Ns) = j (these only occur in the last pass, where j < Ns),
    // so W_{Ns R}^{j + bT} = w * W_{Ns R}^{bT} = w * W_16^{b} since Ns R = L.
    template <int K>
    __device__ __forceinline__ static float2 twiddle_shift(float2 w, int b) {
        return cmul(w, w16<D>(b));
    }

    // all middle passes 1..NPASS-2
    template <int K>
    __device__ __forceinline__ static void middle(float2 *buf, int tid, const float2 *tw) {
        if constexpr (K < NPASS - 1) {
            smem_pass<K>(buf, tid, tw[K]);
            middle<K + 1>(buf, tid, tw);
        }
    }

    // twiddle table for this thread: tw[K] for K = 1..NPASS-1 (tw[0] unused)
    __device__ __forceinline__ static void make_twiddles(int tid, float2 *tw) {
        tw[0] = make_float2(1.f, 0.f);
        fill_tw<1>(tid, tw);
    }
    template <int K>
    __device__ __forceinline__ static void fill_tw(int tid, float2 *tw) {
        if constexpr (K < NPASS) {
            tw[K] = base_twiddle<K>(tid);
            fill_tw<K + 1>(tid, tw);
        }
    }

    // full transform: v (first-pass inputs) -> natural-order result in buf.
    __device__ __forceinline__ static void to_smem(float2 *v, float2 *buf, int tid, const float2 *tw) {
        first_pass(v, buf, tid);
        middle<1>(buf, tid, tw);
        // last pass in place
        float2 o[16];
        last_pass_regs(buf, tid, tw[NPASS - 1], o);
        __syncthreads();
        constexpr int K = NPASS - 1;
        constexpr int R = Pass<K>::R, NB = Pass<K>::NB;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) buf[fft_pad(last_index(tid, b, r))] = o[b * R + r];
        __syncthreads();
    }

    // full transform: v -> registers out (natural index via last_index)
    __device__ __forceinline__ static void to_regs(float2 *v, float2 *buf, int tid, const float2 *tw,
                                                   float2 *out) {
        first_pass(v, buf, tid);
        middle<1>(buf, tid, tw);
        last_pass_regs(buf, tid, tw[NPASS - 1], out);
    }
};

}  // namespace fdas
