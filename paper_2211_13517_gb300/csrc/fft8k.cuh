// 8192-point FFT with 256 threads x 32 points (passes 16 x 16 x 32).
//
// Same Stockham decomposition as fft_cta.cuh (pass k reads the inputs
// j + r L/R of butterfly j, multiplies input r by W_{Ns R}^{r (j mod Ns)},
// does an R-point DFT and writes output r to (j/Ns) Ns R + (j mod Ns) + r Ns),
// but every thread owns 32 points: two radix-16 butterflies (j = t, t + 256)
// in the first two passes and one radix-32 butterfly (j = t) in the last, so a
// transform needs two shared-memory exchanges instead of three.  Both
// radix-16 butterflies of a thread share j mod 16, hence their twiddles.
#pragma once

#include "fft_cta.cuh"

namespace fdas {

// 32 = 2 x 16: Y[a][c] = DFT16 over b of x[a + 2b]; X[c + 16d] = Y[0][c] +
// (-1)^d W32^c Y[1][c]
template <int D>
struct Dft<32, D> {
    __device__ __forceinline__ static void run(float2 *v) {
        float2 e[16], o[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            e[b] = v[2 * b];
            o[b] = v[2 * b + 1];
        }
        Dft<16, D>::run(e);
        Dft<16, D>::run(o);
        constexpr float C32[32] = {
            1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
            0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
            0.19509032201612826785f, 0.0f, -0.19509032201612826785f, -0.38268343236508977173f,
            -0.55557023301960222474f, -0.70710678118654752440f, -0.83146961230254523708f,
            -0.92387953251128675613f, -0.98078528040323044913f, -1.0f, -0.98078528040323044913f,
            -0.92387953251128675613f, -0.83146961230254523708f, -0.70710678118654752440f,
            -0.55557023301960222474f, -0.38268343236508977173f, -0.19509032201612826785f, 0.0f,
            0.19509032201612826785f, 0.38268343236508977173f, 0.55557023301960222474f,
            0.70710678118654752440f, 0.83146961230254523708f, 0.92387953251128675613f,
            0.98078528040323044913f};
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            // W32^c; sin(2 pi c/32) = cos(2 pi (c - 8)/32)
            const float2 t = c == 0 ? o[0] : cmul(o[c], make_float2(C32[c], D * C32[(c + 24) & 31]));
            v[c] = cadd(e[c], t);
            v[c + 16] = csub(e[c], t);
        }
    }
};

template <int D>
struct Fft8k {
    static constexpr int L = 8192;
    static constexpr int T = 256;
    static constexpr int SMEM_ELEMS = L + L / 16;

    // base twiddles of this thread: pass 1 W_256^{t mod 16}, pass 2 W_8192^t
    __device__ __forceinline__ static void make_twiddles(int t, float2 &w1, float2 &w2) {
        w1 = twiddle<D>(t & 15, 256);
        w2 = twiddle<D>(t, 8192);
    }

    // pass 0: v[16 b + r] is input (t + 256 b) + 512 r; writes smem
    __device__ __forceinline__ static void pass0(float2 *v, float2 *buf, int t) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            Dft<16, D>::run(v + 16 * b);
            float2 *dst = buf + 17 * (t + 256 * b);   // fft_pad(16 j + r) = 17 j + r
#pragma unroll
            for (int r = 0; r < 16; ++r) dst[r] = v[16 * b + r];
        }
    }

    // pass 1 (Ns = 16, R = 16), in place
    __device__ __forceinline__ static void pass1(float2 *buf, int t, float2 w1) {
        float2 v[32];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const float2 *src = buf + fft_pad(t + 256 * b);   // + 544 r = fft_pad(j + 512 r)
#pragma unroll
            for (int r = 0; r < 16; ++r) v[16 * b + r] = src[544 * r];
        }
        __syncthreads();
        float2 p[16];
        p[1] = w1;
#pragma unroll
        for (int r = 2; r < 16; ++r) p[r] = cmul(p[r / 2], p[r - r / 2]);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int r = 1; r < 16; ++r) v[16 * b + r] = cmul(v[16 * b + r], p[r]);
            Dft<16, D>::run(v + 16 * b);
            const int j = t + 256 * b;
            float2 *dst = buf + fft_pad((j >> 4) * 256 + (j & 15));   // + 17 r
#pragma unroll
            for (int r = 0; r < 16; ++r) dst[17 * r] = v[16 * b + r];
        }
        __syncthreads();
    }

    // pass 2 (Ns = 256, R = 32) into registers: out[r] is element t + 256 r
    __device__ __forceinline__ static void pass2(const float2 *buf, int t, float2 w2, float2 *out) {
        const float2 *src = buf + fft_pad(t);   // + 272 r = fft_pad(t + 256 r)
#pragma unroll
        for (int r = 0; r < 32; ++r) out[r] = src[272 * r];
        apply_twiddles<32>(out, w2);
        Dft<32, D>::run(out);
    }
};

}  // namespace fdas
