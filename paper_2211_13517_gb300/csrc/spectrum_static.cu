// Allocation-free spectrum entry point: fdas_spectrum_static.
//
// It runs the same kernels as fdas_spectrum (R2C FFT and median
// normalisation) but takes no plan and allocates nothing.  The FFT
// intermediates, which fdas_spectrum keeps in plan workspace, live here in a
// fixed array in device memory that the library itself defines:
// kStaticMaxSamples FP32 complex values (8 MiB) plus a flag word.  Every
// device that loads the library reserves that array until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host it only
// names a host-side stand-in.  The device address is taken once per device,
// on the first call made on that device, with cudaGetSymbolAddress, and
// cached.
#include "fdas_internal.cuh"

#include <mutex>

namespace fdas {
namespace {

constexpr int64_t kStaticMaxSamples = int64_t(1) << 20;
constexpr int kMaxDevices = 64;

// [0, N/2): first FFT intermediate, [N/2, N): second, then the flag word
static __device__ __align__(256) float2 g_spectrum_scratch[kStaticMaxSamples + 32];

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// device address of g_spectrum_scratch on the current device (set up once)
fdas_status static_scratch(void **out) {
    int dev = 0;
    FDAS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fdas_spectrum_static: device index out of range");
        return FDAS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        FDAS_CUDA_TRY(cudaGetSymbolAddress(&p, g_spectrum_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FDAS_OK;
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace fdas

using namespace fdas;

extern "C" fdas_status fdas_spectrum_static(const float *series, int64_t n_samples,
                                            int32_t precision, int32_t norm_mode,
                                            int32_t norm_block, void *spectrum_out,
                                            float *medians_out, void *stream) {
    if (!series || !spectrum_out) {
        set_error("fdas_spectrum_static: NULL series or spectrum_out");
        return FDAS_ERR_ARG;
    }
    if (!pow2(n_samples) || n_samples < (1 << 10) || n_samples > kStaticMaxSamples) {
        set_error("fdas_spectrum_static: n_samples must be a power of two in [2^10, 2^20] "
                  "(its fixed scratch holds at most 2^20 samples); got " +
                  std::to_string(n_samples));
        return FDAS_ERR_ARG;
    }
    if (precision != FDAS_FP32 && precision != FDAS_BF16 && precision != FDAS_FP16) {
        set_error("fdas_spectrum_static: unknown precision");
        return FDAS_ERR_ARG;
    }
    if (norm_mode != FDAS_NORM_MEDIAN && norm_mode != FDAS_NORM_NONE) {
        set_error("fdas_spectrum_static: unknown norm_mode");
        return FDAS_ERR_ARG;
    }
    if (!pow2(norm_block) || norm_block < 16 || norm_block > 8192) {
        set_error("fdas_spectrum_static: norm_block must be a power of two in [16, 8192]");
        return FDAS_ERR_ARG;
    }
    if (((uintptr_t)series & 15u) != 0) {
        set_error("fdas_spectrum_static: series is not 16-byte aligned");
        return FDAS_ERR_ARG;
    }
    void *scratch = nullptr;
    FDAS_TRY(static_scratch(&scratch));

    // a host-side description of the geometry the spectrum kernels read;
    // its buffers point into the fixed array
    Plan p;
    p.n_samples = n_samples;
    p.n_r = n_samples / 2;
    p.prec = precision;
    p.norm_mode = norm_mode;
    p.norm_block = norm_block;
    int lm = 0;
    while ((int64_t(1) << lm) < p.n_r) ++lm;
    if (p.n_r <= 8192) {
        p.fft_m1 = 1;
        p.fft_m2 = (int)p.n_r;
    } else {
        p.fft_m1 = 1 << (lm / 2);
        p.fft_m2 = 1 << (lm - lm / 2);
    }
    float2 *base = static_cast<float2 *>(scratch);
    p.fft_a = base;
    p.fft_b = base + p.n_r;
    p.flags = reinterpret_cast<unsigned int *>(base + kStaticMaxSamples);
    cudaStream_t s = (cudaStream_t)stream;
    // the flag word keeps the previous call's value; start it at zero
    FDAS_CUDA_TRY(cudaMemsetAsync(p.flags, 0, sizeof(unsigned int), s));
    return launch_spectrum(p, series, spectrum_out, medians_out, s);
}
