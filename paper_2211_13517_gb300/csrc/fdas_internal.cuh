// Internal declarations of the FDAS CUDA library (sm_103a).
//
// Shared by the .cu files of the library only.  Nothing here is part of the
// C ABI (include/fdas.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/fdas.h"

namespace fdas {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
fdas_status cuda_status(cudaError_t e, const char *what);

#define FDAS_CUDA_TRY(expr)                                                   \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) return ::fdas::cuda_status(_e, #expr);         \
    } while (0)

#define FDAS_TRY(expr)                                                        \
    do {                                                                      \
        fdas_status _s = (expr);                                              \
        if (_s != FDAS_OK) return _s;                                         \
    } while (0)

// ---------------------------------------------------------------------------
// storage precisions: spectra/templates are complex pairs, planes scalars.
// All arithmetic is FP32; conversion happens on load and store.
// ---------------------------------------------------------------------------
struct PrecF32 {
    using cpx = float2;
    using real = float;
    static constexpr int id = FDAS_FP32;
    static constexpr float plane_scale = 1.0f;       // stored = P * scale
    __device__ __forceinline__ static float2 ld(const cpx &v) { return v; }
    __device__ __forceinline__ static cpx st(float2 v) { return v; }
    __device__ __forceinline__ static float ldr(real v) { return v; }
    __device__ __forceinline__ static real str(float v) { return v; }
};

struct PrecBF16 {
    using cpx = __nv_bfloat162;
    using real = __nv_bfloat16;
    static constexpr int id = FDAS_BF16;
    static constexpr float plane_scale = 1.0f;
    __device__ __forceinline__ static float2 ld(const cpx &v) { return __bfloat1622float2(v); }
    __device__ __forceinline__ static cpx st(float2 v) { return __float22bfloat162_rn(v); }
    __device__ __forceinline__ static float ldr(real v) { return __bfloat162float(v); }
    __device__ __forceinline__ static real str(float v) { return __float2bfloat16_rn(v); }
    // s + (value stored in the low / high half of w, or in h), one FP32
    // rounding: the mixed-precision add converts the 16-bit operand exactly
    __device__ __forceinline__ static float acc_lo(float s, uint32_t w) {
        float d;
        asm("{\n .reg .b16 l, u;\n mov.b32 {l, u}, %1;\n add.rn.f32.bf16 %0, l, %2;\n}\n"
            : "=f"(d) : "r"(w), "f"(s));
        return d;
    }
    __device__ __forceinline__ static float acc_hi(float s, uint32_t w) {
        float d;
        asm("{\n .reg .b16 l, u;\n mov.b32 {l, u}, %1;\n add.rn.f32.bf16 %0, u, %2;\n}\n"
            : "=f"(d) : "r"(w), "f"(s));
        return d;
    }
    __device__ __forceinline__ static float acc16(float s, unsigned short h) {
        float d;
        asm("add.rn.f32.bf16 %0, %1, %2;\n" : "=f"(d) : "h"(h), "f"(s));
        return d;
    }
};

struct PrecF16 {
    using cpx = __half2;
    using real = __half;
    static constexpr int id = FDAS_FP16;
    static constexpr float plane_scale = 0.0625f;    // P/16 keeps P < 1e6 in range
    __device__ __forceinline__ static float2 ld(const cpx &v) { return __half22float2(v); }
    __device__ __forceinline__ static cpx st(float2 v) { return __float22half2_rn(v); }
    __device__ __forceinline__ static float ldr(real v) { return __half2float(v); }
    __device__ __forceinline__ static real str(float v) { return __float2half_rn(v); }
    __device__ __forceinline__ static float acc_lo(float s, uint32_t w) {
        float d;
        asm("{\n .reg .b16 l, u;\n mov.b32 {l, u}, %1;\n add.rn.f32.f16 %0, l, %2;\n}\n"
            : "=f"(d) : "r"(w), "f"(s));
        return d;
    }
    __device__ __forceinline__ static float acc_hi(float s, uint32_t w) {
        float d;
        asm("{\n .reg .b16 l, u;\n mov.b32 {l, u}, %1;\n add.rn.f32.f16 %0, u, %2;\n}\n"
            : "=f"(d) : "r"(w), "f"(s));
        return d;
    }
    __device__ __forceinline__ static float acc16(float s, unsigned short h) {
        float d;
        asm("add.rn.f32.f16 %0, %1, %2;\n" : "=f"(d) : "h"(h), "f"(s));
        return d;
    }
};

inline size_t cpx_bytes(int prec) { return prec == FDAS_FP32 ? 8 : 4; }
inline size_t real_bytes(int prec) { return prec == FDAS_FP32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// candidate records kept on the device during a search
// key bits: [0,23) ir, [23,39) iz, [39,42) stage, [42,64) batch rank
// ---------------------------------------------------------------------------
struct CandRec {
    unsigned long long key;
    float power;
    float pad;
};

__host__ __device__ inline unsigned long long cand_key(uint32_t rank, int stage, int iz,
                                                       uint32_t ir) {
    return ((unsigned long long)rank << 42) | ((unsigned long long)stage << 39) |
           ((unsigned long long)iz << 23) | (unsigned long long)ir;
}

// outcome of a stream-ordered search, computed on the device: the status
// and counts the blocking search derives on the host
struct AsyncResult {
    int64_t n_found;   // true number of crossings (0 on a non-finite or timeout error)
    int64_t n_sort;    // records to order (0 when none are reported)
    int64_t n_out;     // records written to the caller: min(n_sort, capacity)
    int32_t status;    // fdas_status
    int32_t pad;
};

// per-trial statistics and thresholds written on the device
struct TrialStats {
    double mean, std;
    float thr[8];   // T_h per stage (FP32, compared against FP32 sums)
};

// one chunk of templates of the tensor-core correlation: its templates, the
// K range it reads of each spectrum window and where its operand image lives
struct TcChunk {
    // the chunk's 28 column groups in two halves of 14, one per half of the
    // epilogue warps: half h holds templates z_part[h] .. z_part[h] +
    // n_part[h] - 1 (the rest of its columns are 0)
    int32_t z_part[2];
    int32_t n_part[2];
    int32_t kofs;      // first complex element of the window it reads (multiple of 4)
    int32_t ks;        // K steps of 8 complex taps (16 real elements)
    int64_t b_off;     // byte offset of the chunk's template image in tc_bank
};

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct Plan {
    // geometry
    int64_t n_samples, n_r;
    int n_z, iz0, m_max, m_ov, L, V, n_seg, H, n_stages;
    int prec, norm_mode, norm_block, thr_mode;
    double tsamp, z_max, z_step, sigma;
    double G[6];
    int64_t max_cands;
    int64_t store_cap = 0;  // records the kernels may store this call (max_cands)
    int64_t n_allocs = 0;   // device allocations made for the plan so far
    int device;
    int n_zchunk;           // z chunks per segment in the correlation grid
    int n_sms = 1;          // streaming multiprocessors of the device
    int64_t partials_cap = 0;   // double2 entries of each partials buffer
    bool use_graph = false;
    cudaGraphExec_t graph_exec = nullptr;   // last captured batch
    double tuned_ms = 0.0;
    int correlator = FDAS_CORR_FFT;   // FDAS_CORR_FFT or FDAS_CORR_TENSOR
    int harm_mode = FDAS_HARM_TOP;    // FDAS_HARM_TOP or FDAS_HARM_FUNDAMENTAL
    bool interbin = false;            // plane on the half-bin grid (2 n_r columns)
    // tensor-core correlation: template chunks, their operand images and the
    // spectrum window each GEMM tile reads (complex elements)
    TcChunk *tc_chunks = nullptr;
    void *tc_bank = nullptr;
    float *tc_inv_energy = nullptr;   // [n_z] 1 / energy of the 16-bit taps
    float4 *tc_edges = nullptr;       // interbinning: [n_z][n_r / 512][4] first/last F
    // FP32 plans on the tensor cores (FDAS_CORR_TENSOR_SPLIT): operands as
    // BF16 hi + lo parts; the lo template image sits tc_bank_lo bytes after
    // the hi one, the spectrum parts in spec_hi / spec_lo (padded like spec_pad)
    bool tc_split = false;
    int64_t tc_bank_lo = 0;
    int64_t tc_img_bytes = 0;         // bytes of tc_bank (both parts in split mode)
    void *spec_hi = nullptr, *spec_lo = nullptr;
    int64_t tc_split_elems = 0;
    int tc_n_ch = 0, tc_max_ks = 0, tc_win = 0;
    int tc_nbuf = 1;                  // template-image buffers in shared memory (1 or 2)
    // template order of the chunks: 0 = consecutive z, 28 per chunk; 1 =
    // pairs of +-|z| (one half of each chunk z <= 0, the other z > 0), so
    // that a chunk's templates have similar widths
    int tc_order = 1;
    // FFT split of the N/2-point complex FFT in the spectrum stage
    int fft_m1, fft_m2;     // M = m1 * m2 (m1 = 1: single pass)
    // device memory
    void *bank = nullptr;           // [n_z][L] cpx (plan precision)
    double *taps = nullptr;         // FP64 taps, concatenated (re, im)
    double *energy = nullptr;       // [n_z]
    int64_t *tap_off = nullptr;     // [n_z] offsets (complex units)
    int32_t *tap_m = nullptr;       // [n_z]
    int64_t n_taps = 0;
    float2 *fft_a = nullptr, *fft_b = nullptr;   // [M] scratch each
    void *spec_pad = nullptr;       // [n_seg*V + 2 m_ov] cpx, zero-padded
    int64_t spec_pad_elems = 0;     // complex elements of spec_pad (and of spec_hi / spec_lo)
    void *plane[2] = {nullptr, nullptr};   // [n_z][plane_cols] real
    void *corr = nullptr;           // interbinning: [n_z][n_r] complex F
    double2 *partials[2] = {nullptr, nullptr};   // per correlation CTA
    TrialStats *stats = nullptr;    // [stats_cap]
    int64_t stats_cap = 0;
    CandRec *cand = nullptr;        // [max_cands]
    unsigned long long *cand_count = nullptr;
    unsigned int *flags = nullptr;  // [0]: non-finite input seen
    uint32_t *rank_ids = nullptr;   // [stats_cap] trial id per rank
    fdas_candidate *out_stage = nullptr;   // [max_cands] ordered output
    AsyncResult *async_res = nullptr;      // status of the last stream-ordered search
    float *stage = nullptr;         // [n_samples] device copy of a host series
    float *stage2 = nullptr;        // second staging buffer (copies alternate)
    cudaStream_t cpy = nullptr;     // host-to-device copies of host series
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr;         // orders the copy stream after the caller's
    unsigned long long *host_small = nullptr;  // pinned: {count, flags}
    float2 *gl_nodes = nullptr;     // Gauss-Legendre (u, w) on [0, 1] for P(r, z)
    fdas_seed *ref_seeds = nullptr;        // device staging of refine seeds
    fdas_refined *ref_out = nullptr;       // device staging of refine results
    int64_t ref_cap = 0;
    int64_t ws_bytes = 0;
    // checked builds: each device buffer of the plan sits between two guards
    // of canary bytes (base .. base + guard, then after its `bytes`)
    struct GuardedBuf {
        char *base;
        size_t bytes;
        const char *name;
    };
    // the plan's pools, shared with its views (the copies of a Plan made
    // for one series or one stage), so that a view copies no vector
    struct Pools {
        std::vector<cudaEvent_t> events;   // timed intervals of tracing
        std::vector<GuardedBuf> guards;    // checked builds
    };
    std::shared_ptr<Pools> pools = std::make_shared<Pools>();
    bool plant_canary = false;        // FDAS_FAULT=canary for the batch being queued
    // tracing
    bool profiling = false;
    int64_t prof_trials = 0;
    int64_t launches[4] = {0, 0, 0, 0};
    int64_t timed[4] = {0, 0, 0, 0};
    double prof_ms[4] = {0, 0, 0, 0};
    cudaStream_t aux = nullptr;     // second stream (harmonic sum overlap), lowest priority
    cudaStream_t hi = nullptr;      // spectrum + correlation, highest priority
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;   // caller's stream <-> hi
    cudaEvent_t ev_conv[2] = {nullptr, nullptr};
    cudaEvent_t ev_hsum[2] = {nullptr, nullptr};
};

// ---------------------------------------------------------------------------
// launchers (each returns the launch status)
// ---------------------------------------------------------------------------
fdas_status launch_template_bank(Plan &p, cudaStream_t s);
fdas_status launch_spectrum(Plan &p, const float *x, void *spec_out_padded,
                            float *medians, cudaStream_t s);
// cplx: write the complex F (plane of the plan's complex type) instead of
// |F|^2 and its statistics
fdas_status launch_correlate(Plan &p, const void *spec_padded, void *plane,
                             double2 *partials, cudaStream_t s, bool cplx = false);
int correlate_ctas(const Plan &p);
// tensor-core correlation: whether it applies to the plan's geometry, the
// host-side chunk table, the operand images (from the FP64 taps) and launch
bool tc_applicable(const Plan &p, std::string *why);
int tc_image_buffers(const Plan &p);
std::vector<TcChunk> tc_chunk_table(const Plan &p, const std::vector<int32_t> &m, int *win,
                                    int *max_ks);
fdas_status launch_tc_bank(Plan &p, cudaStream_t s);
fdas_status launch_correlate_tc(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                                cudaStream_t s, bool cplx);
int correlate_tc_ctas(const Plan &p);
// interbinning fused into the tensor-core epilogue: the half-bin plane and
// its partials (interbin_tc_partials of them), using the plan's edge table
fdas_status launch_interbin_tc(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                               cudaStream_t s);
int interbin_tc_partials(const Plan &p);
int64_t tc_edge_bytes(const Plan &p);
int64_t tc_bank_bytes(const std::vector<TcChunk> &table);
// interbinning: complex F [n_z][n_r] -> plane [n_z][2 n_r] and one FP64
// (sum P, sum P^2) partial per CTA
fdas_status launch_interbin(Plan &p, const void *F, void *plane, double2 *partials,
                            cudaStream_t s);
int interbin_ctas(const Plan &p);
// columns of the power plane: n_r, or 2 n_r on the half-bin grid
inline int64_t plane_cols(const Plan &p) { return p.interbin ? 2 * p.n_r : p.n_r; }
fdas_status launch_finalize_stats(Plan &p, const double2 *partials, int n_partials,
                                  const double *given_stats, TrialStats *out,
                                  cudaStream_t s);
fdas_status launch_harmonic_threshold(Plan &p, const void *plane,
                                      const TrialStats *st, uint32_t rank,
                                      cudaStream_t s);
fdas_status launch_harmonic_sums(Plan &p, const void *plane, float *out,
                                 cudaStream_t s);
fdas_status launch_stuck_wait(unsigned int *flags, long long limit_cycles, cudaStream_t s);
fdas_status launch_candidates_finish(Plan &p, int64_t n, fdas_candidate *out_dev,
                                     cudaStream_t s);
// stream-ordered end of a search: status and counts into p.async_res, the
// records ordered and the first min(n, capacity) written to out_dev, all
// from the count in device memory
fdas_status launch_candidates_finish_async(Plan &p, int64_t capacity, unsigned int extra_flags,
                                           fdas_candidate *out_dev, cudaStream_t s);
std::vector<float2> gauss_legendre_01(int n);
int refine_nodes();
fdas_status launch_fourier_power(Plan &p, const float2 *X, const double2 *rz, int n, float *power,
                                 float2 *grad, cudaStream_t s);
fdas_status launch_fourier_power_backward(Plan &p, const float2 *X, const double2 *rz, int n,
                                          const float *gP, float2 *grad_X, double2 *grad_rz,
                                          cudaStream_t s);
fdas_status launch_refine(Plan &p, const float2 *X, const fdas_seed *seeds, int n, int n_steps,
                          fdas_refined *out, cudaStream_t s);

}  // namespace fdas
