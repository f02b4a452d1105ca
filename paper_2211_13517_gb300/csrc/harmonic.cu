// Plane statistics, harmonic sum + threshold, and candidate ordering.
//
// Harmonic sum (top-harmonic indexing): the cell (ir, iz) with o = iz - iz0 is
// taken as harmonic H of a signal; harmonic j reads the cell
//     (iz0 + sign(o) floor((|o| j + H/2)/H),  floor((ir j + H/2)/H))
// (rounded half up, the z offset away from zero), and stage h = 2^s sums the
// harmonics j = k H / h, k = 1..h.  Stage s therefore equals stage s-1 plus
// the odd multiples of H/h, so one pass over j = H, H/2, H/4, 3H/4, ... gives
// every stage with H gathers per cell.
//
// Threshold: S_h > T_h (strict).  T_h = mean * G_h, G_h = Q^-1(h, Phibar(sigma))
// (the Gamma(h, 1) tail of a sum of h unit exponentials at the Gaussian
// false-alarm probability), or h mean + sigma sqrt(h) std.  Candidates are
// appended with an atomic counter and ordered afterwards by
// (trial rank, stage, iz, ir), so the list does not depend on scheduling.
#include "fdas_internal.cuh"
#include "fft_cta.cuh"   // cadd
#include "tma.cuh"
#include "check.cuh"

#include <cstring>

#include <algorithm>

namespace fdas {
namespace {

constexpr int ilog2h(int n) { return n <= 1 ? 0 : 1 + ilog2h(n >> 1); }

// ---------------------------------------------------------------------------
// statistics: mean/std from the correlation partials (fixed order) or from a
// given {mean, std}; thresholds per stage
// ---------------------------------------------------------------------------
struct ThrParams {
    double G[6];
    double sigma;
    int mode, n_stages;
    double n_cells;
};

__global__ void finalize_stats_kernel(const double2 *__restrict__ partials, int n_partials,
                                      const double *__restrict__ given, TrialStats *out,
                                      ThrParams tp) {
    __shared__ double sa[256], sb[256];
    const int tid = threadIdx.x;
    double a = 0.0, b = 0.0;
    if (given == nullptr) {
        for (int i = tid; i < n_partials; i += 256) {
            a += partials[i].x;
            b += partials[i].y;
        }
    }
    sa[tid] = a;
    sb[tid] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
            sa[tid] += sa[tid + w];
            sb[tid] += sb[tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) {
        double mean, sd;
        if (given != nullptr) {
            mean = given[0];
            sd = given[1];
        } else {
            mean = sa[0] / tp.n_cells;
            const double var = sb[0] / tp.n_cells - mean * mean;
            sd = sqrt(var > 0.0 ? var : 0.0);
        }
        out->mean = mean;
        out->std = sd;
        for (int s = 0; s < 8; ++s) {
            float t = 0.f;
            if (s < tp.n_stages) {
                const double h = (double)(1 << s);
                t = tp.mode == FDAS_THRESH_GAMMA_TAIL ? (float)(mean * tp.G[s])
                                                     : (float)(h * mean + tp.sigma * sqrt(h) * sd);
            }
            out->thr[s] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// harmonic sum + threshold.
//
// One thread owns NC cells of one top row, ir = ir0 + c * 256 (c < NC), so
// every warp-wide load covers 32 consecutive cells.  Because 256 j / H is an
// integer, the source bin of harmonic j for cell c is exactly
// floor((ir0 j + H/2)/H) + c * 256 j / H: per harmonic one row pointer and one
// 32-bit index, and the NC loads use compile-time offsets.  All NC * H loads
// are issued before the first add (they are independent), which keeps enough
// of them in flight to cover the memory latency.  The sums then run in stage
// order (j = H; H/2; H/4, 3H/4; ...), so stage s is a prefix of the running
// sum, and each stage is compared with its threshold.  The grid covers the
// row exactly (NC * 256 divides N/2), so no load needs a bounds test.
// ---------------------------------------------------------------------------
constexpr int kHsThreads = 256;

// harmonic visited at position idx of the stage order
__host__ __device__ constexpr int j_at(int H, int idx) {
    return idx == 0 ? H : ((2 * (idx - (1 << ilog2h(idx))) + 1) * H) >> (ilog2h(idx) + 1);
}

__host__ __device__ constexpr int src_off(int H, int o, int j) {
    return o < 0 ? -(((-o) * j + H / 2) / H) : ((o * j + H / 2) / H);
}


// element offset of the source row of every harmonic for top row iz (the
// same for the whole CTA): threads 0..H-1 fill it, then the CTA synchronises
template <int H>
__device__ __forceinline__ void hs_row_offsets(int iz0, int iz, int64_t n_r, int64_t *rowoff) {
    if (threadIdx.x < H) {
        const int j = threadIdx.x + 1;
        rowoff[threadIdx.x] = (int64_t)(iz0 + src_off(H, iz - iz0, j)) * n_r;
    }
    __syncthreads();
}

template <class P, int H, int NC>
struct HsLoad {
    // v[idx][c]: harmonic j_at(H, idx) of cell c (ir0 + c * kHsThreads)
    template <int IDX>
    __device__ __forceinline__ static void run(const typename P::real *__restrict__ plane,
                                               const int64_t *rowoff, unsigned ir0,
                                               float (&v)[H][NC]) {
        if constexpr (IDX < H) {
            constexpr int J = j_at(H, IDX);
            constexpr unsigned STEP = kHsThreads * J / H;
            constexpr int SH = ilog2h(H);
            const typename P::real *src = plane + rowoff[J - 1] + ((ir0 * J + H / 2) >> SH);
#pragma unroll
            for (int c = 0; c < NC; ++c) v[IDX][c] = P::ldr(__ldg(src + c * STEP));
            run<IDX + 1>(plane, rowoff, ir0, v);
        }
    }
};

// sums in stage order (pairs of cells with packed FP32x2 adds); stage(s, S)
// at the end of every stage
template <int H, int NC, class F>
__device__ __forceinline__ void hs_sums(const float (&v)[H][NC], F &&stage) {
    static_assert(NC % 2 == 0, "cells come in pairs");
    float2 S2[NC / 2];
#pragma unroll
    for (int c = 0; c < NC / 2; ++c) S2[c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int idx = 0; idx < H; ++idx) {
#pragma unroll
        for (int c = 0; c < NC / 2; ++c)
            S2[c] = cadd(S2[c], make_float2(v[idx][2 * c], v[idx][2 * c + 1]));
        if (((idx + 1) & idx) == 0) {
            float S[NC];
#pragma unroll
            for (int c = 0; c < NC / 2; ++c) {
                S[2 * c] = S2[c].x;
                S[2 * c + 1] = S2[c].y;
            }
            stage(ilog2h(idx + 1), S);
        }
    }
}

template <class P, int H, int NC>
__global__ void __launch_bounds__(kHsThreads)
    harmonic_threshold_kernel(const typename P::real *__restrict__ plane, int64_t n_r, int iz0,
                              const TrialStats *__restrict__ st, uint32_t rank,
                              CandRec *__restrict__ cand, unsigned long long *__restrict__ count,
                              int64_t cap) {
    const unsigned ir0 = blockIdx.x * (kHsThreads * NC) + threadIdx.x;
    const int iz = blockIdx.y;
    __shared__ int64_t rowoff[H];
    hs_row_offsets<H>(iz0, iz, n_r, rowoff);
    float v[H][NC];
    HsLoad<P, H, NC>::template run<0>(plane, rowoff, ir0, v);
    const float inv = 1.0f / P::plane_scale;
    hs_sums<H, NC>(v, [&](int s, float (&S)[NC]) {
        const float th = st->thr[s];
        float m = S[0];
#pragma unroll
        for (int c = 1; c < NC; ++c) m = fmaxf(m, S[c]);
        if (m * inv > th) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float val = S[c] * inv;
                if (val > th) {
                    const unsigned long long idx = atomicAdd(count, 1ull);
                    if ((int64_t)idx < cap) {
                        CandRec rec;
                        rec.key = cand_key(rank, s, iz, (uint32_t)(ir0 + c * kHsThreads));
                        rec.power = val;
                        rec.pad = 0.f;
                        cand[idx] = rec;
                    }
                }
            }
        }
    });
}

// all stage sums written out (checking entry point)
template <class P, int H, int NC>
__global__ void __launch_bounds__(kHsThreads)
    harmonic_sums_kernel(const typename P::real *__restrict__ plane, int64_t n_r, int n_z,
                         int iz0, float *__restrict__ out) {
    const unsigned ir0 = blockIdx.x * (kHsThreads * NC) + threadIdx.x;
    const int iz = blockIdx.y;
    __shared__ int64_t rowoff[H];
    hs_row_offsets<H>(iz0, iz, n_r, rowoff);
    float v[H][NC];
    HsLoad<P, H, NC>::template run<0>(plane, rowoff, ir0, v);
    const float inv = 1.0f / P::plane_scale;
    hs_sums<H, NC>(v, [&](int s, float (&S)[NC]) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            out[((int64_t)s * n_z + iz) * n_r + ir0 + c * kHsThreads] = S[c] * inv;
    });
}

// ---------------------------------------------------------------------------
// harmonic sum + threshold for H <= 16 with consecutive cells per thread.
//
// Thread t of a CTA owns the R = 16 consecutive cells b = B + 16 t + i of a
// top row (B = the CTA's first cell, a multiple of 16 T).  Because 16 is a
// multiple of H, harmonic j of cell i reads source bin
//     j (B + 16 t)/H + d_i,   d_i = floor((i j + H/2)/H) <= DMAX_j,
// so the thread needs only the DMAX_j + 1 consecutive bins starting at
// j (B + 16 t)/H, and which of them each cell adds is a compile-time index.
// A CTA (T = 128 threads, 2048 cells) walks QROWS consecutive top rows.  For
// each row, lane j of warp 0 copies, if harmonic j_at(H, j) reads another
// source row than for the previous row (for the first row, every harmonic),
// the span of that source row the CTA needs (starting at j B / H, a multiple
// of 128 elements, so 16-byte aligned) into the harmonic's place in shared
// memory with one bulk asynchronous copy; the lanes issue their copies side
// by side (the span constants of each lane are set once per CTA), which
// keeps the copy issue off the critical path of the row.  From one top row
// to the next, source row o_j changes with probability j/H, so the walk
// copies about 30% fewer bytes than copying every span for every row.  The
// copies of each stage complete on that stage's own mbarrier (bounded waits;
// one phase per row), so the first stages are summed while later spans are
// still arriving.  With 16-bit planes the top row itself (j = H, changed
// every row) is not staged: each thread loads its 16 cells of it from global
// memory into registers one row ahead, which leaves a smaller shared-memory
// footprint (7 CTAs per SM instead of 6).  Each thread reads its values with
// the widest aligned shared-memory loads (a 16-bit window that starts on an
// odd element is read as the aligned 32-bit words around it and shifted down
// by 16 bits), adds them to its cells (16-bit planes: one mixed-precision add
// each), compares each completed stage with its threshold and appends every
// crossing.
// ---------------------------------------------------------------------------
template <class P, int H>
struct Dedup {
    using real = typename P::real;
    static constexpr int R = 16;                                  // cells per thread
    static constexpr int T = 128;                                 // threads per CTA
    static constexpr int CELLS = T * R;
    static constexpr int EPV = 16 / (int)sizeof(real);
    static constexpr int dmax(int j) { return ((R - 1) * j + H / 2) / H; }
    static constexpr int len(int j) { return (R / H) * j * (T - 1) + dmax(j) + 1; }
    // (16-bit planes: + 4, because a window that starts on an odd element is
    // read from the word below, up to two elements past its end; this is
    // shared-memory room only: a copy never reads past the source row's last
    // bin that a cell of the row can read)
    static constexpr int MARGIN = sizeof(real) == 2 ? 4 : 0;
    static constexpr int padlen(int j) { return (len(j) + MARGIN + EPV - 1) / EPV * EPV; }
    static constexpr int off(int j) { return j <= 1 ? 0 : off(j - 1) + padlen(j - 1); }
    // 16-bit planes read the top row (j = H) from global memory into
    // registers, one row ahead; FP32 planes stage it like the others
    static constexpr bool kTopRegs = sizeof(real) == 2;
    static constexpr int SMEM_ELEMS = kTopRegs ? off(H) : off(H + 1);
    // consecutive top rows one CTA walks: from a top row to the next, the
    // source row o_j of harmonic j changes with probability j/H, and only the
    // spans that change are copied again
    static constexpr int QROWS = 16;
    // widest load (elements, power of two <= EPV) that the per-thread start
    // (R/H) j t is always aligned to
    static constexpr int width(int j) {
        int w = 1;
        while (w < EPV && (((R / H) * j) % (2 * w)) == 0) w *= 2;
        return w;
    }
};

// raw vector type of `bytes` bytes
template <int BYTES>
struct RawVec;
template <>
struct RawVec<2> { using type = unsigned short; };
template <>
struct RawVec<4> { using type = uint32_t; };
template <>
struct RawVec<8> { using type = uint2; };
template <>
struct RawVec<16> { using type = uint4; };

// W consecutive stored values (W * sizeof(real) bytes, aligned) -> FP32
template <class P, int W>
struct VecLoad {
    __device__ __forceinline__ static void run(const typename P::real *p, float *o) {
        using R = typename P::real;
        using V = typename RawVec<W * (int)sizeof(R)>::type;
        const V u = *reinterpret_cast<const V *>(p);
        R e[W];
        static_assert(sizeof(e) == sizeof(u), "vector width");
        memcpy(e, &u, sizeof(u));
#pragma unroll
        for (int k = 0; k < W; ++k) o[k] = P::ldr(e[k]);
    }
};

template <class P, int H>
struct DedupSteps {
    using D = Dedup<P, H>;
    using real = typename P::real;

    // harmonics are consumed in stage order j_at(H, 0), j_at(H, 1), ...; the
    // harmonics of stage g (indices [2^(g-1), 2^g), index 0 for g = 0) are
    // copied on barrier g, so the sums of a stage start as soon as its own
    // spans have landed while the later ones are still in flight
    static constexpr int NG = ilog2h(H) + 1;
    static constexpr int group_of(int idx) { return idx == 0 ? 0 : ilog2h(idx) + 1; }
    // bytes of the span of harmonic J for a CTA whose cells all lie inside
    // the row: the full padded length, a compile-time constant
    static constexpr unsigned full_bytes(int J) { return (unsigned)(D::padlen(J) * sizeof(real)); }

    // The span a lane of warp 0 copies: lane IDX takes harmonic j_at(H, IDX),
    // on the barrier of its stage.  Set once per CTA from compile-time values;
    // j = 0 for lanes without a span (and for the top row when it is held in
    // registers).
    struct Lane {
        int j = 0, g = 0, off = 0;
        unsigned full = 0;
    };
    template <int IDX>
    __device__ __forceinline__ static void lane_span(int lane, Lane &L) {
        if constexpr (IDX < H) {
            constexpr int J = j_at(H, IDX), G = group_of(IDX), OFF = D::off(J);
            constexpr unsigned FULL = full_bytes(J);
            constexpr bool kSkip = IDX == 0 && D::kTopRegs;
            if (!kSkip && lane == IDX) {
                L.j = J;
                L.g = G;
                L.off = OFF;
                L.full = FULL;
            }
            lane_span<IDX + 1>(lane, L);
        }
    }
    // per top row: the lane's span if its source row differs from the
    // previous row's (every span for the first row of a walk), copied over
    // the previous row's span with its bytes announced on its stage's
    // barrier; the lanes of warp 0 issue their copies side by side, and one
    // arrival per barrier follows
    __device__ __forceinline__ static void copy_lane(const Lane &L, const real *__restrict__ plane,
                                                     int iz0, int o, int64_t n_r, int64_t B,
                                                     bool first, real *sm, uint64_t *bars,
                                                     int n_z) {
        if (L.j == 0) return;
        if (!first && src_off(H, o, L.j) == src_off(H, o - 1, L.j)) return;
        // the span, but never past the last bin of the source row that a cell
        // of the row reads (c0 and n_r are multiples of EPV, so the rounded
        // end stays within the row)
        const int64_t c0 = (int64_t)L.j * B / H;
        const int64_t maxsrc = ((n_r - 1) * L.j + H / 2) / H;
        int64_t n = maxsrc < c0 ? 0 : (maxsrc - c0 + 1 + D::EPV - 1) / D::EPV * D::EPV;
        if (n * (int64_t)sizeof(real) > (int64_t)L.full) n = L.full / sizeof(real);
        const unsigned bytes = (unsigned)(n * (int64_t)sizeof(real));
        if (bytes == 0) return;
        const int64_t row = iz0 + src_off(H, o, L.j);
        if (!FDAS_IN_BOUNDS(row, 1, n_z, kSiteHsSpanRow) ||
            !FDAS_IN_BOUNDS((int64_t)L.j * B / H, n, n_r, kSiteHsSpanRange))
            return;
        fence_proxy_async_smem();
        mbar_expect_tx(&bars[L.g], bytes);
        bulk_copy_g2s(sm + L.off, plane + row * n_r + (int64_t)L.j * B / H, bytes, &bars[L.g]);
    }

    // 16 consecutive 16-bit cells (32 bytes, aligned) into 8 words
    __device__ __forceinline__ static void load_top(const real *p, uint32_t (&tv)[8]) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
        tv[0] = a.x; tv[1] = a.y; tv[2] = a.z; tv[3] = a.w;
        tv[4] = b.x; tv[5] = b.y; tv[6] = b.z; tv[7] = b.w;
    }

    // add harmonic j_at(H, IDX) to the thread's cells; stage(s, S) at the end
    // of every stage.  False if a stage's copies did not land in time.
    template <int IDX, class F>
    __device__ __forceinline__ static bool sums(const real *sm, uint64_t *bars, unsigned parity,
                                                int t, float2 (&S2)[D::R / 2], F &&stage,
                                                uint32_t (&tv)[8], const real *next_top) {
        if constexpr (IDX == 0 && D::kTopRegs) {
            // j = H: the thread's own 16 cells of the top row, loaded one row
            // earlier; then the load of the next row's is issued
#pragma unroll
            for (int i = 0; i < D::R; ++i) {
                float &s = (i & 1) ? S2[i / 2].y : S2[i / 2].x;
                s = (i & 1) ? P::acc_hi(s, tv[i / 2]) : P::acc_lo(s, tv[i / 2]);
            }
            if (next_top) load_top(next_top, tv);
            stage(0, S2);
            return sums<IDX + 1>(sm, bars, parity, t, S2, stage, tv, next_top);
        } else if constexpr (IDX < H) {
            constexpr int J = j_at(H, IDX);
            if constexpr (IDX == 0 || (IDX & (IDX - 1)) == 0)
                if (!mbar_wait(&bars[group_of(IDX)], parity)) return false;
            constexpr int NVAL = D::dmax(J) + 1;
            constexpr int W = D::width(J);
            constexpr int NLD = (NVAL + W - 1) / W;
            constexpr int OFF = D::off(J);
            const real *p = sm + OFF + (D::R / H) * J * t;
            if constexpr (sizeof(real) == 2) {
                // 16-bit values: keep them packed as loaded and add each to
                // its cell with one mixed-precision add (no conversions)
                if constexpr (W == 1) {
                    // odd start (odd j, H = 16, odd t): read the aligned words
                    // that cover the window and shift them down by 16 bits
                    // (one funnel shift per word), half as many shared-memory
                    // loads as one per 16-bit value
                    constexpr int NR = (NVAL + 1) / 2;          // words after the shift
                    const int e0 = (D::R / H) * J * t;           // first element
                    const uint32_t *pw =
                        reinterpret_cast<const uint32_t *>(sm + OFF) + (e0 >> 1);
                    uint32_t w[NR + 1];
#pragma unroll
                    for (int k = 0; k <= NR; ++k) w[k] = pw[k];
                    const unsigned sh = (unsigned)(e0 & 1) * 16u;
#pragma unroll
                    for (int k = 0; k < NR; ++k) w[k] = __funnelshift_r(w[k], w[k + 1], sh);
#pragma unroll
                    for (int i = 0; i < D::R; ++i) {
                        const int d = (i * J + H / 2) / H;
                        float &s = (i & 1) ? S2[i / 2].y : S2[i / 2].x;
                        s = (d & 1) ? P::acc_hi(s, w[d / 2]) : P::acc_lo(s, w[d / 2]);
                    }
                } else {
                    constexpr int WPL = W / 2;                 // 32-bit words per load
                    using V = typename RawVec<W * 2>::type;
                    uint32_t w[NLD * WPL];
#pragma unroll
                    for (int k = 0; k < NLD; ++k) {
                        const V u = reinterpret_cast<const V *>(p)[k];
                        memcpy(w + k * WPL, &u, sizeof(u));
                    }
#pragma unroll
                    for (int i = 0; i < D::R; ++i) {
                        const int d = (i * J + H / 2) / H;
                        float &s = (i & 1) ? S2[i / 2].y : S2[i / 2].x;
                        s = (d & 1) ? P::acc_hi(s, w[d / 2]) : P::acc_lo(s, w[d / 2]);
                    }
                }
            } else {
                float val[NLD * W];
#pragma unroll
                for (int k = 0; k < NLD; ++k) VecLoad<P, W>::run(p + k * W, val + k * W);
#pragma unroll
                for (int c = 0; c < D::R / 2; ++c) {
                    const int d0 = ((2 * c) * J + H / 2) / H, d1 = ((2 * c + 1) * J + H / 2) / H;
                    S2[c] = cadd(S2[c], make_float2(val[d0], val[d1]));
                }
            }
            if constexpr (((IDX + 1) & IDX) == 0) stage(ilog2h(IDX + 1), S2);
            return sums<IDX + 1>(sm, bars, parity, t, S2, stage, tv, next_top);
        } else {
            return true;
        }
    }
};

template <class P, int H, bool kWriteSums>
__global__ void __launch_bounds__(Dedup<P, H>::T, 7)
    harmonic_dedup_kernel(const typename P::real *__restrict__ plane, int64_t n_r, int n_z,
                          int iz0, const TrialStats *__restrict__ st, uint32_t rank,
                          CandRec *__restrict__ cand, unsigned long long *__restrict__ count,
                          int64_t cap, float *__restrict__ sums_out,
                          unsigned int *__restrict__ flags) {
    using D = Dedup<P, H>;
    using real = typename P::real;
    extern __shared__ __align__(16) unsigned char dd_smem[];
    real *sm = reinterpret_cast<real *>(dd_smem);
    using Steps = DedupSteps<P, H>;
    __shared__ __align__(8) uint64_t bars[Steps::NG];
    const int64_t B = (int64_t)blockIdx.x * D::CELLS;
    const int t = threadIdx.x;
    const int iz_begin = blockIdx.y * D::QROWS;
    const int iz_end = min(iz_begin + D::QROWS, n_z);
    if (t == 0) {
        for (int g = 0; g < Steps::NG; ++g) mbar_init(&bars[g], 1);
        mbar_fence_init();
    }
    const int64_t b = B + (int64_t)D::R * t;   // first cell of this thread
    const bool active = b < n_r;   // thread 0 always is
    typename Steps::Lane lane_sp;
    if (t < 32) Steps::template lane_span<0>(t, lane_sp);
    const float inv = 1.0f / P::plane_scale;
    bool failed = false;
    int q = 0;
    uint32_t tv[8];   // 16-bit planes: the thread's top-row cells, one row ahead
    if constexpr (D::kTopRegs)
        if (active && iz_begin < iz_end &&
            FDAS_IN_BOUNDS((int64_t)iz_begin * n_r + b, D::R, (int64_t)n_z * n_r, kSiteHsTopLoad))
            Steps::load_top(plane + (int64_t)iz_begin * n_r + b, tv);
    for (int iz = iz_begin; iz < iz_end; ++iz, ++q) {
        // every thread is done with the previous row's spans (and, for the
        // first row, the barriers are initialised); stop together after a
        // wait that gave up
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        if (t < 32) {
            // the spans whose source row changed, over the previous row's
            // (their reads by this CTA's threads come before the copies),
            // then one arrival per stage barrier (none on the unused barrier
            // of a top row held in registers)
            Steps::copy_lane(lane_sp, plane, iz0, iz - iz0, n_r, B, q == 0, sm, bars, n_z);
            __syncwarp();
            if (t < Steps::NG && !(t == 0 && D::kTopRegs)) mbar_arrive(&bars[t]);
        }
        if (!active) continue;
        float2 S2[D::R / 2];
#pragma unroll
        for (int c = 0; c < D::R / 2; ++c) S2[c] = make_float2(0.f, 0.f);
        const real *next_top =
            iz + 1 < iz_end && FDAS_IN_BOUNDS((int64_t)(iz + 1) * n_r + b, D::R,
                                              (int64_t)n_z * n_r, kSiteHsTopLoad)
                ? plane + (int64_t)(iz + 1) * n_r + b
                : nullptr;
        const bool ok = Steps::template sums<0>(sm, bars, (unsigned)(q & 1), t, S2,
                                                [&](int s, float2 (&Sv)[D::R / 2]) {
            if constexpr (kWriteSums) {
                if (!FDAS_IN_BOUNDS(((int64_t)s * n_z + iz) * n_r + b, D::R,
                                    (int64_t)(ilog2h(H) + 1) * n_z * n_r, kSiteHsSumsStore))
                    return;
#pragma unroll
                for (int c = 0; c < D::R / 2; ++c) {
                    float *o = sums_out + ((int64_t)s * n_z + iz) * n_r + b + 2 * c;
                    o[0] = Sv[c].x * inv;
                    o[1] = Sv[c].y * inv;
                }
            } else {
                const float th = st->thr[s];
                // largest of the 16 sums: they are >= 0, so their bit patterns
                // order as signed integers (3-input integer max, 8 steps)
                int mi = __vimax3_s32(__float_as_int(Sv[0].x), __float_as_int(Sv[0].y),
                                      __float_as_int(Sv[1].x));
                mi = __vimax3_s32(mi, __float_as_int(Sv[1].y), __float_as_int(Sv[2].x));
#pragma unroll
                for (int c = 2; c < D::R / 2 - 1; ++c)
                    mi = __vimax3_s32(mi, __float_as_int(Sv[c].y), __float_as_int(Sv[c + 1].x));
                mi = max(mi, __float_as_int(Sv[D::R / 2 - 1].y));
                const float m = __int_as_float(mi);
                if (m * inv > th) {
#pragma unroll
                    for (int i = 0; i < D::R; ++i) {
                        const float val = ((i & 1) ? Sv[i / 2].y : Sv[i / 2].x) * inv;
                        if (val > th) {
                            const unsigned long long idx = atomicAdd(count, 1ull);
                            if ((int64_t)idx < cap) {
                                CandRec rec;
                                rec.key = cand_key(rank, s, iz, (uint32_t)(b + i));
                                rec.power = val;
                                rec.pad = 0.f;
                                cand[idx] = rec;
                            }
                        }
                    }
                }
            }
        }, tv, next_top);
        if (!ok) failed = true;
    }
    if (__syncthreads_or(failed)) {
        if (t == 0) atomicOr(flags, 2u);
        // copies still in flight must land before the CTA's shared memory
        // is released (each wait bounded): those of the last row issued
        if (t == 0 && q > 0)
            for (int g = D::kTopRegs ? 1 : 0; g < Steps::NG; ++g)
                (void)mbar_wait(&bars[g], (unsigned)((q - 1) & 1));
    }
}

// ---------------------------------------------------------------------------
// candidate ordering and output
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 1024;
constexpr int kSortChunk = 8192;   // records one CTA sorts in shared memory (128 KB)

__device__ __forceinline__ bool rec_less(const CandRec &a, const CandRec &b) { return a.key < b.key; }

// smallest power of two >= n (n >= 1)
__host__ __device__ __forceinline__ int64_t pow2_at_least(int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

// The record count: from device memory when n_dev is set (the count was
// never brought to the host), else n_host.
__device__ __forceinline__ int64_t sort_count(const int64_t *n_dev, int64_t n_host) {
    return n_dev != nullptr ? *n_dev : n_host;
}

// Bitonic sort of the records [0, n) ascending by key, padded to
// n2 = pow2_at_least(n) with the largest key.  The compare-exchange of
// elements i and i ^ j in stage k sorts ascending where (i & k) == 0 (global
// index), so that every CTA-local part of the network lines up with the
// global one.
//
// sort_chunk_kernel: chunk c = records [c C, c C + C) of the padded array
// in shared memory.  merge_k == 0: every stage k <= min(C, n2) (the whole
// local sort; with n2 <= C this is the complete sort), on the records with
// the padding [n, n2) filled in and written back, so that later steps see n2
// valid entries; merge_k > 0: the steps j < C of stage merge_k, after the
// global steps j >= C of that stage, on the chunk as it stands (records
// and padding have moved by then).
__global__ void __launch_bounds__(kSortThreads) sort_chunk_kernel(CandRec *rec, const int64_t *n_dev,
                                                                  int64_t n_host, int64_t merge_k
                                                                  FDAS_BC_PARAM) {
    extern __shared__ CandRec sh[];
    const int64_t n = sort_count(n_dev, n_host);
    if (n <= 0) return;
    const int64_t n2 = pow2_at_least(n);
    if (merge_k > 0 && (n2 <= kSortChunk || merge_k > n2)) return;
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    if (base >= n2) return;
    const int len = (int)(n2 < kSortChunk ? n2 : kSortChunk);
    if (!FDAS_IN_BOUNDS(base, len, bc.lim[0], kSiteSortRecord)) return;
    const int tid = threadIdx.x;
    for (int i = tid; i < len; i += kSortThreads) {
        if (merge_k > 0 || base + i < n) {
            sh[i] = rec[base + i];
        } else {
            sh[i].key = ~0ull;
            sh[i].power = 0.f;
            sh[i].pad = 0.f;
        }
    }
    __syncthreads();
    auto step = [&](int64_t k, int j) {
        for (int i = tid; i < len; i += kSortThreads) {
            const int ixj = i ^ j;
            if (ixj > i) {
                const bool up = ((base + i) & k) == 0;
                const CandRec a = sh[i], b = sh[ixj];
                if (rec_less(b, a) == up) {
                    sh[i] = b;
                    sh[ixj] = a;
                }
            }
        }
        __syncthreads();
    };
    if (merge_k == 0) {
        for (int k = 2; k <= len; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) step(k, j);
    } else {
        for (int j = len >> 1; j > 0; j >>= 1) step(merge_k, j);
    }
    for (int i = tid; i < len; i += kSortThreads) rec[base + i] = sh[i];
}

// one global compare-exchange step (k, j >= C) over the padded array
// (grid-stride; nothing to do unless C < n2 and k <= n2)
__global__ void bitonic_global_kernel(CandRec *rec, const int64_t *n_dev, int64_t n_host, int64_t k,
                                      int64_t j FDAS_BC_PARAM) {
    const int64_t n = sort_count(n_dev, n_host);
    if (n <= 0) return;
    const int64_t n2 = pow2_at_least(n);
    if (n2 <= kSortChunk || k > n2) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ixj = i ^ j;
        if (ixj <= i) continue;
        if (!FDAS_IN_BOUNDS(ixj, 1, bc.lim[0], kSiteSortRecord)) continue;
        const bool up = (i & k) == 0;
        const CandRec a = rec[i], b = rec[ixj];
        if (rec_less(b, a) == up) {
            rec[i] = b;
            rec[ixj] = a;
        }
    }
}

// the candidate status of a search, computed on the device from the count
// and the error flags (the same rules as the host-side collection)
__global__ void collect_status_kernel(const unsigned long long *__restrict__ count,
                                      const unsigned int *__restrict__ flags, unsigned int extra_flags,
                                      int64_t store_cap, int64_t capacity, AsyncResult *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t total = (int64_t)*count;
    const unsigned int fl = *flags | extra_flags;
    AsyncResult r;
    if (fl & 2u) {
        r.status = FDAS_ERR_TIMEOUT;
        r.n_found = 0;
        r.n_sort = 0;
    } else if (fl & 1u) {
        r.status = FDAS_ERR_NONFINITE;
        r.n_found = 0;
        r.n_sort = 0;
    } else if (total > store_cap) {
        r.status = FDAS_ERR_CAND_STORE_FULL;
        r.n_found = total;
        r.n_sort = 0;
    } else {
        r.status = total > capacity ? FDAS_ERR_CAND_OVERFLOW : FDAS_OK;
        r.n_found = total;
        r.n_sort = total;
    }
    r.n_out = r.n_sort < capacity ? r.n_sort : capacity;
    r.pad = 0;
    *out = r;
}

// log Q(h, x) for integer h: Q = exp(-x) sum_{k<h} x^k / k!
__device__ double log_gamma_tail(int h, double x) {
    if (x <= 0.0) return 0.0;
    const double lx = log(x);
    double lt[32];
    double mx = -1e300, lf = 0.0;
    for (int k = 0; k < h; ++k) {
        if (k > 0) lf += log((double)k);
        lt[k] = k * lx - lf;
        mx = fmax(mx, lt[k]);
    }
    double s = 0.0;
    for (int k = 0; k < h; ++k) s += exp(lt[k] - mx);
    return -x + mx + log(s);
}

// Gaussian-equivalent sigma of an upper-tail probability given as log p
__device__ double sigma_from_logp(double lp) {
    if (lp > -700.0) return -normcdfinv(exp(lp));
    // log Phibar(s) = -s^2/2 - log(s sqrt(2 pi)) + log(1 - 1/s^2 + 3/s^4 - 15/s^6)
    double s = sqrt(-2.0 * lp);
    for (int it = 0; it < 30; ++it) {
        const double s2 = s * s;
        const double corr = log1p(-1.0 / s2 + 3.0 / (s2 * s2) - 15.0 / (s2 * s2 * s2));
        const double f = -0.5 * s2 - log(s) - 0.91893853320467274178 + corr - lp;
        const double df = -s - 1.0 / s;   // derivative of the leading terms
        const double ns = s - f / df;
        if (fabs(ns - s) < 1e-14 * s) {
            s = ns;
            break;
        }
        s = ns;
    }
    return s;
}

// records [0, n) (n = *n_dev when n_dev is set) into caller records; a
// record whose batch rank is not below n_ranks (never one the harmonic
// kernels wrote) is not read further
__global__ void finish_kernel(const CandRec *__restrict__ rec, int64_t n_host,
                              const int64_t *__restrict__ n_dev,
                              const TrialStats *__restrict__ st, const uint32_t *__restrict__ ids,
                              int64_t n_ranks, fdas_candidate *__restrict__ out, int mode) {
    const int64_t n = n_dev != nullptr ? *n_dev : n_host;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const CandRec c = rec[i];
    const uint32_t rank = (uint32_t)(c.key >> 42);
    if ((int64_t)rank >= n_ranks) return;
    const int s = (int)((c.key >> 39) & 7);
    const int iz = (int)((c.key >> 23) & 0xffff);
    const uint32_t ir = (uint32_t)(c.key & 0x7fffff);
    const int h = 1 << s;
    const TrialStats t = st[rank];
    double sig;
    if (mode == FDAS_THRESH_GAMMA_TAIL)
        sig = sigma_from_logp(log_gamma_tail(h, (double)c.power / t.mean));
    else
        sig = ((double)c.power - h * t.mean) / (sqrt((double)h) * t.std);
    fdas_candidate o;
    o.trial_id = ids[rank];
    o.ir = ir;
    o.iz = (uint16_t)iz;
    o.harm = (uint16_t)h;
    o.power = c.power;
    o.sigma = (float)sig;
    out[i] = o;
}

template <class P, int H, bool kWriteSums>
fdas_status launch_dedup(Plan &p, const void *plane, const TrialStats *st, uint32_t rank,
                         float *sums_out, cudaStream_t s) {
    using D = Dedup<P, H>;
    const size_t smem = sizeof(typename P::real) * (size_t)D::SMEM_ELEMS;
    auto k = harmonic_dedup_kernel<P, H, kWriteSums>;
    FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)((p.n_r + D::CELLS - 1) / D::CELLS),
              (unsigned)((p.n_z + D::QROWS - 1) / D::QROWS));
    k<<<grid, D::T, smem, s>>>((const typename P::real *)plane, p.n_r, p.n_z, p.iz0, st, rank,
                               p.cand, p.cand_count, p.store_cap, sums_out, p.flags);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

template <class P, int H, bool kWriteSums>
fdas_status launch_hs(Plan &p, const void *plane, const TrialStats *st, uint32_t rank,
                      float *sums_out, cudaStream_t s) {
    if constexpr (H <= 16) return launch_dedup<P, H, kWriteSums>(p, plane, st, rank, sums_out, s);
    // cells per thread: as many as the register budget allows (NC * H <= 64)
    // and as divide the row into whole CTAs (N/2 is a power of two >= 512)
    constexpr int NCMAX = H >= 32 ? 2 : 4;
    const auto *pl = (const typename P::real *)plane;
    const bool four = NCMAX >= 4 && p.n_r % (kHsThreads * 4) == 0;
    const int nc = four ? 4 : 2;
    dim3 grid((unsigned)(p.n_r / (kHsThreads * nc)), p.n_z);
    if (four) {
        if constexpr (kWriteSums)
            harmonic_sums_kernel<P, H, (NCMAX >= 4 ? 4 : 2)><<<grid, kHsThreads, 0, s>>>(
                pl, p.n_r, p.n_z, p.iz0, sums_out);
        else
            harmonic_threshold_kernel<P, H, (NCMAX >= 4 ? 4 : 2)><<<grid, kHsThreads, 0, s>>>(
                pl, p.n_r, p.iz0, st, rank, p.cand, p.cand_count, p.store_cap);
    } else {
        if constexpr (kWriteSums)
            harmonic_sums_kernel<P, H, 2><<<grid, kHsThreads, 0, s>>>(pl, p.n_r, p.n_z, p.iz0,
                                                                     sums_out);
        else
            harmonic_threshold_kernel<P, H, 2><<<grid, kHsThreads, 0, s>>>(
                pl, p.n_r, p.iz0, st, rank, p.cand, p.cand_count, p.store_cap);
    }
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

// ---------------------------------------------------------------------------
// fundamental-indexed harmonic sum (FDAS_HARM_FUNDAMENTAL).  Thread per
// kFundR = 4 consecutive fundamentals ir = a .. a + 3 of one row o.  Stage 1
// is the cells themselves; stage h adds the exact multiples
// P[iz0 + k o][k ir], k = h/2 + 1 .. h, on the cells where every multiple of
// the stage lies in the plane (h ir <= N_r - 1, |h o| <= K; the domain only
// shrinks as h grows).  For harmonic k the thread loads the contiguous run of
// 4k bins k a .. k (a + 4) - 1 with vector loads (the runs of consecutive
// lanes are adjacent, so the warp reads one contiguous range) and adds its
// every k-th element; cells at the domain's edge take a checked scalar path.
// FP32 sums in the order k = 1, 2, ...
// ---------------------------------------------------------------------------
constexpr int kFundThreads = 256;
constexpr int kFundR = 4;

// the 32-bit words of n bytes at p (16-byte loads when p is 16-byte aligned)
template <int NBYTES>
__device__ __forceinline__ void load_words(const void *p, uint32_t *w, bool aligned16) {
    static_assert(NBYTES % 8 == 0, "8-byte multiples");
    if (aligned16 && NBYTES % 16 == 0) {
#pragma unroll
        for (int q = 0; q < NBYTES / 16; ++q) {
            const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + q);
            w[4 * q] = u.x;
            w[4 * q + 1] = u.y;
            w[4 * q + 2] = u.z;
            w[4 * q + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NBYTES / 8; ++q) {
            const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p) + q);
            w[2 * q] = u.x;
            w[2 * q + 1] = u.y;
        }
    }
}

// element e of the words (16-bit or 32-bit values) as FP32
template <class P>
__device__ __forceinline__ float word_value(const uint32_t *w, int e) {
    if constexpr (sizeof(typename P::real) == 2) {
        const uint32_t x = w[e >> 1];
        const unsigned short h = (unsigned short)((e & 1) ? (x >> 16) : (x & 0xffffu));
        typename P::real r;
        memcpy(&r, &h, 2);
        return P::ldr(r);
    } else {
        return __uint_as_float(w[e]);
    }
}

template <class P, int K>
__device__ __forceinline__ void fund_add_run(const typename P::real *row, int64_t a,
                                             float (&S)[kFundR]) {
    using real = typename P::real;
    constexpr int NBYTES = K * kFundR * (int)sizeof(real);
    uint32_t w[NBYTES / 4];
    const real *p = row + (int64_t)K * a;
    load_words<NBYTES>(p, w, (reinterpret_cast<uintptr_t>(p) & 15u) == 0);
#pragma unroll
    for (int i = 0; i < kFundR; ++i) S[i] += word_value<P>(w, K * i);
}

template <class P, int KLO, int KHI>
__device__ __forceinline__ void fund_add_stage(const typename P::real *plane, int64_t n_r,
                                               int iz0, int o, int64_t a, bool full, int h,
                                               float (&S)[kFundR], int n_z) {
    if constexpr (KLO <= KHI) {
        const typename P::real *row = plane + (int64_t)(iz0 + KLO * o) * n_r;
        if (!FDAS_IN_BOUNDS(iz0 + KLO * o, 1, n_z, kSiteFundRow)) {
        } else if (full) {
            if (FDAS_IN_BOUNDS((int64_t)KLO * a, KLO * kFundR, n_r, kSiteFundRun))
                fund_add_run<P, KLO>(row, a, S);
        } else {
#pragma unroll
            for (int i = 0; i < kFundR; ++i)
                if ((a + i) * h <= n_r - 1) S[i] += P::ldr(row[(int64_t)KLO * (a + i)]);
        }
        fund_add_stage<P, KLO + 1, KHI>(plane, n_r, iz0, o, a, full, h, S, n_z);
    }
}

template <class P, int H, int SV, class F>
__device__ __forceinline__ bool fund_stages(const typename P::real *plane, int64_t n_r, int n_z,
                                            int iz0, int o, int64_t a, float (&S)[kFundR],
                                            int &done, const F &emit) {
    if constexpr ((1 << SV) <= H) {
        constexpr int h = 1 << SV;
        if constexpr (SV > 0) {
            const int top = iz0 + h * o;
            if (top < 0 || top >= n_z || a * h > n_r - 1) return true;
            const bool full = (a + kFundR) * h <= n_r;
            fund_add_stage<P, h / 2 + 1, h>(plane, n_r, iz0, o, a, full, h, S, n_z);
        }
#pragma unroll
        for (int i = 0; i < kFundR; ++i)
            if ((a + i) * h <= n_r - 1) emit(SV, i, S[i]);
        done = SV + 1;
        return fund_stages<P, H, SV + 1, F>(plane, n_r, n_z, iz0, o, a, S, done, emit);
    } else {
        return true;
    }
}

template <class P, int H, bool kWriteSums>
__global__ void __launch_bounds__(kFundThreads)
    harmonic_fund_kernel(const typename P::real *__restrict__ plane, int64_t n_r, int n_z,
                         int iz0, const TrialStats *__restrict__ st, uint32_t rank,
                         CandRec *__restrict__ cand, unsigned long long *__restrict__ count,
                         int64_t cap, float *__restrict__ sums_out) {
    const int64_t a = ((int64_t)blockIdx.x * kFundThreads + threadIdx.x) * kFundR;
    const int iz = blockIdx.y;
    if (a >= n_r) return;   // n_r is a multiple of 4: a .. a + 3 are all inside
    const int o = iz - iz0;
    const float inv = 1.0f / P::plane_scale;
    float S[kFundR];
#pragma unroll
    for (int i = 0; i < kFundR; ++i) S[i] = 0.f;
    // stage 1 is k = 1: the run of the cells themselves
    fund_add_run<P, 1>(plane + (int64_t)iz * n_r, a, S);
    int done = 0;
    auto emit = [&](int sv, int i, float sum) {
        const float val = sum * inv;
        if constexpr (kWriteSums) {
            sums_out[((int64_t)sv * n_z + iz) * n_r + a + i] = val;
        } else {
            if (val > st->thr[sv]) {
                const unsigned long long idx = atomicAdd(count, 1ull);
                if ((int64_t)idx < cap) {
                    CandRec rec;
                    rec.key = cand_key(rank, sv, iz, (uint32_t)(a + i));
                    rec.power = val;
                    rec.pad = 0.f;
                    cand[idx] = rec;
                }
            }
        }
    };
    fund_stages<P, H, 0>(plane, n_r, n_z, iz0, o, a, S, done, emit);
    if constexpr (kWriteSums) {
        // 0 for the stages (and cells) outside the domain
        constexpr int NS = ilog2h(H) + 1;
        for (int sv = 1; sv < NS; ++sv) {
            const int h = 1 << sv;
            const int top = iz0 + h * o;
            for (int i = 0; i < kFundR; ++i)
                if (sv >= done || top < 0 || top >= n_z || (a + i) * h > n_r - 1)
                    sums_out[((int64_t)sv * n_z + iz) * n_r + a + i] = 0.f;
        }
    }
}

template <class P, int H, bool kWriteSums>
fdas_status launch_fund(Plan &p, const void *plane, const TrialStats *st, uint32_t rank,
                        float *sums_out, cudaStream_t s) {
    const int64_t per_cta = (int64_t)kFundThreads * kFundR;
    dim3 grid((unsigned)((p.n_r + per_cta - 1) / per_cta), p.n_z);
    harmonic_fund_kernel<P, H, kWriteSums><<<grid, kFundThreads, 0, s>>>(
        (const typename P::real *)plane, p.n_r, p.n_z, p.iz0, st, rank, p.cand, p.cand_count,
        p.store_cap, sums_out);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

template <class P, int H, bool kWriteSums>
fdas_status launch_hs_mode(Plan &p, const void *plane, const TrialStats *st, uint32_t rank,
                           float *sums_out, cudaStream_t s) {
    if (p.harm_mode == FDAS_HARM_FUNDAMENTAL)
        return launch_fund<P, H, kWriteSums>(p, plane, st, rank, sums_out, s);
    return launch_hs<P, H, kWriteSums>(p, plane, st, rank, sums_out, s);
}

template <class P, bool kWriteSums>
fdas_status launch_hs_P(Plan &p, const void *plane, const TrialStats *st, uint32_t rank,
                        float *sums_out, cudaStream_t s) {
    switch (p.H) {
        case 1: return launch_hs_mode<P, 1, kWriteSums>(p, plane, st, rank, sums_out, s);
        case 2: return launch_hs_mode<P, 2, kWriteSums>(p, plane, st, rank, sums_out, s);
        case 4: return launch_hs_mode<P, 4, kWriteSums>(p, plane, st, rank, sums_out, s);
        case 8: return launch_hs_mode<P, 8, kWriteSums>(p, plane, st, rank, sums_out, s);
        case 16: return launch_hs_mode<P, 16, kWriteSums>(p, plane, st, rank, sums_out, s);
        case 32: return launch_hs_mode<P, 32, kWriteSums>(p, plane, st, rank, sums_out, s);
        default: set_error("bad n_harm"); return FDAS_ERR_ARG;
    }
}

}  // namespace

fdas_status launch_finalize_stats(Plan &p, const double2 *partials, int n_partials,
                                  const double *given_stats, TrialStats *out, cudaStream_t s) {
    ThrParams tp;
    for (int i = 0; i < 6; ++i) tp.G[i] = p.G[i];
    tp.sigma = p.sigma;
    tp.mode = p.thr_mode;
    tp.n_stages = p.n_stages;
    tp.n_cells = (double)p.n_z * (double)p.n_r;
    finalize_stats_kernel<<<1, 256, 0, s>>>(partials, n_partials, given_stats, out, tp);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

fdas_status launch_harmonic_threshold(Plan &p, const void *plane, const TrialStats *st,
                                      uint32_t rank, cudaStream_t s) {
    switch (p.prec) {
        case FDAS_FP32: return launch_hs_P<PrecF32, false>(p, plane, st, rank, nullptr, s);
        case FDAS_BF16: return launch_hs_P<PrecBF16, false>(p, plane, st, rank, nullptr, s);
        default: return launch_hs_P<PrecF16, false>(p, plane, st, rank, nullptr, s);
    }
}

fdas_status launch_harmonic_sums(Plan &p, const void *plane, float *out, cudaStream_t s) {
    switch (p.prec) {
        case FDAS_FP32: return launch_hs_P<PrecF32, true>(p, plane, nullptr, 0, out, s);
        case FDAS_BF16: return launch_hs_P<PrecBF16, true>(p, plane, nullptr, 0, out, s);
        default: return launch_hs_P<PrecF16, true>(p, plane, nullptr, 0, out, s);
    }
}

// sort the first n stored records and convert them to fdas_candidate
// the sort network for n records (host count) or for at most cap records
// with the count in device memory (n_dev): chunk sorts in shared memory, then
// for each stage k > C the global steps j >= C and one chunk merge
static fdas_status launch_sort(Plan &p, int64_t n, const int64_t *n_dev, int64_t cap,
                               cudaStream_t s) {
    const int64_t n2 = pow2_at_least(std::max<int64_t>(1, n_dev ? cap : n));
    const int64_t len = std::min<int64_t>(n2, kSortChunk);
    const unsigned chunks = (unsigned)((n2 + kSortChunk - 1) / kSortChunk);
    const size_t smem = sizeof(CandRec) * (size_t)len;
    [[maybe_unused]] const int64_t rec_cap = pow2_at_least(p.max_cands);   // records p.cand holds
    FDAS_CUDA_TRY(cudaFuncSetAttribute(sort_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(CandRec) * kSortChunk)));
    sort_chunk_kernel<<<chunks, kSortThreads, smem, s>>>(p.cand, n_dev, n, 0 FDAS_BC_ARG(rec_cap));
    FDAS_CUDA_TRY(cudaGetLastError());
    p.launches[FDAS_PROF_FINISH] += 1;
    const unsigned gb = (unsigned)std::min<int64_t>((n2 + 255) / 256, 152 * 16);
    for (int64_t k = 2 * (int64_t)kSortChunk; k <= n2; k <<= 1) {
        for (int64_t j = k >> 1; j >= kSortChunk; j >>= 1) {
            bitonic_global_kernel<<<gb, 256, 0, s>>>(p.cand, n_dev, n, k, j FDAS_BC_ARG(rec_cap));
            FDAS_CUDA_TRY(cudaGetLastError());
            p.launches[FDAS_PROF_FINISH] += 1;
        }
        sort_chunk_kernel<<<chunks, kSortThreads, smem, s>>>(p.cand, n_dev, n, k FDAS_BC_ARG(rec_cap));
        FDAS_CUDA_TRY(cudaGetLastError());
        p.launches[FDAS_PROF_FINISH] += 1;
    }
    return FDAS_OK;
}

fdas_status launch_candidates_finish(Plan &p, int64_t n, fdas_candidate *out_dev, cudaStream_t s) {
    if (n <= 0) return FDAS_OK;
    FDAS_TRY(launch_sort(p, n, nullptr, 0, s));
    finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.cand, n, nullptr, p.stats, p.rank_ids,
                                                               p.stats_cap, out_dev, p.thr_mode);
    FDAS_CUDA_TRY(cudaGetLastError());
    p.launches[FDAS_PROF_FINISH] += 1;
    return FDAS_OK;
}

fdas_status launch_candidates_finish_async(Plan &p, int64_t capacity, unsigned int extra_flags,
                                           fdas_candidate *out_dev, cudaStream_t s) {
    collect_status_kernel<<<1, 32, 0, s>>>(p.cand_count, p.flags, extra_flags, p.store_cap, capacity,
                                           p.async_res);
    FDAS_CUDA_TRY(cudaGetLastError());
    p.launches[FDAS_PROF_FINISH] += 1;
    const int64_t cap = p.store_cap;   // n_sort <= store_cap
    if (cap <= 0) return FDAS_OK;
    FDAS_TRY(launch_sort(p, 0, &p.async_res->n_sort, cap, s));
    const int64_t n_out_max = std::min(cap, capacity);
    if (n_out_max > 0 && out_dev != nullptr) {
        const unsigned gb = (unsigned)((n_out_max + 255) / 256);
        finish_kernel<<<gb, 256, 0, s>>>(p.cand, 0, &p.async_res->n_out, p.stats, p.rank_ids,
                                         p.stats_cap, out_dev, p.thr_mode);
        FDAS_CUDA_TRY(cudaGetLastError());
        p.launches[FDAS_PROF_FINISH] += 1;
    }
    return FDAS_OK;
}

FDAS_BOUNDS_LOG_TU(harmonic)

}  // namespace fdas
