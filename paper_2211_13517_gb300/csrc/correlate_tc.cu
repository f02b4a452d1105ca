// The power plane on the tensor cores: the direct correlation as a GEMM.
//
// The matched filter of paper §2.1, F(r, z) = sum_{|e| <= m(z)} g_z[e] X'_{r-e},
// P = |F|^2, is a product of two dense matrices once the spectrum is read as a
// Hankel matrix.  For a tile of 512 bins starting at r_b and a chunk of 28
// templates:
//
//   row i (0..127) of A holds the spectrum window X'_{r_b - W0 + 4i + q},
//   q = kofs .. (complex, as interleaved 16-bit (re, im) pairs along K);
//   column n = 8 zz + 4 c + p of B holds, at K position (q, re/im), the tap
//   g_z[e] with e = p + W0 - kofs - q arranged so that the dot product gives
//   Re F (c = 0) or Im F (c = 1) at r = r_b + 4i + p, p = 0..3.
//
// Row i + 1 of A is row i moved by 4 complex values = 16 bytes, so A needs no
// copy at all: the window itself, described to the tensor core as a K-major
// operand whose 8-row core matrices are 16 bytes apart along K (LBO = 16) and
// 128 bytes apart along M (SBO = 128), *is* the Hankel matrix.  The four
// phases p live in the template operand instead (B columns shifted by p taps),
// so one accumulator row holds four consecutive bins of every template.
//
// One persistent CTA per SM takes, for every chunk in turn, every G-th tile
// (G = the number of CTAs).  Warp 0 (one thread) bulk-copies the chunk's template image (B, up to
// 208 KB, once per chunk) and the spectrum windows (A, a ring of 4) into shared
// memory; warp 1 (one thread) issues the tcgen05 MMAs (M = 128, N = 224, K = 16
// each, BF16 or FP16 operands, FP32 accumulators) into one of two TMEM
// accumulators; warps 2..9 read the finished accumulator (tcgen05.ld, all
// loads of a tile before one wait, then release the accumulator at once),
// form P = re^2 + im^2 with packed FP32x2 arithmetic (the column order puts
// the re and the im parts of the 4 phases side by side), store 4 consecutive
// bins per template as one 8-byte store, and sum P and P^2 for the plane
// statistics (FP32 per tile, FP64 across tiles).  All waits are bounded; a
// wait that gives up sets flag bit 2.
//
// Unit template energy (noise cells distributed as Exp(1)) is kept for the
// taps as rounded to 16 bits: P is |F|^2 / E'_z with E'_z = sum_e |g'_z[e]|^2
// of the rounded taps g', one FP32 factor per template.
//
// kMode selects the epilogue: kPower writes P as above; kCplx writes the
// complex F / sqrt(E'_z) (4 consecutive bins per template as one 16-byte
// store, no statistics); kInterbin writes the half-bin plane directly: the 4
// bins of a row and their 4 half bins (pi/4)^2 |F(r) - F(r+1)|^2 as one
// 16-byte store into the 2 N_r-column plane, F(r + 1) of a row's last bin
// taken from the next lane.  The last lane of each warp has no next row in
// the warp: it leaves that half bin for tc_ib_fixup_kernel, and lanes 0 and
// 31 record their first and last F of the tile in an edge table from which
// the fix-up computes it (with F(N_r) = 0 after the last tile).
#include <algorithm>
#include <array>

#include "fdas_internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"
#include "check.cuh"

namespace fdas {

namespace {

constexpr int kTcRows = 128;                     // GEMM rows = TMEM lanes per tile
constexpr int kTcPhases = 4;                     // r = r_b + 4 i + p
constexpr int kTcTile = kTcRows * kTcPhases;     // bins per tile
constexpr int kTcZ = 28;                         // templates per chunk
constexpr int kTcN = kTcZ * kTcPhases * 2;       // GEMM columns (224)
constexpr int kTcSlab = kTcN / 8 * 256;          // bytes of B per K step of 16
constexpr int kTcStages = 4;                     // spectrum-window ring
constexpr int kTcEpiWarps = 8;
constexpr int kTcZpt = kTcZ / (kTcEpiWarps / 4);   // templates per epilogue thread
static_assert(kTcZ % (kTcEpiWarps / 4) == 0, "epilogue split");
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);
constexpr int kTcTmemCols = 512;
constexpr int kTcAccStride = 256;                // TMEM column of accumulator 1
constexpr size_t kTcMinSmem = 120 * 1024;        // keeps one CTA (and one TMEM owner) per SM
constexpr int kTcCtasPerSm = 1;                  // persistent CTAs per SM

// The (chunk, tile) items of CTA k of G: for every chunk in turn, the tiles
// k, k + G, k + 2G, ...  Every CTA gets the same mix of chunks (the tile
// counts per chunk differ by at most one between CTAs), so the CTAs finish
// together whatever a chunk's cost, and at any time the G CTAs work on G
// adjacent tiles of one chunk (the spectrum windows and the plane rows they
// touch are contiguous).  Producer, MMA thread and epilogue walk the same
// sequence.
struct TcSchedule {
    int n_ch, c, k, G;
    int64_t n_tiles, t;
    __device__ TcSchedule(const TcChunk *, int n_ch_, int64_t n_tiles_, int k_, int G_)
        : n_ch(n_ch_), c(0), k(k_), G(G_), n_tiles(n_tiles_), t(k_) {}
    __device__ bool next(int &oc, int64_t &ot) {
        while (c < n_ch) {
            if (t < n_tiles) {
                oc = c;
                ot = t;
                t += G;
                return true;
            }
            ++c;
            t = k;
        }
        return false;
    }
};

__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

enum { kPower = 0, kCplx = 1, kInterbin = 2 };
constexpr float kIbFactor = 0.61685027506808491f;   // (pi/4)^2

// P = PrecF32 is the split mode of FP32 plans: spectrum and taps are each
// the sum of two BF16 parts (hi + lo), every K step issues the three MMAs
// hi*hi + hi*lo + lo*hi into the same FP32 accumulator (the lo*lo term,
// about 2^-16 of the product, is dropped), the template image is twice as
// large (its lo half `b_lo` bytes after the hi one), two spectrum windows per
// stage, two stages, and the plane is stored in FP32.
template <class P, int kMode>
__global__ void __launch_bounds__(kTcThreads, 1)
    correlate_tc_kernel(const unsigned char *__restrict__ spec_a,
                        const unsigned char *__restrict__ spec_lo,
                        const unsigned char *__restrict__ bank_img, int64_t b_lo,
                        const TcChunk *__restrict__ chunks, int n_ch,
                        const float *__restrict__ inv_energy,
                        void *__restrict__ out, double2 *__restrict__ partials,
                        int64_t n_r, int win_bytes, int b_bytes_max, int nbuf,
                        unsigned int *flags,
                        float4 *__restrict__ edges FDAS_BC_PARAM) {
    constexpr bool kSplit = P::id == FDAS_FP32;
    constexpr int kStages = kSplit ? 2 : kTcStages;
    constexpr int kParts = kSplit ? 2 : 1;   // hi (+ lo) operand images
    extern __shared__ __align__(128) unsigned char tc_smem[];
    // nbuf (1 or 2) template images, then the spectrum-window ring; with two
    // images the next chunk's is copied while the MMAs of the current one run
    unsigned char *const sB = tc_smem;
    const int b_stride = kParts * b_bytes_max;
    unsigned char *const sA = tc_smem + nbuf * b_stride;
    __shared__ __align__(8) uint64_t a_full[kTcStages], a_empty[kTcStages];
    __shared__ __align__(8) uint64_t b_full[2], b_empty[2], acc_full[2], acc_empty[2], drain;
    __shared__ uint32_t tmem_base_sh;
    __shared__ double red[2][kTcEpiWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = n_r / kTcTile;
    constexpr bool kBF16 = P::id == FDAS_BF16 || kSplit;
    constexpr uint32_t kIdesc = idesc_f16<kBF16>(kTcRows, kTcN);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&b_full[i], 1);
            mbar_init(&b_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kTcEpiWarps);
        }
        mbar_init(&drain, 1);
        mbar_fence_init();
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(&tmem_base_sh, kTcTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            // producer: template image per chunk, spectrum window per tile
            TcSchedule sch(chunks, n_ch, n_tiles, blockIdx.x, gridDim.x);
            int c, cur = -1, run = -1;
            int64_t t;
            int j = 0;
            while (sch.next(c, t)) {
                if (c != cur) {
                    ++run;
                    const int bb = run % nbuf;
                    // the image buffer is free once the MMAs of run - nbuf completed
                    if (run >= nbuf && !mbar_wait(&b_empty[bb], ((run / nbuf) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const unsigned bytes = (unsigned)chunks[c].ks * kTcSlab;
                    unsigned char *const dstB = sB + bb * b_stride;
                    if (FDAS_IN_BOUNDS(0, bytes, b_bytes_max, kSiteTcImageSmem) &&
                        FDAS_IN_BOUNDS(chunks[c].b_off, bytes, kSplit ? b_lo : bc.lim[0],
                                       kSiteTcImageCopy) &&
                        (!kSplit || FDAS_IN_BOUNDS(b_lo + chunks[c].b_off, bytes, bc.lim[0],
                                                   kSiteTcImageCopy))) {
                        mbar_arrive_expect_tx(&b_full[bb], kParts * bytes);
                        bulk_copy_g2s(dstB, bank_img + chunks[c].b_off, bytes, &b_full[bb]);
                        if constexpr (kSplit)
                            bulk_copy_g2s(dstB + b_bytes_max, bank_img + b_lo + chunks[c].b_off,
                                          bytes, &b_full[bb]);
                    } else {
                        mbar_arrive(&b_full[bb]);   // checked build: the copy is skipped
                    }
                    cur = c;
                }
                const int s = j % kStages;
                if (j >= kStages && !mbar_wait(&a_empty[s], ((j / kStages) - 1) & 1)) {
                    ok = false;
                    break;
                }
                // a window of 16-bit (re, im) pairs: 4 bytes per complex value
                const int64_t a_off = t * kTcTile * 4;
                unsigned char *const dstA = sA + s * kParts * win_bytes;
                if (FDAS_IN_BOUNDS(a_off, win_bytes, bc.lim[1], kSiteTcWindowCopy)) {
                    mbar_arrive_expect_tx(&a_full[s], (unsigned)(kParts * win_bytes));
                    bulk_copy_g2s(dstA, spec_a + a_off, (unsigned)win_bytes, &a_full[s]);
                    if constexpr (kSplit)
                        bulk_copy_g2s(dstA + win_bytes, spec_lo + a_off, (unsigned)win_bytes,
                                      &a_full[s]);
                } else {
                    mbar_arrive(&a_full[s]);   // checked build: the copy is skipped
                }
                ++j;
            }
            // every copy issued lands before the CTA can exit (bounded)
            for (int s = 0; s < kStages && s < j; ++s) {
                const int uses = (j - 1 - s) / kStages + 1;
                (void)mbar_wait(&a_full[s], (uses - 1) & 1);
            }
            for (int r = run - nbuf + 1; r <= run; ++r)
                if (r >= 0) (void)mbar_wait(&b_full[r % nbuf], (r / nbuf) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            TcSchedule sch(chunks, n_ch, n_tiles, blockIdx.x, gridDim.x);
            int c, cur = -1, run = -1, ks = 0, kofs = 0;
            int64_t t;
            int j = 0;
            uint64_t bdesc0 = 0, bdesc_lo = 0;
            while (sch.next(c, t)) {
                if (c != cur) {
                    if (cur >= 0) tc_commit(&b_empty[run % nbuf]);   // the old image is free
                    ++run;
                    cur = c;
                    const unsigned char *const img = sB + (run % nbuf) * b_stride;
                    bdesc0 = smem_desc(smem_u32(img), 128, 256);
                    bdesc_lo = smem_desc(smem_u32(img + (kSplit ? b_bytes_max : 0)), 128, 256);
                    if (!mbar_wait(&b_full[run % nbuf], (run / nbuf) & 1)) {
                        ok = false;
                        break;
                    }
                    ks = chunks[c].ks;
                    kofs = chunks[c].kofs;
                }
                const int s = j % kStages, b = j & 1;
                if (!mbar_test(&a_full[s], (j / kStages) & 1) &&
                    !mbar_wait(&a_full[s], (j / kStages) & 1)) {
                    ok = false;
                    break;
                }
                if (j >= 2 && !mbar_test(&acc_empty[b], ((j >> 1) - 1) & 1) &&
                    !mbar_wait(&acc_empty[b], ((j >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kTcAccStride);
                const uint32_t a_addr = smem_u32(sA + s * kParts * win_bytes) + 4u * kofs;
                const uint64_t adesc = smem_desc(a_addr, 16, 128);
                const uint64_t adesc_lo = smem_desc(a_addr + (kSplit ? (uint32_t)win_bytes : 0u), 16, 128);
                // (checked build: no MMA reads past the window or the image)
                const int kn = FDAS_IN_BOUNDS(kofs, 4 * (kTcRows - 1) + 8 * ks, win_bytes / 4,
                                              kSiteTcWindowRead) &&
                                       FDAS_IN_BOUNDS(0, ks * kTcSlab, b_bytes_max, kSiteTcImageSmem)
                                   ? ks
                                   : 0;
                for (int k = 0; k < kn; ++k) {
                    const uint64_t kb = (uint64_t)(kTcSlab >> 4) * k;
                    tc_mma_f16(d, adesc + 2ull * k, bdesc0 + kb, kIdesc, k > 0 ? 1u : 0u);
                    if constexpr (kSplit) {
                        tc_mma_f16(d, adesc + 2ull * k, bdesc_lo + kb, kIdesc, 1u);
                        tc_mma_f16(d, adesc_lo + 2ull * k, bdesc0 + kb, kIdesc, 1u);
                    }
                }
                tc_commit(&acc_full[b]);
                tc_commit(&a_empty[s]);
                ++j;
            }
            // every MMA issued has completed before TMEM is released (bounded)
            tc_commit(&drain);
            (void)mbar_wait(&drain, 0);
        }
    } else {
        // epilogue: TMEM lanes 32 (warp % 4) .. + 31 (rows), templates
        // kTcZpt part .. + kTcZpt - 1 of the chunk, part = (warp - 2) / 4
        const int quarter = warp & 3;
        const int part = (warp - 2) >> 2;
        const int row = 32 * quarter + lane;
        const uint32_t tlane = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(8 * kTcZpt * part);
        TcSchedule sch(chunks, n_ch, n_tiles, blockIdx.x, gridDim.x);
        int c, cur = -1, zvalid = 0;
        int64_t t;
        int j = 0;
        float sc[kTcZpt];   // 1 / E'_z (power) or 1 / sqrt(E'_z) (complex, half bins)
        int zfirst = 0;     // first template of this warp's part of the chunk
        typename P::real *zrow = static_cast<typename P::real *>(out);
        typename P::cpx *zcrow = static_cast<typename P::cpx *>(out);
        float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
        // compensated FP32 sums across tiles (FP64 only once, at the end: the
        // FP64 pipe is a small fraction of the FP32 one)
        float2 k1 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
        float2 k2 = make_float2(0.f, 0.f), c2 = make_float2(0.f, 0.f);
        constexpr float ps = P::plane_scale;
        while (sch.next(c, t)) {
            if (c != cur) {
                cur = c;
                const int zb = chunks[c].z_part[part];
                zvalid = chunks[c].n_part[part];
#pragma unroll
                for (int k = 0; k < kTcZpt; ++k) {
                    const float ie = k < zvalid && FDAS_IN_BOUNDS(zb + k, 1, bc.lim[2], kSiteTcEnergy)
                                         ? __ldg(inv_energy + zb + k)
                                         : 0.f;
                    sc[k] = kMode == kPower ? ie : sqrtf(ie);
                }
                if constexpr (kMode == kCplx)
                    zcrow = static_cast<typename P::cpx *>(out) + (int64_t)zb * n_r + 4 * row;
                else if constexpr (kMode == kInterbin)
                    zrow = static_cast<typename P::real *>(out) + (int64_t)zb * 2 * n_r + 8 * row;
                else
                    zrow = static_cast<typename P::real *>(out) + (int64_t)zb * n_r + 4 * row;
                zfirst = zb;
            }
            const int b = j & 1;
            const bool got = mbar_wait(&acc_full[b], (j >> 1) & 1);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            tc_fence_after();
            uint32_t v[kTcZpt][8];
#pragma unroll
            for (int k = 0; k < kTcZpt; ++k)
                tmem_ld8(tlane + (uint32_t)(b * kTcAccStride + 8 * k), v[k]);
            tmem_ld_wait();
            // the accumulator is in registers: hand it back to the MMA thread
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            if constexpr (kMode == kInterbin) {
                typename P::real *o = zrow + t * (2 * kTcTile);
                const float2 ib = make_float2(kIbFactor, kIbFactor);
#pragma unroll
                for (int k = 0; k < kTcZpt; ++k) {
                    if (k < zvalid) {   // warp-uniform: the shuffles see every lane
                        const float2 sk = make_float2(sc[k], sc[k]);
                        const float2 re01 = __fmul2_rn(make_float2(__uint_as_float(v[k][0]), __uint_as_float(v[k][1])), sk);
                        const float2 re23 = __fmul2_rn(make_float2(__uint_as_float(v[k][2]), __uint_as_float(v[k][3])), sk);
                        const float2 im01 = __fmul2_rn(make_float2(__uint_as_float(v[k][4]), __uint_as_float(v[k][5])), sk);
                        const float2 im23 = __fmul2_rn(make_float2(__uint_as_float(v[k][6]), __uint_as_float(v[k][7])), sk);
                        // F(r + 4) of this row's last bin is the next row's first bin
                        const float nre = __shfl_down_sync(0xffffffffu, re01.x, 1);
                        const float nim = __shfl_down_sync(0xffffffffu, im01.x, 1);
                        const float2 p01 = __ffma2_rn(re01, re01, __fmul2_rn(im01, im01));
                        const float2 p23 = __ffma2_rn(re23, re23, __fmul2_rn(im23, im23));
                        const float2 dr01 = fsub2(re01, make_float2(re01.y, re23.x));
                        const float2 di01 = fsub2(im01, make_float2(im01.y, im23.x));
                        const float2 dr23 = fsub2(re23, make_float2(re23.y, nre));
                        const float2 di23 = fsub2(im23, make_float2(im23.y, nim));
                        const float2 q01 = __fmul2_rn(__ffma2_rn(dr01, dr01, __fmul2_rn(di01, di01)), ib);
                        float2 q23 = __fmul2_rn(__ffma2_rn(dr23, dr23, __fmul2_rn(di23, di23)), ib);
                        if (lane == 31) {
                            // the next row is in another warp or tile: the
                            // fix-up kernel writes this half bin
                            q23.y = 0.f;
                            const int64_t e = ((int64_t)(zfirst + k) * n_tiles + t) * 4 + quarter;
                            if (FDAS_IN_BOUNDS(e, 1, bc.lim[2] * n_tiles * 4, kSiteTcEdgeStore))
                                reinterpret_cast<float2 *>(edges + e)[1] = make_float2(re23.y, im23.y);
                        }
                        if (lane == 0) {
                            const int64_t e = ((int64_t)(zfirst + k) * n_tiles + t) * 4 + quarter;
                            if (FDAS_IN_BOUNDS(e, 1, bc.lim[2] * n_tiles * 4, kSiteTcEdgeStore))
                                reinterpret_cast<float2 *>(edges + e)[0] = make_float2(re01.x, im01.x);
                        }
                        s1 = __fadd2_rn(s1, __fadd2_rn(__fadd2_rn(p01, p23), __fadd2_rn(q01, q23)));
                        s2 = __ffma2_rn(p01, p01, s2);
                        s2 = __ffma2_rn(p23, p23, s2);
                        s2 = __ffma2_rn(q01, q01, s2);
                        s2 = __ffma2_rn(q23, q23, s2);
                        const float2 pss = make_float2(ps, ps);
                        const typename P::cpx w0 = P::st(__fmul2_rn(make_float2(p01.x, q01.x), pss));
                        const typename P::cpx w1 = P::st(__fmul2_rn(make_float2(p01.y, q01.y), pss));
                        const typename P::cpx w2 = P::st(__fmul2_rn(make_float2(p23.x, q23.x), pss));
                        const typename P::cpx w3 = P::st(__fmul2_rn(make_float2(p23.y, q23.y), pss));
                        uint4 u;
                        memcpy(&u.x, &w0, 4);
                        memcpy(&u.y, &w1, 4);
                        memcpy(&u.z, &w2, 4);
                        memcpy(&u.w, &w3, 4);
                        if (FDAS_IN_BOUNDS((int64_t)(zfirst + k) * 2 * n_r + t * (2 * kTcTile) + 8 * row,
                                           8, bc.lim[2] * 2 * n_r, kSiteTcPlaneStore))
                            *reinterpret_cast<uint4 *>(o + (int64_t)k * 2 * n_r) = u;
                    }
                }
            } else if constexpr (kMode == kCplx) {
                typename P::cpx *oc = zcrow + t * kTcTile;
#pragma unroll
                for (int k = 0; k < kTcZpt; ++k) {
                    if (k < zvalid &&
                        FDAS_IN_BOUNDS((int64_t)(zfirst + k) * n_r + t * kTcTile + 4 * row, 4,
                                       bc.lim[2] * n_r, kSiteTcPlaneStore)) {
                        uint32_t w[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const typename P::cpx cq = P::st(make_float2(
                                __uint_as_float(v[k][q]) * sc[k], __uint_as_float(v[k][4 + q]) * sc[k]));
                            memcpy(&w[q], &cq, 4);
                        }
                        *reinterpret_cast<uint4 *>(oc + (int64_t)k * n_r) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                ++j;
                continue;
            } else {
            typename P::real *o = zrow + t * kTcTile;
#pragma unroll
            for (int k = 0; k < kTcZpt; ++k) {
                const float2 sk = make_float2(sc[k], sc[k]);
                const float2 re01 = make_float2(__uint_as_float(v[k][0]), __uint_as_float(v[k][1]));
                const float2 re23 = make_float2(__uint_as_float(v[k][2]), __uint_as_float(v[k][3]));
                const float2 im01 = make_float2(__uint_as_float(v[k][4]), __uint_as_float(v[k][5]));
                const float2 im23 = make_float2(__uint_as_float(v[k][6]), __uint_as_float(v[k][7]));
                const float2 p01 = __fmul2_rn(__ffma2_rn(re01, re01, __fmul2_rn(im01, im01)), sk);
                const float2 p23 = __fmul2_rn(__ffma2_rn(re23, re23, __fmul2_rn(im23, im23)), sk);
                s1 = __fadd2_rn(s1, __fadd2_rn(p01, p23));
                s2 = __ffma2_rn(p01, p01, s2);
                s2 = __ffma2_rn(p23, p23, s2);
                if (k < zvalid &&
                    FDAS_IN_BOUNDS((int64_t)(zfirst + k) * n_r + t * kTcTile + 4 * row, 4,
                                   bc.lim[2] * n_r, kSiteTcPlaneStore)) {
                    if constexpr (kSplit) {
                        *reinterpret_cast<float4 *>(o + (int64_t)k * n_r) =
                            make_float4(p01.x, p01.y, p23.x, p23.y);
                    } else {
                        const typename P::cpx lo =
                            P::st(ps == 1.f ? p01 : __fmul2_rn(p01, make_float2(ps, ps)));
                        const typename P::cpx hi =
                            P::st(ps == 1.f ? p23 : __fmul2_rn(p23, make_float2(ps, ps)));
                        uint2 w;
                        memcpy(&w.x, &lo, 4);
                        memcpy(&w.y, &hi, 4);
                        *reinterpret_cast<uint2 *>(o + (int64_t)k * n_r) = w;
                    }
                }
            }
            }
            // FP32 within a tile, compensated FP32 across tiles
            {
                const float2 y1 = fsub2(s1, c1), t1 = __fadd2_rn(k1, y1);
                c1 = fsub2(fsub2(t1, k1), y1);
                k1 = t1;
                const float2 y2 = fsub2(s2, c2), t2 = __fadd2_rn(k2, y2);
                c2 = fsub2(fsub2(t2, k2), y2);
                k2 = t2;
            }
            s1 = make_float2(0.f, 0.f);
            s2 = make_float2(0.f, 0.f);
            ++j;
        }
        double d1 = ((double)k1.x - (double)c1.x) + ((double)k1.y - (double)c1.y);
        double d2 = ((double)k2.x - (double)c2.x) + ((double)k2.y - (double)c2.y);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            d1 += __shfl_down_sync(0xffffffffu, d1, off);
            d2 += __shfl_down_sync(0xffffffffu, d2, off);
        }
        if (lane == 0) {
            red[0][warp - 2] = d1;
            red[1][warp - 2] = d2;
        }
    }
    if (!ok) atomicOr(flags, 2u);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, q = 0.0;
        for (int w = 0; w < kTcEpiWarps; ++w) {
            a += red[0][w];
            q += red[1][w];
        }
        partials[blockIdx.x] = make_double2(a, q);
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kTcTmemCols);
    }
}

// The template operand of every chunk, laid out exactly as the kernel's
// shared-memory image: per K step a slab of [n-block 28][K core 2][row 8][8
// values]; column n = 8 zz + 4 c + p, K element kk of step k is complex tap
// q = 8 k + kk / 2, component kk % 2 (re, im).
// (split mode: P = PrecBF16 and `lo` set writes the lo part bf16(g - hi) of
// the FP32 tap g, hi = bf16(g))
template <class P>
__global__ void tc_bank_kernel(uint16_t *__restrict__ img, const TcChunk *__restrict__ chunks,
                               const double *__restrict__ taps, const int64_t *__restrict__ off,
                               const int32_t *__restrict__ m, int W0, bool lo) {
    const TcChunk ch = chunks[blockIdx.y];
    const int64_t n_el = (int64_t)ch.ks * (kTcSlab / 2);
    uint16_t *out = img + ch.b_off / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / (kTcSlab / 2));
        const int e_lin = (int)(i % (kTcSlab / 2));
        const int nb = e_lin / 128, cb = (e_lin / 64) & 1, rw = (e_lin / 8) & 7, kk8 = e_lin & 7;
        const int zz = nb, c = rw >> 2, p = rw & 3;
        const int kk = 8 * cb + kk8;
        const int q = 8 * k + kk / 2, comp = kk & 1;
        const int half = zz / kTcZpt, zk = zz % kTcZpt;
        double v = 0.0;
        if (zk < ch.n_part[half]) {
            const int iz = ch.z_part[half] + zk;
            const int e = p + W0 - ch.kofs - q;
            const int mz = m[iz];
            if (e >= -mz && e <= mz) {
                const int64_t ti = off[iz] + e + mz;
                const double gr = taps[2 * ti], gi = taps[2 * ti + 1];
                v = c == 0 ? (comp == 0 ? gr : -gi) : (comp == 0 ? gi : gr);
            }
        }
        const float vf = (float)v;
        const typename P::real h = P::str(vf);
        const typename P::real r = lo ? P::str(vf - P::ldr(h)) : h;
        uint16_t bits;
        memcpy(&bits, &r, 2);
        out[i] = bits;
    }
}

// 1 / E'_z, E'_z = sum_e |g'_z[e]|^2 of the taps as rounded to the plan's
// 16-bit type (one block per template, FP64 sum in a fixed order)
// (split mode: the taps as hi + lo)
template <class P>
__device__ __forceinline__ float tc_tap(double v, bool split) {
    const float f = (float)v;
    const float h = P::ldr(P::str(f));
    return split ? h + P::ldr(P::str(f - h)) : h;
}

template <class P>
__global__ void tc_energy_kernel(float *__restrict__ inv_energy, const double *__restrict__ taps,
                                 const int64_t *__restrict__ off, const int32_t *__restrict__ m,
                                 bool split) {
    __shared__ double sh[128];
    const int iz = blockIdx.x;
    const int n = 2 * m[iz] + 1;
    double a = 0.0;
    for (int e = threadIdx.x; e < n; e += 128) {
        const int64_t ti = off[iz] + e;
        const float gr = tc_tap<P>(taps[2 * ti], split);
        const float gi = tc_tap<P>(taps[2 * ti + 1], split);
        a += (double)gr * gr + (double)gi * gi;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) inv_energy[iz] = sh[0] > 0.0 ? (float)(1.0 / sh[0]) : 0.f;
}

// The half bins the interbinning epilogue leaves: the last row of each
// warp's 32 rows, whose next bin belongs to another warp or tile.  Entry
// (z, tile, quarter) of the edge table holds that quarter's first F (lane 0,
// .x .y) and last F (lane 31, .z .w); the half bin after the last F uses the
// next entry's first F, or F(N_r) = 0 after the last tile.  One FP64 partial
// (sum Q, sum Q^2) per CTA, after the tensor kernel's.
template <class P>
__global__ void __launch_bounds__(256)
    tc_ib_fixup_kernel(const float4 *__restrict__ edges, typename P::real *__restrict__ plane,
                       double2 *__restrict__ partials, int64_t n_r, int n_z) {
    __shared__ double red[2][8];
    const int64_t n_tiles = n_r / kTcTile;
    const int64_t n = (int64_t)n_z * n_tiles * 4;
    float s1 = 0.f, s2 = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const int q = (int)(i & 3);
        const int64_t zt = i >> 2;
        const int64_t t = zt % n_tiles, z = zt / n_tiles;
        const float4 a = edges[i];
        float2 nx = make_float2(0.f, 0.f);
        if (q < 3 || t + 1 < n_tiles) {
            const float4 b = edges[i + 1];
            nx = make_float2(b.x, b.y);
        }
        const float dr = a.z - nx.x, di = a.w - nx.y;
        const float Q = kIbFactor * fmaf(dr, dr, di * di);
        const int64_t r = t * kTcTile + 128 * q + 127;
        plane[z * 2 * n_r + 2 * r + 1] = P::str(Q * P::plane_scale);
        s1 += Q;
        s2 = fmaf(Q, Q, s2);
    }
    double a1 = s1, a2 = s2;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a1 += __shfl_down_sync(0xffffffffu, a1, off);
        a2 += __shfl_down_sync(0xffffffffu, a2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a1;
        red[1][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < 8; ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        partials[blockIdx.x] = make_double2(t1, t2);
    }
}

int tc_ib_fixup_ctas(const Plan &p) {
    const int64_t n = (int64_t)p.n_z * (p.n_r / kTcTile) * 4;
    return (int)std::max<int64_t>(1, std::min<int64_t>(4 * (int64_t)p.n_sms, (n + 255) / 256));
}

// split mode: the spectrum window as two BF16 parts, hi = bf16(x) and
// lo = bf16(x - hi), over the whole padded buffer
__global__ void tc_split_kernel(const float2 *__restrict__ x, __nv_bfloat162 *__restrict__ hi,
                                __nv_bfloat162 *__restrict__ lo, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        const float2 hf = __bfloat1622float2(h);
        hi[i] = h;
        lo[i] = __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
    }
}

size_t tc_smem_bytes(int max_ks, int win, bool split, int nbuf) {
    const size_t parts = split ? 2 : 1, stages = split ? 2 : kTcStages;
    const size_t need = parts * ((size_t)nbuf * max_ks * kTcSlab + stages * (size_t)win * 4);
    return std::max(need, kTcMinSmem);
}

template <class P, int kMode>
fdas_status launch_tc_P(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                        cudaStream_t s) {
    constexpr bool kSplit = P::id == FDAS_FP32;
    const size_t smem = tc_smem_bytes(p.tc_max_ks, p.tc_win, kSplit, p.tc_nbuf);
    auto k = correlate_tc_kernel<P, kMode>;
    FDAS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = correlate_tc_ctas(p);
    const void *spec_a = spec_padded, *spec_lo = nullptr;
    if constexpr (kSplit) {
        // the FP32 padded spectrum -> its BF16 hi and lo parts
        const int64_t n = p.tc_split_elems;
        const int blocks = (int)std::min<int64_t>(8 * (int64_t)p.n_sms, (n + 255) / 256);
        tc_split_kernel<<<blocks, 256, 0, s>>>((const float2 *)spec_padded,
                                               (__nv_bfloat162 *)p.spec_hi,
                                               (__nv_bfloat162 *)p.spec_lo, n);
        FDAS_CUDA_TRY(cudaGetLastError());
        spec_a = p.spec_hi;
        spec_lo = p.spec_lo;
    }
    k<<<grid, kTcThreads, smem, s>>>((const unsigned char *)spec_a, (const unsigned char *)spec_lo,
                                      (const unsigned char *)p.tc_bank, p.tc_bank_lo, p.tc_chunks,
                                      p.tc_n_ch,
                                      p.tc_inv_energy, plane, partials, p.n_r,
                                      p.tc_win * 4,
                                      p.tc_max_ks * kTcSlab, p.tc_nbuf, p.flags, p.tc_edges
                                      FDAS_BC_ARG(p.tc_img_bytes, 4 * p.spec_pad_elems, p.n_z));
    FDAS_CUDA_TRY(cudaGetLastError());
    if constexpr (kMode == kInterbin) {
        tc_ib_fixup_kernel<P><<<tc_ib_fixup_ctas(p), 256, 0, s>>>(
            p.tc_edges, (typename P::real *)plane, partials + grid, p.n_r, p.n_z);
        FDAS_CUDA_TRY(cudaGetLastError());
    }
    return FDAS_OK;
}

}  // namespace

std::vector<TcChunk> tc_chunk_table(const Plan &p, const std::vector<int32_t> &m, int *win,
                                    int *max_ks) {
    static_assert(kTcZ == 2 * kTcZpt, "two halves of epilogue warps per chunk");
    const int W0 = p.m_ov;
    std::vector<TcChunk> out;
    // the templates of each chunk, by half
    std::vector<std::array<int32_t, 4>> parts;   // z_part[0], n_part[0], z_part[1], n_part[1]
    if (p.tc_order == 0) {
        for (int z0 = 0; z0 < p.n_z; z0 += kTcZ) {
            const int n = std::min(kTcZ, p.n_z - z0);
            parts.push_back({z0, std::min(kTcZpt, n), z0 + kTcZpt, std::max(0, n - kTcZpt)});
        }
    } else {
        // half 0: z = 0, -1, -2, ... (rows iz0, iz0 - 1, ...), half 1: z = 1,
        // 2, ...; chunk c takes the c-th run of 14 of each, so its templates
        // span about 15 values of |z|
        for (int c = 0;; ++c) {
            const int hi0 = p.iz0 - kTcZpt * c;             // last row of half 0
            const int lo0 = std::max(0, hi0 - kTcZpt + 1);
            const int n0 = hi0 >= 0 ? hi0 - lo0 + 1 : 0;
            const int lo1 = p.iz0 + 1 + kTcZpt * c;
            const int n1 = std::max(0, std::min(kTcZpt, p.n_z - lo1));
            if (n0 == 0 && n1 == 0) break;
            parts.push_back({n0 > 0 ? lo0 : 0, n0, n1 > 0 ? lo1 : 0, n1});
        }
    }
    int64_t b_off = 0;
    int wmax = 0, kmax = 0;
    for (const auto &pt : parts) {
        TcChunk c;
        c.z_part[0] = pt[0];
        c.n_part[0] = pt[1];
        c.z_part[1] = pt[2];
        c.n_part[1] = pt[3];
        int mc = 0;
        for (int h = 0; h < 2; ++h)
            for (int iz = c.z_part[h]; iz < c.z_part[h] + c.n_part[h]; ++iz) mc = std::max(mc, m[iz]);
        c.kofs = (W0 - mc) & ~3;
        const int kc = (W0 - c.kofs + mc + 4 + 7) / 8 * 8;   // complex taps q in [0, kc)
        c.ks = kc / 8;
        c.b_off = b_off;
        b_off += (int64_t)c.ks * kTcSlab;
        wmax = std::max(wmax, c.kofs + kc);
        kmax = std::max(kmax, c.ks);
        out.push_back(c);
    }
    *win = (4 * (kTcRows - 1) + wmax + 3) / 4 * 4;
    *max_ks = kmax;
    return out;
}

bool tc_applicable(const Plan &p, std::string *why) {
    if (p.prec == FDAS_FP32 && !p.tc_split) {
        if (why) *why = "the tensor-core correlation takes 16-bit storage (FDAS_BF16/FDAS_FP16), "
                        "or FP32 storage with FDAS_CORR_TENSOR_SPLIT";
        return false;
    }
    if (p.n_r % kTcTile != 0) {
        if (why) *why = "the tensor-core correlation needs n_samples >= 1024";
        return false;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        optin = 0;
    }
    if (tc_smem_bytes(p.tc_max_ks, p.tc_win, p.tc_split, 1) + 1024 > (size_t)optin) {
        if (why) *why = "the widest template chunk does not fit in shared memory (z_max too large)";
        return false;
    }
    return true;
}

// template-image buffers of the tensor-core correlation: two where both fit
// beside the window ring (the next chunk's image then loads while the
// current one is in use), else one
int tc_image_buffers(const Plan &p) {
    if (p.tc_split) return 1;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return tc_smem_bytes(p.tc_max_ks, p.tc_win, false, 2) + 1024 <= (size_t)optin ? 2 : 1;
}

int correlate_tc_ctas(const Plan &p) {
    const int64_t items = (p.n_r / kTcTile) * (int64_t)p.tc_n_ch;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)kTcCtasPerSm * p.n_sms, items));
}

int64_t tc_bank_bytes(const std::vector<TcChunk> &table) {
    int64_t b = 0;
    for (const TcChunk &c : table) b = std::max<int64_t>(b, c.b_off + (int64_t)c.ks * kTcSlab);
    return b;
}

fdas_status launch_tc_bank(Plan &p, cudaStream_t s) {
    dim3 grid(64, p.tc_n_ch);
    switch (p.prec) {
        case FDAS_BF16:
            tc_bank_kernel<PrecBF16><<<grid, 256, 0, s>>>((uint16_t *)p.tc_bank, p.tc_chunks, p.taps,
                                                          p.tap_off, p.tap_m, p.m_ov, false);
            tc_energy_kernel<PrecBF16><<<p.n_z, 128, 0, s>>>(p.tc_inv_energy, p.taps, p.tap_off,
                                                             p.tap_m, false);
            break;
        case FDAS_FP16:
            tc_bank_kernel<PrecF16><<<grid, 256, 0, s>>>((uint16_t *)p.tc_bank, p.tc_chunks, p.taps,
                                                         p.tap_off, p.tap_m, p.m_ov, false);
            tc_energy_kernel<PrecF16><<<p.n_z, 128, 0, s>>>(p.tc_inv_energy, p.taps, p.tap_off,
                                                            p.tap_m, false);
            break;
        case FDAS_FP32:   // split mode: BF16 hi and lo images
            tc_bank_kernel<PrecBF16><<<grid, 256, 0, s>>>((uint16_t *)p.tc_bank, p.tc_chunks, p.taps,
                                                          p.tap_off, p.tap_m, p.m_ov, false);
            tc_bank_kernel<PrecBF16><<<grid, 256, 0, s>>>(
                (uint16_t *)((unsigned char *)p.tc_bank + p.tc_bank_lo), p.tc_chunks, p.taps,
                p.tap_off, p.tap_m, p.m_ov, true);
            tc_energy_kernel<PrecBF16><<<p.n_z, 128, 0, s>>>(p.tc_inv_energy, p.taps, p.tap_off,
                                                             p.tap_m, true);
            break;
        default:
            set_error("tensor-core correlation: 16-bit precisions only");
            return FDAS_ERR_UNSUPPORTED;
    }
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

fdas_status launch_correlate_tc(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                                cudaStream_t s, bool cplx) {
    switch (p.prec) {
        case FDAS_BF16:
            return cplx ? launch_tc_P<PrecBF16, kCplx>(p, spec_padded, plane, partials, s)
                        : launch_tc_P<PrecBF16, kPower>(p, spec_padded, plane, partials, s);
        case FDAS_FP16:
            return cplx ? launch_tc_P<PrecF16, kCplx>(p, spec_padded, plane, partials, s)
                        : launch_tc_P<PrecF16, kPower>(p, spec_padded, plane, partials, s);
        case FDAS_FP32:
            if (cplx) {
                set_error("the split tensor-core correlation writes power planes only");
                return FDAS_ERR_UNSUPPORTED;
            }
            return launch_tc_P<PrecF32, kPower>(p, spec_padded, plane, partials, s);
        default:
            set_error("tensor-core correlation: 16-bit precisions only");
            return FDAS_ERR_UNSUPPORTED;
    }
}

fdas_status launch_interbin_tc(Plan &p, const void *spec_padded, void *plane, double2 *partials,
                               cudaStream_t s) {
    if (!p.tc_edges) {
        set_error("tensor-core interbinning: the plan holds no edge table");
        return FDAS_ERR_UNSUPPORTED;
    }
    switch (p.prec) {
        case FDAS_BF16: return launch_tc_P<PrecBF16, kInterbin>(p, spec_padded, plane, partials, s);
        case FDAS_FP16: return launch_tc_P<PrecF16, kInterbin>(p, spec_padded, plane, partials, s);
        default:
            set_error("tensor-core correlation: 16-bit precisions only");
            return FDAS_ERR_UNSUPPORTED;
    }
}

int interbin_tc_partials(const Plan &p) { return correlate_tc_ctas(p) + tc_ib_fixup_ctas(p); }

int64_t tc_edge_bytes(const Plan &p) { return (int64_t)p.n_z * (p.n_r / kTcTile) * 4 * (int64_t)sizeof(float4); }

FDAS_BOUNDS_LOG_TU(correlate_tc)

}  // namespace fdas
