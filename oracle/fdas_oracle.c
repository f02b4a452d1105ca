/*
 * FP64 CPU oracle for the FDAS hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is part of the correctness oracle.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  The
 * product (the CUDA library) never links, calls or includes anything here,
 * and this file includes nothing from the product.
 *
 * It holds the two loops that are too slow in numpy at full size:
 *
 *  1. the matched filter written as a DIRECT correlation (paper §2.1: FDAS is
 *     a matched filter over acceleration trials; §2.2: FDAS evaluates it as a
 *     convolution, which is mathematically this sum):
 *
 *         F(r, z) = sum_{e=-m(z)}^{m(z)} X'_{r-e} * g_z[e],   P = |F|^2,
 *
 *     with X'_k = 0 for k outside [0, N_r) and g_z[e] = conj(rho(e,z))/sqrt(E_z)
 *     supplied by the caller (computed by quadrature in fdas_oracle.py);
 *
 *  2. the top-harmonic-indexed harmonic sum: for the cell (ir, iz) with
 *     o = iz - iz0, harmonic j of H reads the cell
 *         ir_j = floor((ir*j + H/2)/H),  o_j = sign(o)*floor((|o|*j + H/2)/H)
 *     and stage h (a power of two <= H) sums the harmonics j = k*H/h, k=1..h.
 *
 * Everything is plain FP64 with no blocking or reordering beyond an OpenMP
 * split of the outer loops.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* One cell of the direct correlation, F = (*fr, *fi).  g holds 2m+1 taps,
 * g[e+m] = g_z[e]. */
static void cell_corr(const double *xr, const double *xi, int64_t n_r, int64_t r,
                      int m, const double *gr, const double *gi, double *fr,
                      double *fi)
{
    double sr = 0.0, si = 0.0;
    for (int e = -m; e <= m; ++e) {
        int64_t k = r - e;
        if (k < 0 || k >= n_r)
            continue;
        double ar = xr[k], ai = xi[k];
        double br = gr[e + m], bi = gi[e + m];
        sr += ar * br - ai * bi;
        si += ar * bi + ai * br;
    }
    *fr = sr;
    *fi = si;
}

static double cell_power(const double *xr, const double *xi, int64_t n_r,
                         int64_t r, int m, const double *gr, const double *gi)
{
    double fr, fi;
    cell_corr(xr, xi, n_r, r, m, gr, gi, &fr, &fi);
    return fr * fr + fi * fi;
}

/*
 * Power plane P[iz][r] for iz < n_z, r < n_r (row-major, r contiguous).
 * Template iz has 2*m[iz]+1 taps starting at goff[iz] in gr/gi.
 */
void oracle_plane(const double *xr, const double *xi, int64_t n_r, int n_z,
                  const int32_t *m, const int64_t *goff, const double *gr,
                  const double *gi, double *P)
{
    const int64_t rb = 4096;
    const int64_t n_rb = (n_r + rb - 1) / rb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int iz = 0; iz < n_z; ++iz) {
        for (int64_t b = 0; b < n_rb; ++b) {
            int64_t r_end = (b + 1) * rb < n_r ? (b + 1) * rb : n_r;
            for (int64_t r = b * rb; r < r_end; ++r)
                P[(int64_t)iz * n_r + r] =
                    cell_power(xr, xi, n_r, r, m[iz], gr + goff[iz], gi + goff[iz]);
        }
    }
}

/* The complex correlation plane F[iz][r] = (Fr, Fi), laid out as P above
 * (the input of interbinning, which needs F at neighbouring bins). */
void oracle_corr_plane(const double *xr, const double *xi, int64_t n_r, int n_z,
                       const int32_t *m, const int64_t *goff, const double *gr,
                       const double *gi, double *Fr, double *Fi)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int iz = 0; iz < n_z; ++iz)
        for (int64_t r = 0; r < n_r; ++r)
            cell_corr(xr, xi, n_r, r, m[iz], gr + goff[iz], gi + goff[iz],
                      Fr + (int64_t)iz * n_r + r, Fi + (int64_t)iz * n_r + r);
}

/* The complex sum at an explicit list of cells (sampled interbinning checks). */
void oracle_cells_corr(const double *xr, const double *xi, int64_t n_r,
                       const int32_t *m, const int64_t *goff, const double *gr,
                       const double *gi, int64_t n_cells, const int32_t *iz,
                       const int64_t *r, double *out_re, double *out_im)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_cells; ++c)
        cell_corr(xr, xi, n_r, r[c], m[iz[c]], gr + goff[iz[c]], gi + goff[iz[c]],
                  out_re + c, out_im + c);
}

/* The same sum at an explicit list of cells (sampled checks at full size). */
void oracle_cells(const double *xr, const double *xi, int64_t n_r,
                  const int32_t *m, const int64_t *goff, const double *gr,
                  const double *gi, int64_t n_cells, const int32_t *iz,
                  const int64_t *r, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_cells; ++c)
        out[c] = cell_power(xr, xi, n_r, r[c], m[iz[c]], gr + goff[iz[c]],
                            gi + goff[iz[c]]);
}

static int64_t harm_r(int64_t ir, int j, int H)
{
    return (ir * j + H / 2) / H;
}

static int harm_o(int o, int j, int H)
{
    int a = o < 0 ? -o : o;
    int v = (a * j + H / 2) / H;
    return o < 0 ? -v : v;
}

/* S_h at one cell, straight from the definition. */
static double stage_sum(const double *P, int64_t n_r, int iz0, int H, int h,
                        int iz, int64_t ir)
{
    int o = iz - iz0;
    double s = 0.0;
    for (int k = 1; k <= h; ++k) {
        int j = k * (H / h);
        s += P[(int64_t)(iz0 + harm_o(o, j, H)) * n_r + harm_r(ir, j, H)];
    }
    return s;
}

/* All stage planes: S[st][iz][ir], st = 0..log2(H), h = 2^st. */
void oracle_harmonic_planes(const double *P, int64_t n_r, int n_z, int iz0,
                            int H, double *S)
{
    int n_st = 0;
    while ((1 << n_st) <= H)
        ++n_st;
#pragma omp parallel for collapse(2) schedule(static)
    for (int st = 0; st < n_st; ++st)
        for (int iz = 0; iz < n_z; ++iz)
            for (int64_t ir = 0; ir < n_r; ++ir)
                S[((int64_t)st * n_z + iz) * n_r + ir] =
                    stage_sum(P, n_r, iz0, H, 1 << st, iz, ir);
}

/*
 * Every (stage, iz, ir) with S_h > lo[st]; written in (iz, st, ir) order.
 * Returns the number of such cells; only the first `cap` are stored.
 */
int64_t oracle_harmonic_cells(const double *P, int64_t n_r, int n_z, int iz0,
                              int H, const double *lo, int64_t cap,
                              int32_t *out_st, int32_t *out_iz,
                              int64_t *out_ir, double *out_s)
{
    int n_st = 0;
    while ((1 << n_st) <= H)
        ++n_st;
    int64_t *cnt = (int64_t *)calloc((size_t)n_z, sizeof(int64_t));
    int64_t **rows_ir = (int64_t **)calloc((size_t)n_z, sizeof(int64_t *));
    int32_t **rows_st = (int32_t **)calloc((size_t)n_z, sizeof(int32_t *));
    double **rows_s = (double **)calloc((size_t)n_z, sizeof(double *));
#pragma omp parallel for schedule(dynamic, 1)
    for (int iz = 0; iz < n_z; ++iz) {
        int64_t n = 0, c = 0;
        for (int st = 0; st < n_st; ++st) {
            for (int64_t ir = 0; ir < n_r; ++ir) {
                double s = stage_sum(P, n_r, iz0, H, 1 << st, iz, ir);
                if (s > lo[st]) {
                    if (n == c) {
                        c = c ? 2 * c : 64;
                        rows_ir[iz] = (int64_t *)realloc(rows_ir[iz], (size_t)c * sizeof(int64_t));
                        rows_st[iz] = (int32_t *)realloc(rows_st[iz], (size_t)c * sizeof(int32_t));
                        rows_s[iz] = (double *)realloc(rows_s[iz], (size_t)c * sizeof(double));
                    }
                    rows_ir[iz][n] = ir;
                    rows_st[iz][n] = st;
                    rows_s[iz][n] = s;
                    ++n;
                }
            }
        }
        cnt[iz] = n;
    }
    int64_t total = 0;
    for (int iz = 0; iz < n_z; ++iz) {
        for (int64_t i = 0; i < cnt[iz]; ++i, ++total) {
            if (total < cap) {
                out_st[total] = rows_st[iz][i];
                out_iz[total] = iz;
                out_ir[total] = rows_ir[iz][i];
                out_s[total] = rows_s[iz][i];
            }
        }
        free(rows_ir[iz]);
        free(rows_st[iz]);
        free(rows_s[iz]);
    }
    free(cnt);
    free(rows_ir);
    free(rows_st);
    free(rows_s);
    return total;
}

/* S_h at an explicit list of (stage, iz, ir) cells. */
void oracle_harmonic_at(const double *P, int64_t n_r, int iz0, int H,
                        int64_t n_cells, const int32_t *st, const int32_t *iz,
                        const int64_t *ir, double *out)
{
    for (int64_t c = 0; c < n_cells; ++c)
        out[c] = stage_sum(P, n_r, iz0, H, 1 << st[c], iz[c], ir[c]);
}

/*
 * Fundamental-indexed harmonic sums (the variant in which a candidate is
 * labelled by its fundamental): S_h(iz, ir) = sum_{k=1..h} P[iz0 + k o][k ir],
 * o = iz - iz0, defined where every harmonic k <= h lies in the plane:
 * h ir <= n_r - 1 and 0 <= iz0 + h o < n_z.
 */
static int fund_in_domain(int64_t n_r, int n_z, int iz0, int h, int iz, int64_t ir)
{
    const int64_t top = (int64_t)iz0 + (int64_t)h * (iz - iz0);
    return ir * h <= n_r - 1 && top >= 0 && top < n_z;
}

static double fund_sum(const double *P, int64_t n_r, int iz0, int h, int iz, int64_t ir)
{
    const int o = iz - iz0;
    double s = 0.0;
    for (int k = 1; k <= h; ++k)
        s += P[(int64_t)(iz0 + k * o) * n_r + (int64_t)k * ir];
    return s;
}

/* S[st][iz][ir] (0 outside the stage's domain). */
void oracle_fund_planes(const double *P, int64_t n_r, int n_z, int iz0, int H, double *S)
{
    int n_st = 0;
    while ((1 << n_st) <= H)
        ++n_st;
#pragma omp parallel for collapse(2) schedule(static)
    for (int st = 0; st < n_st; ++st)
        for (int iz = 0; iz < n_z; ++iz)
            for (int64_t ir = 0; ir < n_r; ++ir)
                S[((int64_t)st * n_z + iz) * n_r + ir] =
                    fund_in_domain(n_r, n_z, iz0, 1 << st, iz, ir)
                        ? fund_sum(P, n_r, iz0, 1 << st, iz, ir) : 0.0;
}

/* Every in-domain (stage, iz, ir) with S_h > lo[st], in (iz, st, ir) order;
 * returns the count, stores the first `cap`. */
int64_t oracle_fund_cells(const double *P, int64_t n_r, int n_z, int iz0, int H,
                          const double *lo, int64_t cap, int32_t *out_st,
                          int32_t *out_iz, int64_t *out_ir, double *out_s)
{
    int n_st = 0;
    while ((1 << n_st) <= H)
        ++n_st;
    int64_t total = 0;
    for (int iz = 0; iz < n_z; ++iz)
        for (int st = 0; st < n_st; ++st)
            for (int64_t ir = 0; ir < n_r; ++ir) {
                if (!fund_in_domain(n_r, n_z, iz0, 1 << st, iz, ir))
                    continue;
                const double v = fund_sum(P, n_r, iz0, 1 << st, iz, ir);
                if (v > lo[st]) {
                    if (total < cap) {
                        out_st[total] = st;
                        out_iz[total] = iz;
                        out_ir[total] = ir;
                        out_s[total] = v;
                    }
                    ++total;
                }
            }
    return total;
}

/* Number of OpenMP threads the loops above use (for reporting). */
int oracle_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
