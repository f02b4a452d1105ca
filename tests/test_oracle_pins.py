"""Pins of the FP64 oracle against what mathematics and the paper fix.

None of these compares the oracle with itself: each one checks a step against
a brute-force definition, a closed form, an independent library route
(scipy's Fresnel integrals, scipy's incomplete gamma) or an invariant, chosen
so that a dropped term, a wrong sign or index, or a transposed operand fails
at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sps

import oracle as O
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rho_fresnel(q, z):
    """rho(q, z) through scipy's Fresnel integrals (independent of quadrature).

    With a = z/2 the phase is 2 pi (a u^2 + (q - z/2) u); completing the square
    gives t0 = (q - z/2)/sqrt(z/2), t1 = (q + z/2)/sqrt(z/2) and
    rho = exp(-i pi (q - z/2)^2 / z) / (2 sqrt(z/2)) * [E(t1) - E(t0)],
    E(t) = C(t) + i S(t).  Negative z uses rho(q, -z) = conj(rho(-q, z)).
    """
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    if z == 0:
        return np.exp(1j * np.pi * q) * np.sinc(q)
    if z < 0:
        return np.conj(rho_fresnel(-q, -z))
    a = z / 2.0
    sa = math.sqrt(a)
    b = q - a
    s0, c0 = sps.fresnel(b / sa)
    s1, c1 = sps.fresnel((2 * a + b) / sa)
    return np.exp(-1j * np.pi * b * b / (2 * a)) / (2 * sa) * ((c1 - c0) + 1j * (s1 - s0))


# --------------------------------------------------------------------------
# spectrum
# --------------------------------------------------------------------------
def test_spectrum_matches_brute_force_dft():
    n = 1024
    x = S.white_noise(n, 11)
    k = np.arange(n // 2)[:, None]
    t = np.arange(n)[None, :]
    ref = (x.astype(np.float64)[None, :] * np.exp(-2j * np.pi * k * t / n)).sum(axis=1)
    ref[0] = 0.0
    X = O.spectrum(x)
    assert X.shape == (n // 2,)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_spectrum_parseval():
    n = 1 << 14
    x = S.white_noise(n, 12).astype(np.float64)
    X = O.spectrum(x)
    dc = x.sum()
    nyq = (x * (-1.0) ** np.arange(n)).sum()
    lhs = (x * x).sum()
    rhs = (dc * dc + 2 * np.sum(np.abs(X[1:]) ** 2) + nyq * nyq) / n
    assert abs(lhs - rhs) <= 1e-12 * lhs


def test_spectrum_sign_convention_pure_tone():
    n, k0 = 4096, 37
    x = np.sin(2 * np.pi * k0 * np.arange(n) / n)
    X = O.spectrum(x)
    # forward DFT with exp(-2 pi i k n/N): sin -> -i N/2 at k0
    assert abs(X[k0] - (-0.5j * n)) < 1e-9 * n
    X[k0] = 0
    assert np.max(np.abs(X)) < 1e-9 * n


# --------------------------------------------------------------------------
# normalisation
# --------------------------------------------------------------------------
def test_block_medians_even_and_odd_counts():
    B = 16
    rng = np.random.default_rng(5)
    p = np.empty(4 * B)
    p[0] = 1e9                                  # k = 0 is skipped
    p[1:B] = rng.permutation(np.arange(1, B))  # 15 values: median = 8
    for b in range(1, 4):
        p[b * B:(b + 1) * B] = rng.permutation(np.arange(1, B + 1)) * b  # even
    X = np.sqrt(p).astype(np.complex128)
    meds = O.block_medians(X, B)
    assert abs(meds[0] - B / 2) < 1e-12 * B
    for b in range(1, 4):
        # mean of the two middle values
        assert abs(meds[b] - b * (B + 1) / 2) < 1e-12 * B * b


def test_normalised_noise_is_unit_exponential():
    x = S.white_noise(1 << 18, 13)
    Xn, _ = O.normalise(O.spectrum(x), 2048)
    p = np.abs(Xn[1:]) ** 2
    # Exp(1): mean 1, median ln 2
    assert abs(p.mean() - 1.0) < 0.01
    assert abs(np.median(p) - math.log(2)) < 0.01


def test_normalise_none_is_identity():
    X = O.spectrum(S.white_noise(4096, 3))
    Xn, meds = O.normalise(X, 2048, "none")
    assert meds is None and np.array_equal(Xn, X)


# --------------------------------------------------------------------------
# templates
# --------------------------------------------------------------------------
def test_rho_zero_z_is_fourier_interpolation_kernel():
    q = np.array([-7.3, -2.5, -0.25, 0.0, 0.1, 0.5, 3.7, 11.0])
    ref = np.exp(1j * np.pi * q) * np.sinc(q)
    assert np.max(np.abs(O.rho(q, 0.0) - ref)) < 1e-13
    e = np.arange(-20, 21)
    d = O.rho(e, 0.0)
    assert abs(d[20] - 1) < 1e-14 and np.max(np.abs(np.delete(d, 20))) < 1e-13


@pytest.mark.parametrize("z", [0.5, 1.0, 7.5, -3.0, 16.0, -48.0, 96.0, -96.0])
def test_rho_quadrature_matches_fresnel_route(z):
    m = 8 + math.ceil(abs(z) / 2)
    q = np.concatenate([np.arange(-m, m + 1), [0.3, -5.7, 2.5]])
    a = O.rho(q, z)
    b = rho_fresnel(q, z)
    assert np.max(np.abs(a - b)) < 1e-12


def test_rho_conjugate_symmetry():
    q = np.linspace(-30, 30, 61) + 0.17
    for z in (3.0, 40.0, 95.0):
        assert np.max(np.abs(O.rho(q, -z) - np.conj(O.rho(-q, z)))) < 1e-13


def test_rho_window_energy_approaches_one():
    # sum over integer shifts of |rho(q+e, z)|^2 = 1 (Parseval for the
    # unit-modulus signal on [0,1)); the truncated sum grows towards 1.
    z, q = 20.0, 0.3
    prev = 0.0
    for M in (10, 40, 160):
        e = np.arange(-M, M + 1)
        s = np.sum(np.abs(rho_fresnel(q + e, z)) ** 2)
        o = np.sum(np.abs(O.rho(q + e, z)) ** 2)
        assert abs(s - o) < 1e-12
        assert prev < o < 1.0
        prev = o
    assert 1.0 - prev < 5e-3


def test_template_bank_geometry_and_energy():
    g = O.geometry(1 << 17, 16.0, 2.0, 4)
    assert g.n_z == 17 and g.iz0 == 8
    assert list(g.m) == [8 + math.ceil(abs(z) / 2) for z in g.z]
    assert g.m_max == 16
    bank = O.template_bank(g)
    assert abs(bank.energy[g.iz0] - 1.0) < 1e-13
    for iz, t in enumerate(bank.taps):
        assert t.shape[0] == 2 * g.m[iz] + 1
        assert abs(np.sum(np.abs(t) ** 2) - 1.0) < 1e-12
        # taps are conj(rho(e,z))/sqrt(E): compare with the Fresnel route
        e = np.arange(-g.m[iz], g.m[iz] + 1)
        ref = np.conj(rho_fresnel(e, g.z[iz])) / math.sqrt(bank.energy[iz])
        assert np.max(np.abs(t - ref)) < 1e-12


def test_paper_workload_geometry():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        pw = json.load(f)["ska_like_workload"]
    g = O.geometry(1 << 23, 96.0, 1.0, 16)
    assert g.n_z == pw["acceleration_trials"]
    # 600 s at 64 us is 9.375e6 samples; the power-of-two length used is 2^23
    n_paper = pw["t_obs_s"] / (pw["tsamp_us"] * 1e-6)
    assert (1 << 23) <= n_paper < (1 << 24)


# --------------------------------------------------------------------------
# correlation (power plane)
# --------------------------------------------------------------------------
def _small_geom():
    return O.geometry(1 << 12, 16.0, 2.0, 4)


def test_zero_z_row_is_normalised_power_spectrum():
    g = _small_geom()
    x = S.white_noise(g.n_samples, 21)
    Xn, _ = O.normalise(O.spectrum(x), 512)
    P = O.power_plane(Xn, O.template_bank(g))
    assert np.max(np.abs(P[g.iz0] - np.abs(Xn) ** 2)) < 1e-12 * np.max(P[g.iz0])


@pytest.mark.parametrize("r0,z0", [(700, 6.0), (1500, -14.0), (20, 16.0), (2030, -2.0)])
def test_fourier_domain_injection_peak_closed_form(r0, z0):
    """X_k = c rho(r0 - k, z0): the plane peaks at (r0, z0) with P = |c|^2 E_z0."""
    g = _small_geom()
    k = np.arange(g.n_r)
    c = 3.0 - 4.0j
    X = c * rho_fresnel(r0 - k, z0)
    X[0] = 0.0
    P = O.power_plane(X, O.template_bank(g))
    iz = int(round(z0 / g.z_step)) + g.iz0
    m = g.m[iz]
    e = np.arange(-m, m + 1)
    Ez = np.sum(np.abs(rho_fresnel(e, z0)) ** 2)
    assert abs(P[iz, r0] - abs(c) ** 2 * Ez) < 1e-10 * abs(c) ** 2
    assert np.unravel_index(np.argmax(P), P.shape) == (iz, r0)


def test_time_domain_chirp_matches_closed_form():
    """A noise-free accelerated sinusoid gives X_k ~ (aN/2) e^{i pi z/4} rho(r-k, z)."""
    n, r_bar, z0, a = 1 << 14, 1234.3, 7.5, 0.05
    g = O.geometry(n, 16.0, 2.0, 4)
    x = S.inject_sinusoid(np.zeros(n, np.float32), r_bar, z0, a).astype(np.float64)
    # inject in FP64 to keep the float32 rounding out of the comparison
    u = np.arange(n) / n
    x = a * np.cos(2 * np.pi * (r_bar * u + z0 * (u - 0.5) ** 2 / 2))
    bank = O.template_bank(g)
    P = O.power_plane(O.spectrum(x), bank)
    peak = np.unravel_index(np.argmax(P), P.shape)
    # closed form at every cell of a 5 x 7 neighbourhood
    best, best_cell = -1.0, None
    for iz in range(g.n_z):
        m = g.m[iz]
        e = np.arange(-m, m + 1)
        for r in range(1228, 1241):
            F = (a * n / 2) * np.sum(rho_fresnel(r_bar - r + e, z0)
                                     * np.conj(rho_fresnel(e, g.z[iz]))) / math.sqrt(bank.energy[iz])
            ref = abs(F) ** 2
            if abs(iz - peak[0]) <= 2 and abs(r - peak[1]) <= 3:
                assert abs(P[iz, r] - ref) <= 2e-3 * P[peak] , (iz, r)
            if ref > best:
                best, best_cell = ref, (iz, r)
    assert best_cell == peak
    assert abs(P[peak] - best) < 1e-3 * best


def test_plane_stats_are_mean_and_population_std():
    P = np.arange(12, dtype=np.float64).reshape(3, 4)
    m, s = O.plane_stats(P)
    assert m == 5.5 and abs(s - math.sqrt(143 / 12)) < 1e-14


# --------------------------------------------------------------------------
# harmonic sum
# --------------------------------------------------------------------------
def test_harmonic_index_rounding_reading():
    # round half up in r, half away from zero in the z offset, top index kept
    assert O.harmonic_indices(8, 8, 8, 16, 1) == (8, 1)
    assert O.harmonic_indices(7, 8, 8, 16, 1) == (8, 0)
    assert O.harmonic_indices(9, 8, 8, 16, 1) == (8, 1)
    assert O.harmonic_indices(24, 0, 8, 16, 1) == (7, 2)   # o=-8 -> -1; 24/16=1.5 -> 2
    assert O.harmonic_indices(100, 3, 8, 16, 16) == (3, 100)
    for ir in range(50):
        for iz in range(17):
            assert O.harmonic_indices(ir, iz, 8, 4, 4) == (iz, ir)


def test_harmonic_stage_one_is_the_plane_and_constant_plane():
    g = O.geometry(256, 8.0, 1.0, 16)
    rng = np.random.default_rng(0)
    P = rng.random((g.n_z, g.n_r))
    Sp = O.harmonic_planes(P, g)
    assert np.array_equal(Sp[0], P)
    Sc = O.harmonic_planes(np.full((g.n_z, g.n_r), 2.5), g)
    for st, h in enumerate(g.stages):
        assert np.all(Sc[st] == 2.5 * h)


@pytest.mark.parametrize("of", [3, -2, 0])
def test_harmonic_sum_spike_train(of):
    """Spikes v_j = 2^j at harmonic j of a fundamental; S_h at the top cell
    must be exactly the binary sum of the harmonics that stage h reads."""
    H = 16
    g = O.geometry(4096, 48.0, 1.0, H)
    rf = 97
    P = np.zeros((g.n_z, g.n_r))
    for j in range(1, H + 1):
        P[g.iz0 + j * of, j * rf] += 2.0 ** j
    top = (g.iz0 + H * of, H * rf)
    Sp = O.harmonic_planes(P, g)
    for st, h in enumerate(g.stages):
        want = sum(2.0 ** (k * H // h) for k in range(1, h + 1))
        assert Sp[st][top] == want, (h, Sp[st][top], want)


def test_harmonic_sum_brute_force_small():
    g = O.geometry(128, 4.0, 1.0, 8)
    rng = np.random.default_rng(1)
    P = rng.random((g.n_z, g.n_r))
    Sp = O.harmonic_planes(P, g)
    for st, h in enumerate(g.stages):
        for iz in range(g.n_z):
            for ir in range(g.n_r):
                s = 0.0
                for k in range(1, h + 1):
                    j = k * (g.n_harm // h)
                    siz, sir = O.harmonic_indices(ir, iz, g.iz0, g.n_harm, j)
                    s += P[siz, sir]
                assert abs(Sp[st, iz, ir] - s) < 1e-12


# --------------------------------------------------------------------------
# fundamental-indexed harmonic sum (variant)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("H", [1, 2, 4, 8, 16])
def test_fundamental_sums_equal_top_harmonic_sums_at_multiple_cells(H):
    """At a top cell whose offsets are h times a fundamental's, top-harmonic
    stage h reads harmonics j = k H/h at (k o_f, k r_f) with no rounding: the
    same cells the fundamental-indexed stage h sums.  Pins the variant to the
    independently written top-harmonic oracle."""
    g = O.geometry(2048, 40.0, 1.0, H)
    rng = np.random.default_rng(H)
    P = rng.random((g.n_z, g.n_r))
    top = O.harmonic_planes(P, g)
    fund = O.fund_planes(P, g)
    n = 0
    for st, h in enumerate(g.stages):
        for o in range(-(g.iz0 // h), g.iz0 // h + 1):
            for rf in range(0, (g.n_r - 1) // h + 1, 7):
                assert fund[st, g.iz0 + o, rf] == top[st, g.iz0 + h * o, h * rf]
                n += 1
    assert n > 100


@pytest.mark.parametrize("H", [2, 8, 16])
def test_fundamental_domain_size_closed_form(H):
    """Stage h is defined on ceil(N_r / h) bins x (2 floor(K / h) + 1) rows;
    outside it the sums are 0 and no cell is ever a candidate."""
    g = O.geometry(1024, 20.0, 1.0, H)
    P = np.ones((g.n_z, g.n_r))
    S = O.fund_planes(P, g)
    for st, h in enumerate(g.stages):
        inside = S[st] > 0
        assert inside.sum() == -(-g.n_r // h) * (2 * (g.iz0 // h) + 1)
        assert np.all(S[st][inside] == h)          # constant plane: S_h = h
    # candidates (a low threshold, so there are many) lie in their stage's
    # domain and carry the stage sum
    R = np.random.default_rng(H).exponential(size=(g.n_z, g.n_r))
    SR = O.fund_planes(R, g)
    m, sd = O.plane_stats(R)
    c, _ = O.candidates(R, g, m, sd, sigma=1.0, harmonic_mode=O.FUNDAMENTAL)
    assert len(c) > 1000
    for rec in c[::37]:
        h = int(rec["harm"])
        st = g.stages.index(h)
        assert O.fund_domain(g, h, int(rec["iz"]), int(rec["ir"]))
        assert rec["power"] == SR[st, rec["iz"], rec["ir"]]


@pytest.mark.parametrize("of", [3, -2, 0])
def test_fundamental_sum_spike_train(of):
    """Spikes 2^k at the exact multiples (k o_f, k r_f): stage h at the
    fundamental is 2^1 + ... + 2^h, and stage 1 is the plane."""
    H = 16
    g = O.geometry(4096, 48.0, 1.0, H)
    rf = 97
    P = np.zeros((g.n_z, g.n_r))
    for k in range(1, H + 1):
        P[g.iz0 + k * of, k * rf] += 2.0 ** k
    S = O.fund_planes(P, g)
    assert np.array_equal(S[0], P)
    for st, h in enumerate(g.stages):
        assert S[st][g.iz0 + of, rf] == sum(2.0 ** k for k in range(1, h + 1))


# --------------------------------------------------------------------------
# thresholds
# --------------------------------------------------------------------------
def test_gamma_tail_factors_closed_form():
    p = 0.5 * math.erfc(6 / math.sqrt(2))
    G = O.gamma_tail_factors(16, 6.0)
    assert abs(G[0] - (-math.log(p))) < 1e-10          # Q(1, x) = e^-x
    for h, x in zip([1, 2, 4, 8, 16], G):
        q = math.exp(-x) * sum(x ** k / math.factorial(k) for k in range(h))
        assert abs(q - p) < 1e-9 * p


def test_log_gamma_tail_matches_scipy_and_sigma_is_six_at_threshold():
    for h in (1, 2, 4, 8, 16, 32):
        for x in (0.5, 3.0, 20.0, 60.0):
            assert abs(O.log_gamma_tail(h, x) - math.log(sps.gammaincc(h, x))) < 1e-9
    G = O.gamma_tail_factors(16, 6.0)
    for h, x in zip([1, 2, 4, 8, 16], G):
        assert abs(O.sigma_equiv(x * 1.7, h, 1.7, 1.0, O.GAMMA_TAIL) - 6.0) < 1e-8


def test_mean_plus_ksigma_threshold():
    T = O.thresholds(4, 6.0, O.MEAN_PLUS_KSIGMA, 1.1, 0.9)
    assert np.allclose(T, [1.1 + 6 * 0.9, 2.2 + 6 * math.sqrt(2) * 0.9, 4.4 + 12 * 0.9])


# --------------------------------------------------------------------------
# interbinning (half-bin grid from the complex correlation)
# --------------------------------------------------------------------------
def _rho0(q):
    """rho(q, 0) = (exp(2 pi i q) - 1) / (2 pi i q), rho(0, 0) = 1."""
    q = np.asarray(q, dtype=np.float64)
    out = np.ones(q.shape, dtype=np.complex128)
    nz = q != 0
    out[nz] = (np.exp(2j * np.pi * q[nz]) - 1.0) / (2j * np.pi * q[nz])
    return out


def test_cell_powers_and_correlations_equal_the_plane_and_a_direct_sum():
    """The one-cell routes the full-size tests check the GPU with: P at random
    cells (every z, both edges of the spectrum) equals the whole-plane direct
    correlation at those cells and a plain numpy sum written out here from
    the definition F(r, z) = sum_e X'_{r-e} g_z[e] (X'_k = 0 outside
    [0, N_r)), so an iz/r swap, a dtype slip or a tap offset in their
    marshalling fails."""
    g = O.geometry(1 << 12, 10.0, 1.0, 4)
    Xn, _ = O.normalise(O.spectrum(S.white_noise(g.n_samples, 21)), 512)
    bank = O.template_bank(g)
    P = O.power_plane(Xn, bank)
    F = O.correlation_plane(Xn, bank)
    rng = np.random.default_rng(5)
    iz = rng.integers(0, g.n_z, 400)
    r = rng.integers(0, g.n_r, 400)
    iz[:g.n_z] = np.arange(g.n_z)          # every template at least once
    r[:4] = [0, 1, g.n_r - 2, g.n_r - 1]   # windows cut by both edges
    v = O.cell_powers(Xn, bank, iz, r)
    assert np.max(np.abs(v - P[iz, r]) / np.maximum(P[iz, r], 1e-3)) < 1e-12
    c = O.cell_correlations(Xn, bank, iz, r)
    assert np.max(np.abs(c - F[iz, r])) < 1e-12 * max(1.0, np.max(np.abs(F)))
    for c in range(60):
        a, b = int(iz[c]), int(r[c])
        m = int(g.m[a])
        s = 0j
        for e in range(-m, m + 1):
            if 0 <= b - e < g.n_r:
                s += Xn[b - e] * bank.taps[a][e + m]
        assert abs(abs(s) ** 2 - v[c]) < 1e-11 * max(1.0, abs(s) ** 2)


def test_harmonic_at_equals_the_stage_planes_and_brute_force():
    """The per-cell harmonic sums used by the full-size checks: every stage at
    random cells (both z edges, r edges) equals the whole-plane sums and a
    sum over harmonic_indices written out here."""
    g = O.geometry(1 << 11, 12.0, 1.0, 16)
    rng = np.random.default_rng(8)
    P = rng.exponential(size=(g.n_z, g.n_r))
    Sp = O.harmonic_planes(P, g)
    n = 500
    st = rng.integers(0, len(g.stages), n)
    iz = rng.integers(0, g.n_z, n)
    ir = rng.integers(0, g.n_r, n)
    iz[:4] = [0, g.n_z - 1, g.iz0, g.iz0 - 1]
    ir[:4] = [g.n_r - 1, 0, g.n_r - 1, 1]
    st[:4] = len(g.stages) - 1
    v = O.harmonic_at(P, g, st, iz, ir)
    assert np.max(np.abs(v - Sp[st, iz, ir])) < 1e-12 * np.max(Sp)
    for c in range(100):
        h = g.stages[st[c]]
        s = 0.0
        for k in range(1, h + 1):
            siz, sir = O.harmonic_indices(int(ir[c]), int(iz[c]), g.iz0, g.n_harm,
                                          k * (g.n_harm // h))
            s += P[siz, sir]
        assert abs(v[c] - s) < 1e-12 * s


def test_correlation_plane_squared_is_the_power_plane():
    g = _small_geom()
    Xn, _ = O.normalise(O.spectrum(S.white_noise(g.n_samples, 5)), 512)
    bank = O.template_bank(g)
    F = O.correlation_plane(Xn, bank)
    P = O.power_plane(Xn, bank)
    assert F.shape == P.shape
    assert np.max(np.abs(np.abs(F) ** 2 - P)) < 1e-12 * np.max(P)


def test_interbin_brute_force_small():
    rng = np.random.default_rng(3)
    F = rng.standard_normal((3, 7)) + 1j * rng.standard_normal((3, 7))
    P = O.interbin_plane(F)
    assert P.shape == (3, 14)
    for iz in range(3):
        for c in range(14):
            r = c // 2
            if c % 2 == 0:
                ref = abs(F[iz, r]) ** 2
            else:
                nxt = F[iz, r + 1] if r + 1 < 7 else 0.0
                ref = (math.pi / 4) ** 2 * abs(F[iz, r] - nxt) ** 2
            assert abs(P[iz, c] - ref) <= 1e-14 * max(1.0, ref)


@pytest.mark.parametrize("k0", [100, 777, 2046])
def test_interbin_half_bin_tone_closed_form(k0):
    """X_k = c rho(k0 + 1/2 - k, 0): the half-bin column 2 k0 + 1 recovers |c|^2
    exactly (the z = 0 template is the unit impulse), while the two bins read
    only (2/pi)^2 |c|^2."""
    g = O.geometry(1 << 12, 0.0, 1.0, 1)
    k = np.arange(g.n_r)
    c = 1.5 - 2.0j
    X = c * _rho0(k0 + 0.5 - k)
    P = O.interbin_plane(O.correlation_plane(X, O.template_bank(g)))
    assert abs(P[0, 2 * k0 + 1] - abs(c) ** 2) < 1e-10 * abs(c) ** 2
    for b in (k0, k0 + 1):
        assert abs(P[0, 2 * b] - (2 / math.pi) ** 2 * abs(c) ** 2) < 1e-10 * abs(c) ** 2
    assert int(np.argmax(P[0])) == 2 * k0 + 1


def test_interbin_integer_tone_neighbours_and_last_column():
    """A tone on bin k0: the half bins on either side read (pi/4)^2 |c|^2
    (rho(+-1, 0) = 0); the last column uses F(N_r) = 0."""
    g = O.geometry(1 << 11, 0.0, 1.0, 1)
    k = np.arange(g.n_r)
    k0 = 300
    c = 2.0 + 0.5j
    X = c * _rho0(k0 - k)
    F = O.correlation_plane(X, O.template_bank(g))
    P = O.interbin_plane(F)
    want = (math.pi / 4) ** 2 * abs(c) ** 2
    assert abs(P[0, 2 * k0 + 1] - want) < 1e-10 * want
    assert abs(P[0, 2 * k0 - 1] - want) < 1e-10 * want
    assert abs(P[0, 2 * k0] - abs(c) ** 2) < 1e-10 * abs(c) ** 2
    assert P[0, -1] == pytest.approx((math.pi / 4) ** 2 * abs(F[0, -1]) ** 2, rel=1e-14)


def test_half_bin_cells_one_by_one_equal_the_plane():
    g = O.geometry(1 << 12, 8.0, 2.0, 4)
    Xn, _ = O.normalise(O.spectrum(S.white_noise(g.n_samples, 3)), 512)
    bank = O.template_bank(g)
    P = O.interbin_plane(O.correlation_plane(Xn, bank))
    rng = np.random.default_rng(1)
    iz = rng.integers(0, g.n_z, 300)
    col = rng.integers(0, 2 * g.n_r, 300)
    col[:5] = 2 * g.n_r - 1                       # the last half bin reads F(N_r) = 0
    v = O.half_bin_cells(Xn, bank, iz, col)
    assert np.max(np.abs(v - P[iz, col]) / np.maximum(P[iz, col], 1e-3)) < 1e-12


def test_interbin_search_recovers_half_bin_sinusoid():
    """A time-domain sinusoid half-way between bins loses (2/pi)^2 of its power
    on the integer grid; the interbinned plane recovers most of it at the
    half-bin column (up to the truncation of the half-bin estimate)."""
    n, a = 1 << 14, 0.05
    u = np.arange(n) / n
    r_bar = 1234.5
    x = a * np.cos(2 * np.pi * r_bar * u)
    full = (a * n / 2) ** 2
    plain = O.search(x, 4.0, 2.0, 1, norm="none")
    ib = O.search(x, 4.0, 2.0, 1, norm="none", interbin=True)
    g = plain["geom"]
    assert ib["P"].shape == (g.n_z, 2 * g.n_r)
    assert np.allclose(ib["P"][:, 0::2], plain["P"], rtol=1e-12, atol=0.0)
    best_plain = plain["P"][g.iz0].max()
    assert abs(best_plain / full - (2 / math.pi) ** 2) < 0.01
    assert ib["P"][g.iz0, 2 * 1234 + 1] > 0.95 * full
    assert int(np.argmax(ib["P"][g.iz0])) == 2 * 1234 + 1
    c = ib["candidates"]
    assert np.any((c["ir"] == 2 * 1234 + 1) & (c["iz"] == g.iz0))


# --------------------------------------------------------------------------
# dedispersion (upstream of the search)
# --------------------------------------------------------------------------
def test_dm_delay_textbook_value():
    """DM 100 pc cm^-3 between 1400 and 1200 MHz: 76.44 ms (4.148808 ms x 100 x
    (1/1.2^2 - 1/1.4^2) with frequencies in GHz), 1194 samples of 64 us; the top
    channel has no delay."""
    d = O.dm_delays(2, 1400.0, 200.0, 64e-6, 100.0, 0.0, 1)
    assert d.shape == (1, 2)
    assert d[0, 0] == 0 and d[0, 1] == 1194
    d2 = O.dm_delays(2, 1400.0, 200.0, 1e-6, 100.0, 0.0, 1)
    assert abs(d2[0, 1] * 1e-6 - 0.0764380) < 2e-6


def test_dm_delays_monotone_and_zero_dm():
    d = O.dm_delays(64, 1500.0, 2.0, 64e-6, 0.0, 5.0, 20)
    assert np.all(d[0] == 0)                       # DM 0
    assert np.all(np.diff(d, axis=0) >= 0)         # grows with DM
    assert np.all(np.diff(d, axis=1) >= 0)         # grows down the band
    assert np.all(d[:, 0] == 0)


def test_dedisperse_zero_dm_is_the_channel_sum():
    fb = S.filterbank_noise(16, 300, 4)
    out = O.dedisperse(fb, np.zeros((1, 16), dtype=np.int64), 300)
    assert np.allclose(out[0], fb.astype(np.float64).sum(axis=0), rtol=0, atol=1e-12)


def test_dedisperse_brute_force_small():
    rng = np.random.default_rng(9)
    fb = rng.standard_normal((5, 40))
    delays = rng.integers(0, 12, size=(3, 5))
    out = O.dedisperse(fb, delays, 33)
    for d in range(3):
        for t in range(33):
            ref = sum(fb[c, t + delays[d, c]] if t + delays[d, c] < 40 else 0.0
                      for c in range(5))
            assert abs(out[d, t] - ref) < 1e-12


def test_dedisperse_collapses_a_dispersed_pulse():
    """A unit pulse planted along the delay curve of DM_k lands as one sample of
    height n_chan at DM_k, and lower at every other DM."""
    n_chan, n_t, t0 = 32, 2000, 123
    delays = O.dm_delays(n_chan, 1450.0, 4.0, 256e-6, 0.0, 20.0, 12)
    k = 7
    fb = S.add_at_samples(np.zeros((n_chan, n_t), np.float32), t0 + delays[k], 1.0)
    out = O.dedisperse(fb, delays, 1000)
    assert out[k, t0] == n_chan
    assert np.unravel_index(np.argmax(out), out.shape) == (k, t0)
    others = np.delete(out, k, axis=0)
    assert others.max() < n_chan


def test_dedisperse_counts_zero_past_the_end():
    n_chan, n_t = 8, 100
    delays = np.arange(n_chan, dtype=np.int64)[None, :] * 3    # 0, 3, ..., 21
    out = O.dedisperse(np.ones((n_chan, n_t)), delays, n_t)
    for t in (0, 78, 79, 90, 99):
        assert out[0, t] == sum(1 for c in range(n_chan) if t + 3 * c < n_t)


# --------------------------------------------------------------------------
# whole path on the 2^17-sample workload
# --------------------------------------------------------------------------
def test_sinusoid_workload_detected_at_expected_cell():
    x = S.sinusoid_series()
    r = O.search(x, 16.0, 2.0, 4)
    P, g = r["P"], r["geom"]
    iz, ir = np.unravel_index(np.argmax(P), P.shape)
    assert ir == 5000 and g.z[iz] in (6.0, 8.0)
    c = r["candidates"]
    assert len(c) > 0 and np.all(np.diff(c["harm"]) >= 0)
    assert np.any((c["ir"] == 5000) & (c["harm"] == 1))
    # noise statistics after normalisation: mean near 1
    assert abs(r["mean"] - 1.0) < 0.02


def test_noise_only_false_alarms_are_rare():
    x = S.white_noise(1 << 17, 99)
    r = O.search(x, 16.0, 2.0, 4)
    assert len(r["candidates"]) <= 3


# --------------------------------------------------------------------------
# Fourier-interpolated power (refinement)
# --------------------------------------------------------------------------
def test_fourier_power_integer_r_zero_z_is_the_bin():
    X = O.spectrum(S.white_noise(4096, 8))
    for r in (10, 500, 1999):
        P, F = O.fourier_power(X, float(r), 0.0)
        assert abs(F - X[r]) < 1e-10 * abs(X[r])


@pytest.mark.parametrize("r0,z0", [(1000.37, 12.6), (1500.81, -33.2)])
def test_fourier_power_peak_of_an_injection(r0, z0):
    n_r = 4096
    k = np.arange(n_r)
    c = 2.0 + 1.0j
    X = c * rho_fresnel(r0 - k, z0)
    P, F = O.fourier_power(X, r0, z0)
    w = O.refine_window(r0, z0, n_r)
    E = np.sum(np.abs(rho_fresnel(r0 - w, z0)) ** 2)
    assert abs(F - c * E) < 1e-10 * abs(c)          # F = c sum |rho|^2 on the window
    assert 0.99 < E < 1.0
    for dr, dz in ((0.03, 0), (-0.03, 0), (0, 0.3), (0, -0.3)):
        assert O.fourier_power(X, r0 + dr, z0 + dz)[0] < P


def test_silent_series_gives_no_candidates():
    """An all-zero series: every block median is 0, so every block gets the
    factor 0 (the reading for a block without power); the plane, its
    statistics and both kinds of threshold are 0, nothing crosses, and no NaN
    appears anywhere."""
    x = np.zeros(1 << 12, np.float32)
    for mode in (O.GAMMA_TAIL, O.MEAN_PLUS_KSIGMA):
        r = O.search(x, 4.0, 1.0, 4, mode=mode)
        assert np.all(r["medians"] == 0.0) and np.all(r["Xn"] == 0.0)
        assert np.all(r["P"] == 0.0) and r["mean"] == 0.0 and r["std"] == 0.0
        assert np.all(r["T"] == 0.0) and len(r["candidates"]) == 0

