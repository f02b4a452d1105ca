"""Plain FP64 CPU oracle for the FDAS hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The CUDA library never calls it and it
imports nothing from the product package; the two share only the seeded input
generators in ``synthetic``.

What it computes, in the order of the method (paper §2.1 "FDAS": a matched
filter over a grid of constant-acceleration templates; §2.2: the filter is a
convolution evaluated in the Fourier domain; the rest of the pipeline -- the
normalisation, the harmonic sum and the threshold -- is not spelled out in the
paper and follows the stated readings):

1. ``spectrum``      X_k = sum_n x_n exp(-2 pi i k n / N), k in [0, N/2),
                     with X_0 set to 0 (numpy's FFT is the library step).
2. ``normalise``     per block of B bins, X'_k = X_k sqrt(ln 2 / median|X|^2)
                     (block 0 skips k = 0; even counts take the mean of the two
                     middle values): white noise then has |X'|^2 ~ Exp(1).
3. ``rho``           the response of an accelerated sinusoid,
                     rho(q, z) = int_0^1 exp(2 pi i [(q - z/2) u + z u^2/2]) du,
                     by Gauss-Legendre quadrature (deliberately not the Fresnel
                     closed form the CUDA path uses).
   ``template_bank`` g_z[e] = conj(rho(e, z)) / sqrt(E_z), |e| <= m(z),
                     E_z = sum |rho(e, z)|^2, m(z) = 8 + ceil(|z|/2).
4. ``power_plane``   the DIRECT correlation F(r, z) = sum_e X'_{r-e} g_z[e],
                     P = |F|^2 (C loop in fdas_oracle.c).  Overlap-save is an
                     exact re-arrangement of this sum, which is why the oracle
                     does not use it.
5. ``plane_stats``   mean and population standard deviation of P over the
                     whole n_z x N_r plane.
6. ``harmonic_*``    top-harmonic-indexed sums S_h, h = 1, 2, 4, ..., H
                     (C loop in fdas_oracle.c); ``fund_planes`` the variant
                     labelled by the fundamental, S_h = sum_{k<=h} P at the
                     exact multiples (k o, k ir), in its domain.
7. ``thresholds``    S_h > T_h with T_h = mean * Q^-1(h, Phibar(sigma))
                     (Gamma(h,1) tail at the Gaussian-equivalent false-alarm
                     probability of `sigma`), or T_h = h*mean + sigma*sqrt(h)*std.
8. ``candidates``    every cell above threshold, sorted by (trial, h, iz, ir).
   ``interbin_plane`` (option) the plane on a half-bin grid from the complex
                     correlation F: column 2r holds |F(r)|^2 and column 2r + 1
                     the interbinned power (pi/4)^2 |F(r) - F(r+1)|^2, with
                     F(N_r) = 0 beyond the last bin; stats, harmonic sums and
                     candidates then run on that 2 N_r-column plane.
0. ``dm_delays``     (upstream of the search, optional) incoherent
   ``dedisperse``    dedispersion of a filterbank into DM-trial series:
                     delay of channel c (frequency f_c = f_top - c df, MHz)
                     at DM_d = dm_lo + d dm_step is the cold-plasma delay
                     relative to the top of the band in samples,
                     Delta(c, d) = floor(K_DM DM_d (f_c^-2 - f_top^-2) / tsamp
                     + 1/2), K_DM = 4.148808e3 MHz^2 pc^-1 cm^3 s, and
                     out[d][t] = sum_c in[c][t + Delta(c, d)] (0 past n_t).
9. ``fourier_power`` the off-grid power used to refine candidates:
                     F(r, z) = sum_k X'_k conj(rho(r - k, z)) over the bins
                     within 32 + ceil(|z|/2) of round(r), unnormalised rho,
                     P = |F|^2 (gradients are checked by finite differences
                     of this function in the tests).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.special as sps

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "fdas_oracle.c")

GAMMA_TAIL = 0
MEAN_PLUS_KSIGMA = 1


# --------------------------------------------------------------------------
# C part
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile fdas_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _c():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_plane.argtypes = [P, P, i64, i32, P, P, P, P, P]
        lib.oracle_plane.restype = None
        lib.oracle_corr_plane.argtypes = [P, P, i64, i32, P, P, P, P, P, P]
        lib.oracle_corr_plane.restype = None
        lib.oracle_cells_corr.argtypes = [P, P, i64, P, P, P, P, i64, P, P, P, P]
        lib.oracle_cells_corr.restype = None
        lib.oracle_cells.argtypes = [P, P, i64, P, P, P, P, i64, P, P, P]
        lib.oracle_cells.restype = None
        lib.oracle_harmonic_planes.argtypes = [P, i64, i32, i32, i32, P]
        lib.oracle_harmonic_planes.restype = None
        lib.oracle_harmonic_cells.argtypes = [P, i64, i32, i32, i32, P, i64,
                                              P, P, P, P]
        lib.oracle_harmonic_cells.restype = i64
        lib.oracle_harmonic_at.argtypes = [P, i64, i32, i32, i64, P, P, P, P]
        lib.oracle_harmonic_at.restype = None
        lib.oracle_fund_planes.argtypes = [P, i64, i32, i32, i32, P]
        lib.oracle_fund_planes.restype = None
        lib.oracle_fund_cells.argtypes = [P, i64, i32, i32, i32, P, i64, P, P, P, P]
        lib.oracle_fund_cells.restype = i64
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = i32
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads used by the C loops."""
    return int(_c().oracle_threads())


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# geometry of the search grid
# --------------------------------------------------------------------------
@dataclass
class Geometry:
    n_samples: int
    z_max: float
    z_step: float
    n_harm: int
    n_r: int = field(init=False)
    K: int = field(init=False)          # index of z = 0 (iz0)
    n_z: int = field(init=False)
    z: np.ndarray = field(init=False)
    m: np.ndarray = field(init=False)
    stages: list = field(init=False)

    def __post_init__(self):
        self.n_r = self.n_samples // 2
        ratio = self.z_max / self.z_step
        self.K = int(round(ratio))
        if abs(ratio - self.K) > 1e-9 * max(1.0, ratio):
            raise ValueError("z_max / z_step must be an integer")
        self.n_z = 2 * self.K + 1
        idx = np.arange(self.n_z) - self.K
        self.z = idx * float(self.z_step)
        # m(z) = 8 + ceil(|z|/2), evaluated on the exact grid offset
        self.m = np.array([8 + math.ceil(abs(i) * self.z_step / 2.0 - 1e-9)
                           for i in idx], dtype=np.int32)
        self.stages = [1 << s for s in range(int(math.log2(self.n_harm)) + 1)]

    @property
    def iz0(self) -> int:
        return self.K

    @property
    def m_max(self) -> int:
        return int(self.m.max())


def geometry(n_samples: int, z_max: float, z_step: float, n_harm: int) -> Geometry:
    return Geometry(n_samples, z_max, z_step, n_harm)


# --------------------------------------------------------------------------
# 1-2: spectrum and normalisation
# --------------------------------------------------------------------------
def spectrum(x: np.ndarray) -> np.ndarray:
    """X_k for k in [0, N/2) in FP64; DC removed (X_0 = 0), Nyquist dropped."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    X = np.fft.rfft(x)[: n // 2].astype(np.complex128)
    X[0] = 0.0
    return X


def block_medians(X: np.ndarray, block: int = 2048) -> np.ndarray:
    """median(|X_k|^2) per block of `block` bins (block 0 without k = 0)."""
    p = np.abs(X) ** 2
    b = min(block, p.shape[0])
    nb = p.shape[0] // b
    meds = np.empty(nb)
    for i in range(nb):
        seg = p[i * b:(i + 1) * b]
        if i == 0:
            seg = seg[1:]
        meds[i] = np.median(seg)
    return meds


def normalise(X: np.ndarray, block: int = 2048, mode: str = "median"):
    """Return (X', medians).  Exp(1) noise has median ln 2, hence sqrt(ln2/med).

    A block whose median is 0 (no power at all) gets the factor 0.
    """
    if mode == "none":
        return X.copy(), None
    meds = block_medians(X, block)
    b = min(block, X.shape[0])
    with np.errstate(divide="ignore"):
        f = np.where(meds > 0, np.sqrt(math.log(2.0) / np.where(meds > 0, meds, 1.0)), 0.0)
    return X * np.repeat(f, b), meds


# --------------------------------------------------------------------------
# 3: templates
# --------------------------------------------------------------------------
def rho(q, z: float, n_nodes: int | None = None) -> np.ndarray:
    """rho(q, z) = int_0^1 exp(2 pi i [(q - z/2) u + z u^2 / 2]) du (quadrature).

    Gauss-Legendre on [0, 1] with n >= 4 (|q| + |z|) + 64 nodes: the
    integrand turns through at most |q| + |z|/2 cycles, so this is far past
    convergence in FP64.
    """
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    if n_nodes is None:
        n_nodes = int(4 * (np.max(np.abs(q)) + abs(z))) + 64
    t, w = np.polynomial.legendre.leggauss(n_nodes)
    u = 0.5 * (t + 1.0)
    w = 0.5 * w
    ph = 2.0 * np.pi * ((q[:, None] - z / 2.0) * u[None, :] + z * u[None, :] ** 2 / 2.0)
    return (np.exp(1j * ph) * w[None, :]).sum(axis=1)


@dataclass
class Bank:
    geom: Geometry
    taps: list          # taps[iz][e + m] = g_z[e], complex128
    energy: np.ndarray  # E_z


def template_bank(geom: Geometry) -> Bank:
    taps, energy = [], np.empty(geom.n_z)
    for iz in range(geom.n_z):
        m = int(geom.m[iz])
        e = np.arange(-m, m + 1, dtype=np.float64)
        r = rho(e, float(geom.z[iz]))
        E = float(np.sum(np.abs(r) ** 2))
        energy[iz] = E
        taps.append(np.conj(r) / math.sqrt(E))
    return Bank(geom, taps, energy)


def _flat_taps(bank: Bank):
    offs = np.zeros(bank.geom.n_z, dtype=np.int64)
    acc = 0
    for i, t in enumerate(bank.taps):
        offs[i] = acc
        acc += t.shape[0]
    flat = np.concatenate(bank.taps)
    return (np.ascontiguousarray(flat.real), np.ascontiguousarray(flat.imag),
            offs, np.ascontiguousarray(bank.geom.m.astype(np.int32)))


# --------------------------------------------------------------------------
# 4: direct correlation
# --------------------------------------------------------------------------
def power_plane(Xn: np.ndarray, bank: Bank) -> np.ndarray:
    """P[iz][r] = |sum_e X'_{r-e} g_z[e]|^2 over the whole plane (FP64)."""
    n_r = Xn.shape[0]
    xr = np.ascontiguousarray(Xn.real)
    xi = np.ascontiguousarray(Xn.imag)
    gr, gi, offs, m = _flat_taps(bank)
    P = np.empty((bank.geom.n_z, n_r), dtype=np.float64)
    _c().oracle_plane(_ptr(xr), _ptr(xi), n_r, bank.geom.n_z, _ptr(m),
                      _ptr(offs), _ptr(gr), _ptr(gi), _ptr(P))
    return P


def correlation_plane(Xn: np.ndarray, bank: Bank) -> np.ndarray:
    """F[iz][r] = sum_e X'_{r-e} g_z[e] over the whole plane (complex, FP64)."""
    n_r = Xn.shape[0]
    xr = np.ascontiguousarray(Xn.real)
    xi = np.ascontiguousarray(Xn.imag)
    gr, gi, offs, m = _flat_taps(bank)
    Fr = np.empty((bank.geom.n_z, n_r), dtype=np.float64)
    Fi = np.empty((bank.geom.n_z, n_r), dtype=np.float64)
    _c().oracle_corr_plane(_ptr(xr), _ptr(xi), n_r, bank.geom.n_z, _ptr(m),
                           _ptr(offs), _ptr(gr), _ptr(gi), _ptr(Fr), _ptr(Fi))
    return Fr + 1j * Fi


# Interbinning: the response half-way between two bins estimated from the
# complex values at the two bins.  For a sinusoid exactly between bins k and
# k + 1 (rho(1/2, 0) = 2i/pi, rho(-1/2, 0) = -2i/pi) the difference
# F(k) - F(k+1) is 4/pi times the full response, hence the factor pi/4 on the
# amplitude, (pi/4)^2 on the power.
INTERBIN_POWER = (math.pi / 4.0) ** 2


def interbin_plane(F: np.ndarray) -> np.ndarray:
    """P[iz][c] on the half-bin grid c = 0 .. 2 N_r - 1 (r = c / 2):
    P[iz][2r] = |F(r)|^2, P[iz][2r+1] = (pi/4)^2 |F(r) - F(r+1)|^2, F(N_r) = 0."""
    n_z, n_r = F.shape
    Fnext = np.zeros_like(F)
    Fnext[:, :-1] = F[:, 1:]
    P = np.empty((n_z, 2 * n_r), dtype=np.float64)
    P[:, 0::2] = np.abs(F) ** 2
    P[:, 1::2] = INTERBIN_POWER * np.abs(F - Fnext) ** 2
    return P


def cell_powers(Xn: np.ndarray, bank: Bank, iz, r) -> np.ndarray:
    """P at the cells (iz[c], r[c]) by the same direct sum."""
    iz = np.ascontiguousarray(np.asarray(iz, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.int64))
    xr = np.ascontiguousarray(Xn.real)
    xi = np.ascontiguousarray(Xn.imag)
    gr, gi, offs, m = _flat_taps(bank)
    out = np.empty(iz.shape[0], dtype=np.float64)
    _c().oracle_cells(_ptr(xr), _ptr(xi), Xn.shape[0], _ptr(m), _ptr(offs),
                      _ptr(gr), _ptr(gi), iz.shape[0], _ptr(iz), _ptr(r),
                      _ptr(out))
    return out


def cell_correlations(Xn: np.ndarray, bank: Bank, iz, r) -> np.ndarray:
    """Complex F at the cells (iz[c], r[c]) by the direct sum; F = 0 for
    r >= N_r (past the last bin, as interbinning reads it)."""
    iz = np.ascontiguousarray(np.asarray(iz, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.int64))
    xr = np.ascontiguousarray(Xn.real)
    xi = np.ascontiguousarray(Xn.imag)
    gr, gi, offs, m = _flat_taps(bank)
    re = np.empty(iz.shape[0], dtype=np.float64)
    im = np.empty(iz.shape[0], dtype=np.float64)
    _c().oracle_cells_corr(_ptr(xr), _ptr(xi), Xn.shape[0], _ptr(m), _ptr(offs), _ptr(gr),
                           _ptr(gi), iz.shape[0], _ptr(iz), _ptr(r), _ptr(re), _ptr(im))
    F = re + 1j * im
    F[r >= Xn.shape[0]] = 0.0
    return F


def half_bin_cells(Xn: np.ndarray, bank: Bank, iz, col) -> np.ndarray:
    """Cells (iz[c], col[c]) of the half-bin plane (interbin_plane) one by one."""
    iz = np.asarray(iz, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    r = col // 2
    F0 = cell_correlations(Xn, bank, iz, r)
    F1 = cell_correlations(Xn, bank, iz, r + 1)
    return np.where(col % 2 == 0, np.abs(F0) ** 2, INTERBIN_POWER * np.abs(F0 - F1) ** 2)


def plane_stats(P: np.ndarray):
    """(mean, population std) of the plane in FP64."""
    return float(P.mean(dtype=np.float64)), float(P.std(dtype=np.float64))


# --------------------------------------------------------------------------
# 6: harmonic sum
# --------------------------------------------------------------------------
def harmonic_indices(ir: int, iz: int, iz0: int, H: int, j: int):
    """(source iz, source ir) that harmonic j of H reads for the cell (ir, iz)."""
    o = iz - iz0
    a = abs(o)
    oj = (a * j + H // 2) // H
    return iz0 + (-oj if o < 0 else oj), (ir * j + H // 2) // H


def harmonic_planes(P: np.ndarray, geom: Geometry) -> np.ndarray:
    """S[st][iz][ir] for every stage h = 2^st <= H."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    S = np.empty((len(geom.stages),) + P.shape, dtype=np.float64)
    _c().oracle_harmonic_planes(_ptr(P), P.shape[1], P.shape[0], geom.iz0,
                                geom.n_harm, _ptr(S))
    return S


# fundamental-indexed variant: the candidate is labelled by its fundamental
# (iz, ir) and harmonic k reads the exact multiple (iz0 + k o, k ir); stage h
# is defined where every k <= h lies inside the plane (h ir <= N_r - 1 and
# |h o| <= K)
TOP_HARMONIC, FUNDAMENTAL = 0, 1


def fund_domain(geom: Geometry, h: int, iz: int, ir: int) -> bool:
    o = iz - geom.iz0
    return ir * h <= geom.n_r - 1 and 0 <= geom.iz0 + h * o < geom.n_z


def fund_planes(P: np.ndarray, geom: Geometry) -> np.ndarray:
    """S[st][iz][ir] = sum_{k<=h} P[iz0 + k o][k ir] in the stage's domain, 0
    outside it, for every stage h = 2^st <= H."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    S = np.empty((len(geom.stages),) + P.shape, dtype=np.float64)
    _c().oracle_fund_planes(_ptr(P), P.shape[1], P.shape[0], geom.iz0, geom.n_harm, _ptr(S))
    return S


def harmonic_at(P: np.ndarray, geom: Geometry, st, iz, ir) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    st = np.ascontiguousarray(np.asarray(st, dtype=np.int32))
    iz = np.ascontiguousarray(np.asarray(iz, dtype=np.int32))
    ir = np.ascontiguousarray(np.asarray(ir, dtype=np.int64))
    out = np.empty(st.shape[0])
    _c().oracle_harmonic_at(_ptr(P), P.shape[1], geom.iz0, geom.n_harm,
                            st.shape[0], _ptr(st), _ptr(iz), _ptr(ir), _ptr(out))
    return out


# --------------------------------------------------------------------------
# 7: thresholds
# --------------------------------------------------------------------------
def false_alarm_prob(sigma: float) -> float:
    """Gaussian upper tail Phibar(sigma)."""
    return float(0.5 * sps.erfc(sigma / math.sqrt(2.0)))


def gamma_tail_factors(H: int, sigma: float) -> np.ndarray:
    """G_h = Q^-1(h, Phibar(sigma)) for h = 1, 2, 4, ..., H (scipy)."""
    p = false_alarm_prob(sigma)
    return np.array([sps.gammainccinv(h, p) for h in _stages(H)])


def _stages(H: int):
    return [1 << s for s in range(int(math.log2(H)) + 1)]


def thresholds(H: int, sigma: float, mode: int, mean: float, std: float) -> np.ndarray:
    hs = np.array(_stages(H), dtype=np.float64)
    if mode == GAMMA_TAIL:
        return mean * gamma_tail_factors(H, sigma)
    return hs * mean + sigma * np.sqrt(hs) * std


def log_gamma_tail(h: int, x: float) -> float:
    """log Q(h, x) for integer h: Q = exp(-x) sum_{k<h} x^k / k! (Poisson)."""
    if x <= 0:
        return 0.0
    k = np.arange(h, dtype=np.float64)
    lt = k * math.log(x) - sps.gammaln(k + 1.0)
    mx = lt.max()
    return -x + mx + math.log(np.exp(lt - mx).sum())


def sigma_equiv(S: float, h: int, mean: float, std: float, mode: int) -> float:
    """Gaussian-equivalent significance of a harmonic sum S at stage h."""
    if mode == GAMMA_TAIL:
        return float(-sps.ndtri_exp(log_gamma_tail(h, S / mean)))
    return float((S - h * mean) / (math.sqrt(h) * std))


# --------------------------------------------------------------------------
# 8: candidates
# --------------------------------------------------------------------------
CAND_DTYPE = np.dtype([("trial", np.uint32), ("harm", np.int32), ("iz", np.int32),
                       ("ir", np.int64), ("power", np.float64), ("sigma", np.float64)])


def candidates(P: np.ndarray, geom: Geometry, mean: float, std: float,
               sigma: float = 6.0, mode: int = GAMMA_TAIL, trial: int = 0,
               guard: float = 0.0, cap: int = 1 << 22, harmonic_mode: int = TOP_HARMONIC):
    """(candidates, guard_cells).

    candidates: every (h, iz, ir) with S_h > T_h, sorted by (trial, h, iz, ir)
    (top-harmonic sums, or fundamental-indexed sums in their domain).
    guard_cells: the cells with |S_h - T_h| <= guard * T_h (same dtype),
    where a rounding difference may flip the decision.
    """
    P = np.ascontiguousarray(P, dtype=np.float64)
    T = thresholds(geom.n_harm, sigma, mode, mean, std)
    lo = np.ascontiguousarray(T * (1.0 - guard))
    out_st = np.empty(cap, dtype=np.int32)
    out_iz = np.empty(cap, dtype=np.int32)
    out_ir = np.empty(cap, dtype=np.int64)
    out_s = np.empty(cap, dtype=np.float64)
    cells = _c().oracle_fund_cells if harmonic_mode == FUNDAMENTAL else _c().oracle_harmonic_cells
    n = cells(_ptr(P), P.shape[1], P.shape[0], geom.iz0, geom.n_harm, _ptr(lo), cap,
              _ptr(out_st), _ptr(out_iz), _ptr(out_ir), _ptr(out_s))
    if n > cap:
        raise RuntimeError(f"oracle candidate buffer too small ({n} > {cap})")
    st, iz, ir, s = out_st[:n], out_iz[:n], out_ir[:n], out_s[:n]
    rec = np.empty(n, dtype=CAND_DTYPE)
    rec["trial"] = trial
    rec["harm"] = np.left_shift(1, st)
    rec["iz"] = iz
    rec["ir"] = ir
    rec["power"] = s
    rec["sigma"] = [sigma_equiv(float(v), int(h), mean, std, mode)
                    for v, h in zip(s, rec["harm"])]
    thr = T[st]
    is_cand = s > thr
    in_guard = np.abs(s - thr) <= guard * thr
    cands = np.sort(rec[is_cand], order=["trial", "harm", "iz", "ir"])
    guards = np.sort(rec[in_guard], order=["trial", "harm", "iz", "ir"])
    return cands, guards


# --------------------------------------------------------------------------
# 0: dedispersion (the stage that produces the DM-trial series)
# --------------------------------------------------------------------------
K_DM = 4.148808e3   # dispersion constant, MHz^2 pc^-1 cm^3 s


def dm_delays(n_chan: int, f_top: float, df: float, tsamp: float, dm_lo: float,
              dm_step: float, n_dm: int) -> np.ndarray:
    """Delta[d][c] in samples (int64), every operation one IEEE FP64 rounding
    in this order: f = f_top - c*df; a = 1/(f*f); b = 1/(f_top*f_top);
    dm = dm_lo + d*dm_step; x = ((K_DM*dm)*(a - b))/tsamp; floor(x + 1/2)."""
    c = np.arange(n_chan, dtype=np.float64)
    f = f_top - c * df
    a = 1.0 / (f * f)
    b = 1.0 / (f_top * f_top)
    dm = dm_lo + np.arange(n_dm, dtype=np.float64) * dm_step
    x = ((K_DM * dm)[:, None] * (a - b)[None, :]) / tsamp
    return np.floor(x + 0.5).astype(np.int64)


def dedisperse(fb: np.ndarray, delays: np.ndarray, n_out: int) -> np.ndarray:
    """out[d][t] = sum_c fb[c][t + delays[d][c]] for t < n_out, samples at or
    past the end of the filterbank counted as 0 (FP64)."""
    n_chan, n_t = fb.shape
    n_dm = delays.shape[0]
    pad = int(delays.max()) + n_out
    x = np.zeros((n_chan, max(n_t, pad)), dtype=np.float64)
    x[:, :n_t] = fb
    out = np.zeros((n_dm, n_out), dtype=np.float64)
    for d in range(n_dm):
        for c in range(n_chan):
            k = int(delays[d, c])
            out[d] += x[c, k:k + n_out]
    return out


# --------------------------------------------------------------------------
# Fourier-interpolated power for candidate refinement
# --------------------------------------------------------------------------
def refine_window(r: float, z: float, n_r: int) -> np.ndarray:
    """Bins k with |k - round(r)| <= 32 + ceil(|z|/2), clipped to [0, N_r)."""
    k0 = int(math.floor(r + 0.5))
    m = 32 + math.ceil(abs(z) / 2.0 - 1e-12)
    return np.arange(max(0, k0 - m), min(n_r, k0 + m + 1))


def fourier_power(Xn: np.ndarray, r: float, z: float):
    """(P, F) with F(r, z) = sum_k X'_k conj(rho(r - k, z)) over refine_window
    and P = |F|^2, rho unnormalised (a signal X_k = c rho(r0 - k, z0) gives
    P(r0, z0) ~ |c|^2, independent of z0)."""
    k = refine_window(r, z, Xn.shape[0])
    F = np.sum(Xn[k] * np.conj(rho(r - k, z)))
    return float(abs(F) ** 2), complex(F)


# --------------------------------------------------------------------------
# the whole path for one series
# --------------------------------------------------------------------------
def search(x: np.ndarray, z_max: float, z_step: float, n_harm: int,
           sigma: float = 6.0, mode: int = GAMMA_TAIL, norm: str = "median",
           norm_block: int = 2048, trial: int = 0, guard: float = 0.0,
           bank: Bank | None = None, harmonic_mode: int = TOP_HARMONIC,
           interbin: bool = False):
    """Run steps 1-8 on one series; returns a dict of every intermediate.
    With interbin, P is the 2 N_r-column half-bin plane and candidate ir
    values are half-bin columns (r = ir / 2)."""
    geom = geometry(x.shape[0], z_max, z_step, n_harm)
    X = spectrum(x)
    Xn, meds = normalise(X, norm_block, norm)
    if bank is None:
        bank = template_bank(geom)
    P = interbin_plane(correlation_plane(Xn, bank)) if interbin else power_plane(Xn, bank)
    mean, std = plane_stats(P)
    cands, guards = candidates(P, geom, mean, std, sigma, mode, trial, guard,
                               harmonic_mode=harmonic_mode)
    return dict(geom=geom, X=X, Xn=Xn, medians=meds, bank=bank, P=P,
                mean=mean, std=std, T=thresholds(n_harm, sigma, mode, mean, std),
                candidates=cands, guard=guards)
