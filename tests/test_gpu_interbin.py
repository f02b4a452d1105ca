"""Interbinning (the half-bin plane) through the C ABI against the FP64 oracle.

The option samples the plane every half bin: column 2r = |F(r)|^2, column
2r + 1 = (pi/4)^2 |F(r) - F(r+1)|^2 with F(N_r) = 0, F the complex matched-
filter output.  Tolerances, from the arithmetic:

* complex F, FP32 path: |F_gpu - F_ora| <= 1e-4 max(|F_ora|, 1) (half the
  relative error of the FP32 power plane bound, |F| ~ 1 on unit-power noise);
  16-bit storage: 1.5e-2 max(|F_ora|, 1) (half of the 3% power bound).
* even columns: as the power plane, 1e-4 (FP32) / 3% (16-bit) of
  max(P, mean).
* odd columns: the error of F(r) - F(r+1) scales with |F(r)| + |F(r+1)|, so
  the bound is taken against the largest of the cell and its two bin
  neighbours (and the mean): 2e-4 (FP32) / 6% (16-bit).
* statistics of the half-bin plane: 1e-6 (FP32) / 1e-3 (16-bit) relative.
* candidates: the oracle's set outside the guard band (1e-4 FP32, 3% 16-bit).
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    O.build()
    return c


def _cplx(t):
    a = t.float().cpu().numpy().astype(np.float64)
    return a[..., 0::2] + 1j * a[..., 1::2]


def _spectrum(plan, n, seed, z_max):
    x = S.sinusoid_series(n=n, seed=seed, r0=0.3 * n / 2 + 0.5, z0=z_max * 0.45, amp=0.1)
    Xn, _ = O.normalise(O.spectrum(x), 2048)
    il = np.empty(2 * Xn.shape[0], dtype=np.float32)
    il[0::2], il[1::2] = Xn.real, Xn.imag
    spec = torch.from_numpy(il).cuda().to(plan.spec_dtype)
    return spec, _cplx(spec)   # the oracle sees the spectrum as the GPU stored it


CASES = [  # (precision, correlator)
    (0, 1), (1, 1), (1, 2), (2, 2), (2, 1),
]


@pytest.mark.parametrize("prec,corr", CASES)
def test_correlation_plane_matches_direct_sum(capi, prec, corr):
    n, z_max, z_step, L = 1 << 15, 16.0, 2.0, 2048
    plan = capi.Plan(n, 64e-6, z_max, z_step, L, 4, precision=prec, correlator=corr)
    assert plan.info.correlator == corr
    spec, Xs = _spectrum(plan, n, 11, z_max)
    F = _cplx(plan.correlation_plane(spec))
    torch.cuda.synchronize()
    ref = O.correlation_plane(Xs, O.template_bank(O.geometry(n, z_max, z_step, 4)))
    tol = 1e-4 if prec == 0 else 1.5e-2
    err = np.abs(F - ref) / np.maximum(np.abs(ref), 1.0)
    assert err.max() < tol, (err.max(), np.unravel_index(np.argmax(err), err.shape))
    plan.close()


def _check_half_bin_plane(got, P, prec):
    mean = P.mean()
    even_tol, odd_tol = (1e-4, 2e-4) if prec == 0 else (0.03, 0.06)
    e = np.abs(got[:, 0::2] - P[:, 0::2]) / np.maximum(P[:, 0::2], mean)
    assert e.max() < even_tol, (e.max(), np.unravel_index(np.argmax(e), e.shape))
    Pe = P[:, 0::2]
    nb = np.maximum(Pe, np.concatenate([Pe[:, 1:], np.zeros((P.shape[0], 1))], axis=1))
    o = np.abs(got[:, 1::2] - P[:, 1::2]) / np.maximum(np.maximum(P[:, 1::2], nb), mean)
    assert o.max() < odd_tol, (o.max(), np.unravel_index(np.argmax(o), o.shape))


@pytest.mark.parametrize("prec,corr", CASES)
@pytest.mark.parametrize("n,z_max,z_step,L", [
    (1 << 15, 16.0, 2.0, 2048),     # several segments / tiles, ragged last segment
    (1 << 10, 2.0, 1.0, 1024),      # one 512-bin tile, one segment
    (1 << 16, 96.0, 1.0, 8192),     # the 193-template grid
])
def test_half_bin_plane_matches_oracle(capi, prec, corr, n, z_max, z_step, L):
    plan = capi.Plan(n, 64e-6, z_max, z_step, L, 4, precision=prec, correlator=corr,
                     interbin=True)
    assert plan.info.interbin == 1 and plan.info.plane_cols == n
    spec, Xs = _spectrum(plan, n, 5, z_max)
    plane, stats = plan.power_plane(spec)
    torch.cuda.synchronize()
    g = O.geometry(n, z_max, z_step, 4)
    P = O.interbin_plane(O.correlation_plane(Xs, O.template_bank(g)))
    got = plane.float().cpu().numpy().astype(np.float64)
    if prec == 2:
        got *= 16.0          # FP16 planes hold P/16
    assert got.shape == P.shape == (g.n_z, n)
    _check_half_bin_plane(got, P, prec)
    mean, std = O.plane_stats(P)
    s = stats.cpu().numpy()
    stol = 1e-6 if prec == 0 else 1e-3
    assert abs(s[0] / mean - 1) < stol and abs(s[1] / std - 1) < stol, (s, mean, std)
    plan.close()


def test_half_bin_tone_is_recovered_on_the_gpu(capi):
    """A sinusoid half-way between bins: the integer plane keeps (2/pi)^2 of
    its power, the half-bin column nearly all of it."""
    n, a, k0 = 1 << 14, 0.05, 1234
    u = np.arange(n) / n
    x = (a * np.cos(2 * np.pi * (k0 + 0.5) * u)).astype(np.float32)
    full = (a * n / 2) ** 2
    plan = capi.Plan(n, 64e-6, 4.0, 2.0, 1024, 1, norm_mode=capi.FDAS_NORM_NONE, interbin=True)
    spec = plan.spectrum(torch.from_numpy(x).cuda())
    plane, _ = plan.power_plane(spec)
    row = plane[plan.info.iz0].cpu().numpy().astype(np.float64)
    assert int(np.argmax(row)) == 2 * k0 + 1
    assert row[2 * k0 + 1] > 0.95 * full
    assert abs(row[2 * k0] / full - (2 / math.pi) ** 2) < 0.01
    plan.close()


def _compare(cands, ref, guard, rel_power):
    gk = {(int(h), int(z), int(r)): float(p)
          for h, z, r, p in zip(cands["harm"], cands["iz"], cands["ir"], cands["power"])}
    rk = {(int(h), int(z), int(r)): float(p)
          for h, z, r, p in zip(ref["harm"], ref["iz"], ref["ir"], ref["power"])}
    gd = {(int(h), int(z), int(r)) for h, z, r in zip(guard["harm"], guard["iz"], guard["ir"])}
    diff = (set(gk) ^ set(rk)) - gd
    assert not diff, sorted(diff)[:10]
    worst = max([abs(gk[k] / rk[k] - 1) for k in set(gk) & set(rk)] or [0.0])
    assert worst <= rel_power, worst


@pytest.mark.parametrize("prec,H", [(0, 4), (1, 16), (2, 8)])
def test_interbinned_search_matches_oracle(capi, prec, H):
    n = 1 << 15
    x, _ = S.pulsar_series(n, seed=31, height=1.0, z_abs=10.0)
    guard = 1e-4 if prec == 0 else 0.03
    ref = O.search(x, 16.0, 2.0, H, guard=guard, interbin=True)
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, H, precision=prec, interbin=True)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands) and nf > 0
    assert cands["ir"].max() < n            # half-bin columns
    _compare(cands, ref["candidates"], ref["guard"], guard)
    plan.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_interbinned_uneven_batch(capi, prec):
    """Full-length and decimated series in one call, each on its own
    half-bin plane (FP32: FFT correlator + interbinning kernel; BF16: the
    tensor-core epilogue and its edge table at two plane widths)."""
    n = 1 << 14
    xs = [S.pulsar_series(n, seed=41, height=1.0, z_abs=6.0)[0],
          S.pulsar_series(n // 2, seed=42, height=1.0, z_abs=6.0)[0],
          S.pulsar_series(n // 4, seed=43, height=1.0, z_abs=6.0)[0]]
    guard = 1e-4 if prec == 0 else 0.03
    plan = capi.Plan(n, 64e-6, 8.0, 2.0, 1024, 4, interbin=True, precision=prec)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda() for x in xs], trial_ids=[7, 9, 11],
                                capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands)
    for tid, x in zip((7, 9, 11), xs):
        ref = O.search(x, 8.0, 2.0, 4, guard=guard, interbin=True)
        mine = cands[cands["trial_id"] == tid]
        assert len(ref["candidates"]) > 0
        _compare(mine, ref["candidates"], ref["guard"], guard)
    plan.close()
