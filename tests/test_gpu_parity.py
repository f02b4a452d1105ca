"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
* templates: FP64 Fresnel (GPU) vs FP64 quadrature (oracle): 1e-12 absolute.
* spectrum (FP32 FFT, N <= 2^23): max |X'_gpu - X'_ora| <= 3e-5 rms|X'| +
  2e-6 max|X'| (rounding of ~log2 N FP32 butterfly stages on unit-power
  data, plus the round-off leakage of the strongest bin).
* power plane, FP32 path: |P_gpu - P_ora| <= 1e-4 * max(P_ora, mean) per cell.
* harmonic sums of an FP32 plane: relative 2e-6 (at most 32 FP32 additions).
* candidates, FP32 path: the same (trial, h, iz, ir) set as the oracle
  except cells within the guard band |S - T| <= 1e-4 T, where rounding may
  decide; powers of common candidates within 1e-4 relative.
* BF16/FP16 storage: max detection-power error over the oracle's candidate
  cells <= 3% (paper §2.2 reports 2.7% for its BF16 convolution stage);
  candidate sets agree outside a 3% guard band.
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


def _plan(capi, n, z_max, z_step, L, H, **kw):
    return capi.Plan(n, 64e-6, z_max, z_step, L, H, **kw)


def _cplx(t):
    a = t.float().cpu().numpy().astype(np.float64)
    return a[0::2] + 1j * a[1::2]


def _keys(c, trial_field="trial"):
    return {(int(t), int(h), int(z), int(r))
            for t, h, z, r in zip(c[trial_field], c["harm"], c["iz"], c["ir"])}


# ---------------------------------------------------------------------------
# a0: template bank
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("z_max,z_step,L", [(16.0, 2.0, 2048), (96.0, 1.0, 8192), (7.5, 0.5, 1024)])
def test_template_taps_match_quadrature(capi, z_max, z_step, L):
    plan = _plan(capi, 1 << 14, z_max, z_step, L, 4)
    taps, energy = plan.template_bank()
    g = O.geometry(1 << 14, z_max, z_step, 4)
    bank = O.template_bank(g)
    assert len(taps) == g.n_z
    for iz in range(g.n_z):
        assert np.max(np.abs(taps[iz] - bank.taps[iz])) < 1e-12, iz
    assert np.max(np.abs(energy - bank.energy)) < 1e-12
    plan.close()


# ---------------------------------------------------------------------------
# a1-a2: spectrum + normalisation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1 << 10, 1 << 14, 1 << 15, 1 << 17, 1 << 20, 1 << 23])
def test_spectrum_matches_oracle(capi, n):
    x = S.white_noise(n, 31) + 0.5 * np.sin(np.arange(n) * 0.3).astype(np.float32)
    x = x.astype(np.float32)
    plan = _plan(capi, n, 4.0, 1.0, 1024, 2)
    spec, med = plan.spectrum(torch.from_numpy(x).cuda(), medians=True)
    torch.cuda.synchronize()
    got = _cplx(spec)
    Xn, meds = O.normalise(O.spectrum(x), 2048)
    rms = math.sqrt(np.mean(np.abs(Xn) ** 2))
    err = np.max(np.abs(got - Xn))
    # FP32 round-off of ~log2 N butterfly stages, on the noise level and on
    # the leakage of the strongest bin (the injected tone)
    assert err <= 3e-5 * rms + 2e-6 * np.max(np.abs(Xn)), (err, rms)
    assert np.max(np.abs(med.cpu().numpy() / meds - 1)) < 2e-5
    plan.close()


@pytest.mark.parametrize("block", [16, 128, 2048, 8192])
def test_block_medians_at_every_block_size(capi, block):
    # exact middle order statistics of every block: odd counts (block 0 has
    # no k = 0), crowded and sparse first-digit bins over 2048 blocks of 16
    n = 1 << 16
    x = S.white_noise(n, 11)
    plan = _plan(capi, n, 4.0, 1.0, 1024, 2, norm_block=block)
    spec, med = plan.spectrum(torch.from_numpy(x).cuda(), medians=True)
    _, meds = O.normalise(O.spectrum(x), block)
    assert med.shape[0] == meds.shape[0] == (n // 2) // block
    assert np.max(np.abs(med.cpu().numpy() / meds - 1)) < 2e-5
    plan.close()


@pytest.mark.parametrize("shift", [0, 1])
def test_block_medians_of_equal_powers(capi, shift):
    # an impulse: every |X_k|^2 is 1, exactly (shift 0: Z_k = 1) or up to
    # rounding of |W^k|^2 (shift 1: X_k = W_N^k), so each block's keys share
    # one first-digit bin and the selection takes its radix passes
    n = 1 << 15
    x = np.zeros(n, np.float32)
    x[shift] = 1.0
    plan = _plan(capi, n, 4.0, 1.0, 1024, 2)
    spec, med = plan.spectrum(torch.from_numpy(x).cuda(), medians=True)
    m = med.cpu().numpy()
    if shift == 0:
        assert np.all(m == 1.0)
        got = _cplx(spec)
        ref = np.full(n // 2, math.sqrt(math.log(2.0)), np.complex128)
        ref[0] = 0.0
        assert np.max(np.abs(got - ref)) < 1e-6
    else:
        assert np.max(np.abs(m - 1.0)) < 1e-6
    plan.close()


def test_spectrum_without_normalisation(capi):
    n = 1 << 16
    x = S.white_noise(n, 5)
    plan = _plan(capi, n, 4.0, 1.0, 1024, 2, norm_mode=capi.FDAS_NORM_NONE)
    got = _cplx(plan.spectrum(torch.from_numpy(x).cuda()))
    X = O.spectrum(x)
    assert np.max(np.abs(got - X)) <= 3e-5 * math.sqrt(np.mean(np.abs(X) ** 2))
    plan.close()


# ---------------------------------------------------------------------------
# a3-a6: correlation / power plane / statistics
# ---------------------------------------------------------------------------
def _plane_case(capi, n, z_max, z_step, L, seed=7, prec=0, corr=None, **kw):
    x = S.sinusoid_series(n=n, seed=seed, r0=0.3 * n / 2 + 0.4, z0=z_max * 0.45, amp=0.1)
    g = O.geometry(n, z_max, z_step, 4)
    Xn, _ = O.normalise(O.spectrum(x), 2048)
    plan = _plan(capi, n, z_max, z_step, L, 4, precision=prec, correlator=corr, **kw)
    if corr is not None:
        assert plan.info.correlator == corr
    il = np.empty(2 * Xn.shape[0], dtype=np.float32)
    il[0::2], il[1::2] = Xn.real, Xn.imag
    spec = torch.from_numpy(il).cuda().to(plan.spec_dtype)
    plane, stats = plan.power_plane(spec)
    torch.cuda.synchronize()
    # the oracle sees the spectrum exactly as the GPU stored it
    Xs = _cplx(spec)
    P = O.power_plane(Xs, O.template_bank(g))
    return plan, plane, stats, P, g


@pytest.mark.parametrize("n,z_max,z_step,L", [
    (1 << 17, 16.0, 2.0, 2048),     # the 2^17 / 17 z / 2048 workload
    (1 << 14, 16.0, 2.0, 1024),
    (1 << 15, 40.0, 1.0, 4096),
    (1 << 16, 96.0, 1.0, 8192),     # the 193-template grid, 8192 segments
    (1 << 12, 0.0, 1.0, 1024),      # a single template (z = 0)
])
def test_power_plane_fp32_matches_direct_correlation(capi, n, z_max, z_step, L):
    plan, plane, stats, P, g = _plane_case(capi, n, z_max, z_step, L)
    got = plane.cpu().numpy().astype(np.float64)
    mean, std = O.plane_stats(P)
    tol = 1e-4 * np.maximum(P, mean)
    bad = np.abs(got - P) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], P[bad][:5])
    s = stats.cpu().numpy()
    assert abs(s[0] / mean - 1) < 1e-6 and abs(s[1] / std - 1) < 1e-5
    plan.close()


@pytest.mark.parametrize("corr", [1, 2])
@pytest.mark.parametrize("prec", [1, 2])
def test_power_plane_low_precision_storage(capi, prec, corr):
    """Both correlators (overlap-save FFTs, tensor-core GEMM) at BF16/FP16:
    every cell within 3% of max(P, mean), statistics within 1e-3."""
    plan, plane, stats, P, g = _plane_case(capi, 1 << 17, 16.0, 2.0, 2048, prec=prec, corr=corr)
    got = plane.float().cpu().numpy().astype(np.float64)
    if prec == 2:
        got *= 16.0          # FP16 planes hold P/16
    mean, std = O.plane_stats(P)
    rel = np.abs(got - P) / np.maximum(P, mean)
    assert rel.max() < 0.03, rel.max()
    s = stats.cpu().numpy()
    assert abs(s[0] / mean - 1) < 1e-3 and abs(s[1] / std - 1) < 1e-3, (s, mean, std)
    plan.close()


@pytest.mark.parametrize("n,z_max,z_step", [
    (1 << 10, 2.0, 1.0),        # one 512-bin tile
    (1 << 12, 0.0, 1.0),        # a single template (z = 0)
    (1 << 14, 7.5, 0.5),        # half-step grid, ragged last chunk (31 templates)
    (1 << 16, 96.0, 1.0),       # the 193-template grid: 7 chunks of 28
    (1 << 15, 200.0, 4.0),      # widest templates (m = 108), 101 templates
])
@pytest.mark.parametrize("prec,order", [(1, 2), (2, 2), (1, 1), (2, 1)])
def test_tensor_plane_matches_direct_correlation(capi, n, z_max, z_step, prec, order):
    """The tensor-core correlation against the FP64 direct sum over the whole
    plane (every tile, chunk and phase), on the spectrum exactly as stored:
    within 3% of max(P, mean) (16-bit taps and plane, FP32 sums); both
    template orders of the chunks (paired +-|z|, consecutive z)."""
    plan, plane, stats, P, g = _plane_case(capi, n, z_max, z_step, 1024 if z_max < 100 else 2048,
                                           prec=prec, corr=capi.FDAS_CORR_TENSOR,
                                           template_order=order)
    assert plan.info.template_order == order
    got = plane.float().cpu().numpy().astype(np.float64)
    if prec == 2:
        got *= 16.0
    mean, std = O.plane_stats(P)
    rel = np.abs(got - P) / np.maximum(P, mean)
    assert rel.max() < 0.03, (rel.max(), np.unravel_index(np.argmax(rel), rel.shape))
    s = stats.cpu().numpy()
    assert abs(s[0] / mean - 1) < 1e-3 and abs(s[1] / std - 1) < 1e-3, (s, mean, std)
    plan.close()


def test_longest_segment_needs_the_tensor_cores(capi):
    """seg_len 16384: a tensor-core plan (no segments in its direct sum)
    searches exactly like one with 8192-bin segments; the overlap-save
    correlator does not take it."""
    n = 1 << 17
    x = torch.from_numpy(S.sinusoid_series()).cuda()
    res = []
    for L in (8192, 16384):
        plan = _plan(capi, n, 16.0, 2.0, L, 4, precision=capi.FDAS_BF16)
        assert plan.info.seg_len == L and plan.info.correlator == capi.FDAS_CORR_TENSOR
        st, c, nf = plan.search([x])
        assert st == capi.FDAS_OK and nf > 0
        res.append(c.tobytes())
        plan.close()
    assert res[0] == res[1]
    with pytest.raises(capi.FdasError) as ei:
        _plan(capi, n, 16.0, 2.0, 16384, 4, precision=capi.FDAS_FP32)
    assert ei.value.status == capi.FDAS_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,z_max,z_step", [
    (1 << 10, 2.0, 1.0),        # one 512-bin tile
    (1 << 14, 7.5, 0.5),        # half-step grid, ragged last chunk
    (1 << 16, 96.0, 1.0),       # the 193-template grid: the widest chunks that fit
])
def test_tensor_split_fp32_plane(capi, n, z_max, z_step):
    """FP32 storage on the tensor cores (BF16 hi + lo operands, three
    products per term): every cell within the FP32 bound 1e-4 * max(P, mean)
    of the FP64 direct sum, statistics within 1e-5."""
    plan, plane, stats, P, g = _plane_case(capi, n, z_max, z_step, 1024 if n < (1 << 16) else 8192,
                                           prec=0, corr=capi.FDAS_CORR_TENSOR_SPLIT)
    got = plane.cpu().numpy().astype(np.float64)
    mean, std = O.plane_stats(P)
    rel = np.abs(got - P) / np.maximum(P, mean)
    assert rel.max() < 1e-4, (rel.max(), np.unravel_index(np.argmax(rel), rel.shape))
    s = stats.cpu().numpy()
    assert abs(s[0] / mean - 1) < 1e-5 and abs(s[1] / std - 1) < 1e-5, (s, mean, std)
    plan.close()


def test_tensor_split_fp32_search(capi):
    n = 1 << 16
    x, _ = S.pulsar_series(n, seed=21, height=1.0, z_abs=14.0)
    ref = O.search(x, 16.0, 2.0, 16, guard=1e-4)
    plan = _plan(capi, n, 16.0, 2.0, 2048, 16, correlator=capi.FDAS_CORR_TENSOR_SPLIT)
    assert plan.info.correlator == capi.FDAS_CORR_TENSOR_SPLIT
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands) and nf > 0
    _compare_cands(cands, ref["candidates"], ref["guard"], rel_power=1e-4)
    plan.close()


def test_tensor_correlator_is_refused_where_it_does_not_apply(capi):
    with pytest.raises(capi.FdasError) as ei:
        _plan(capi, 1 << 14, 16.0, 2.0, 2048, 4, precision=capi.FDAS_FP32,
              correlator=capi.FDAS_CORR_TENSOR)
    assert ei.value.status == capi.FDAS_ERR_ARG
    auto32 = _plan(capi, 1 << 14, 16.0, 2.0, 2048, 4)
    assert auto32.info.correlator == capi.FDAS_CORR_FFT
    auto16 = _plan(capi, 1 << 14, 16.0, 2.0, 2048, 4, precision=capi.FDAS_BF16)
    assert auto16.info.correlator == capi.FDAS_CORR_TENSOR
    auto32.close()
    auto16.close()


# ---------------------------------------------------------------------------
# a7: harmonic sums
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("H", [1, 2, 4, 8, 16, 32])
def test_harmonic_sums_match_oracle(capi, H):
    n, z_max = 1 << 12, 24.0
    g = O.geometry(n, z_max, 1.0, H)
    rng = np.random.default_rng(H)
    P = rng.exponential(size=(g.n_z, g.n_r)).astype(np.float32)
    plan = _plan(capi, n, z_max, 1.0, 1024, H)
    sums = plan.harmonic_sums(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    ref = O.harmonic_planes(P.astype(np.float64), g)
    got = sums.cpu().numpy()
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref) / ref) < 2e-6
    plan.close()


def test_harmonic_spike_train_through_gpu(capi):
    H = 16
    n = 1 << 13
    g = O.geometry(n, 48.0, 1.0, H)
    P = np.zeros((g.n_z, g.n_r), dtype=np.float32)
    rf, of = 97, -2
    for j in range(1, H + 1):
        P[g.iz0 + j * of, j * rf] += 2.0 ** j
    plan = _plan(capi, n, 48.0, 1.0, 1024, H)
    sums = plan.harmonic_sums(torch.from_numpy(P).cuda()).cpu().numpy()
    top = (g.iz0 + H * of, H * rf)
    for st, h in enumerate(g.stages):
        assert sums[st][top] == sum(2.0 ** (k * H // h) for k in range(1, h + 1))
    plan.close()


# ---------------------------------------------------------------------------
# a8: threshold and candidate list
# ---------------------------------------------------------------------------
def _compare_cands(got, ref, guard, rel_power=1e-4, trial_field="trial_id"):
    gk = {(int(t), int(h), int(z), int(r)): (float(p), float(s))
          for t, h, z, r, p, s in zip(got[trial_field], got["harm"], got["iz"], got["ir"],
                                      got["power"], got["sigma"])}
    rk = {(int(t), int(h), int(z), int(r)): (float(p), float(s))
          for t, h, z, r, p, s in zip(ref["trial"], ref["harm"], ref["iz"], ref["ir"],
                                      ref["power"], ref["sigma"])}
    gd = _keys(guard)
    diff = (set(gk) ^ set(rk)) - gd
    assert not diff, sorted(diff)[:10]
    worst = 0.0
    for k in set(gk) & set(rk):
        worst = max(worst, abs(gk[k][0] / rk[k][0] - 1))
    assert worst <= rel_power, worst
    return gk, rk


def test_threshold_on_oracle_plane(capi):
    n = 1 << 15
    x = S.sinusoid_series(n=n, seed=3, r0=3000.3, z0=-5.0, amp=0.15)
    ref = O.search(x, 16.0, 2.0, 4, guard=1e-4)
    plan = _plan(capi, n, 16.0, 2.0, 2048, 4)
    plane = torch.from_numpy(ref["P"].astype(np.float32)).cuda()
    stats = torch.tensor([ref["mean"], ref["std"]], dtype=torch.float64, device="cuda")
    st, cands, nf = plan.threshold(plane, stats, trial_id=0)
    assert st == capi.FDAS_OK and nf == len(cands) and nf > 0
    gk, rk = _compare_cands(cands, ref["candidates"], ref["guard"], rel_power=2e-6)
    for k in set(gk) & set(rk):
        assert abs(gk[k][1] - rk[k][1]) < 1e-3 * max(1.0, abs(rk[k][1]))
    # ordered by (trial, harm, iz, ir)
    order = list(zip(cands["harm"], cands["iz"], cands["ir"]))
    assert order == sorted(order)
    plan.close()


def test_mean_plus_ksigma_mode(capi):
    n = 1 << 14
    x = S.sinusoid_series(n=n, seed=4, r0=2000.5, z0=3.0, amp=0.2)
    ref = O.search(x, 16.0, 2.0, 4, sigma=4.0, mode=O.MEAN_PLUS_KSIGMA, guard=1e-4)
    plan = _plan(capi, n, 16.0, 2.0, 2048, 4, threshold_sigma=4.0,
                 threshold_mode=capi.FDAS_THRESH_MEAN_PLUS_KSIGMA)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()])
    assert st == capi.FDAS_OK
    gk, rk = _compare_cands(cands, ref["candidates"], ref["guard"])
    for k in set(gk) & set(rk):
        assert abs(gk[k][1] - rk[k][1]) < 1e-3 * max(1.0, abs(rk[k][1]))
    plan.close()


# ---------------------------------------------------------------------------
# whole path
# ---------------------------------------------------------------------------
def test_search_sinusoid_workload_fp32(capi):
    """2^17 samples, 17 templates (z in [-16, 16] step 2), 2048-bin segments,
    4 harmonics, 6-sigma: the candidate list equals the oracle's."""
    x = S.sinusoid_series()
    ref = O.search(x, 16.0, 2.0, 4, guard=1e-4)
    plan = _plan(capi, 1 << 17, 16.0, 2.0, 2048, 4)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()])
    assert st == capi.FDAS_OK and nf == len(cands) > 0
    gk, rk = _compare_cands(cands, ref["candidates"], ref["guard"])
    for k in set(gk) & set(rk):
        assert abs(gk[k][1] - rk[k][1]) < 1e-3 * max(1.0, abs(rk[k][1]))
    assert any(k[1] == 1 and k[3] == 5000 for k in gk)
    plan.close()


@pytest.mark.parametrize("corr", [1, 2])
@pytest.mark.parametrize("prec", [1, 2])
def test_search_low_precision_within_three_percent(capi, prec, corr):
    x = S.sinusoid_series()
    ref = O.search(x, 16.0, 2.0, 4, guard=0.03)
    plan = _plan(capi, 1 << 17, 16.0, 2.0, 2048, 4, precision=prec, correlator=corr)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()])
    assert st == capi.FDAS_OK and nf > 0
    gk, rk = _compare_cands(cands, ref["candidates"], ref["guard"], rel_power=0.03)
    plan.close()


@pytest.mark.parametrize("H,prec", [(32, 0), (32, 1), (16, 2), (2, 1)])
def test_search_other_harmonic_counts(capi, H, prec):
    """Whole searches with H = 32 (the direct gather kernel), H = 16 at FP16
    and H = 2, against the oracle (FP32: 1e-4 guard; 16-bit: 3%)."""
    n = 1 << 16
    x, _ = S.pulsar_series(n, seed=21, height=1.0, z_abs=14.0)
    guard = 1e-4 if prec == 0 else 0.03
    ref = O.search(x, 16.0, 2.0, H, guard=guard)
    plan = _plan(capi, n, 16.0, 2.0, 2048, H, precision=prec)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands) and nf > 0
    _compare_cands(cands, ref["candidates"], ref["guard"], rel_power=guard)
    plan.close()


def test_batch_order_host_input_and_reuse(capi):
    n = 1 << 15
    xs, refs = [], []
    for i in range(4):
        x, _ = S.batch_series(i, n=n)
        x = (x + S.inject_sinusoid(np.zeros(n, np.float32), 1000.0 + 300 * i, 4.0, 0.1)).astype(np.float32)
        xs.append(x)
        refs.append(O.search(x, 16.0, 2.0, 4, trial=[30, 10, 20, 0][i], guard=1e-4))
    plan = _plan(capi, n, 16.0, 2.0, 2048, 4)
    ids = [30, 10, 20, 0]
    dev = [torch.from_numpy(x).cuda() for x in xs]
    host = [torch.from_numpy(x) for x in xs]          # pageable host memory
    for run in range(2):
        st, cands, nf = plan.search(dev if run == 0 else host, trial_ids=ids)
        assert st == capi.FDAS_OK
        ref = np.sort(np.concatenate([r["candidates"] for r in refs]),
                      order=["trial", "harm", "iz", "ir"])
        guard = np.concatenate([r["guard"] for r in refs])
        _compare_cands(cands, ref, guard)
        tid = list(cands["trial_id"])
        assert tid == sorted(tid)
    plan.close()


def test_empty_batch_and_overflow(capi):
    n = 1 << 14
    x = S.sinusoid_series(n=n, seed=9, r0=1500.2, z0=2.0, amp=0.3)
    plan = _plan(capi, n, 16.0, 2.0, 2048, 4)
    st, cands, nf = plan.search([])
    assert st == capi.FDAS_OK and nf == 0
    st, full, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 14)
    assert st == capi.FDAS_OK and nf > 4
    st, part, nf2 = plan.search([torch.from_numpy(x).cuda()], capacity=3)
    assert st == capi.FDAS_ERR_CAND_OVERFLOW and nf2 == nf
    assert part.tolist() == full[:3].tolist()
    plan.close()


@pytest.mark.parametrize("prec,corr", [(0, 1), (1, 2)])
def test_silent_series_in_a_batch(capi, prec, corr):
    """A degenerate input: an all-zero series (every block median 0, factor 0)
    between two ordinary ones.  Its spectrum and plane are exactly 0 and it
    gives no candidate in either threshold mode; the other series' lists are
    the oracle's (FP32: 1e-4 guard band; BF16: 3%)."""
    n = 1 << 14
    zero = np.zeros(n, np.float32)
    xs = [S.sinusoid_series(n=n, seed=31, r0=2000.3, z0=3.0, amp=0.3), zero,
          S.sinusoid_series(n=n, seed=32, r0=3100.6, z0=-5.0, amp=0.3)]
    guard = 1e-4 if prec == 0 else 0.03
    for mode in (capi.FDAS_THRESH_GAMMA_TAIL, capi.FDAS_THRESH_MEAN_PLUS_KSIGMA):
        plan = _plan(capi, n, 16.0, 2.0, 2048, 4, precision=prec, correlator=corr,
                     threshold_mode=mode)
        spec = plan.spectrum(torch.from_numpy(zero).cuda())
        assert not torch.any(spec.float() != 0)
        plane, stats = plan.power_plane(spec)
        assert not torch.any(plane.float() != 0) and not torch.any(stats != 0)
        st, cands, nf = plan.search([torch.from_numpy(x).cuda() for x in xs], trial_ids=[0, 1, 2])
        assert st == capi.FDAS_OK and nf == len(cands) > 0
        assert not np.any(cands["trial_id"] == 1)
        for t in (0, 2):
            ref = O.search(xs[t], 16.0, 2.0, 4, mode=mode, trial=t, guard=guard)
            _compare_cands(cands[cands["trial_id"] == t], ref["candidates"], ref["guard"],
                           rel_power=guard)
        plan.close()


@pytest.mark.parametrize("prec,corr", [(0, 1), (1, 2)])
def test_single_template_search(capi, prec, corr):
    """z_max = 0: one template (a plain Fourier search with harmonic sums
    along the z = 0 row), against the oracle."""
    n = 1 << 15
    x, _ = S.pulsar_series(n, seed=23, height=1.0, z_abs=0.0)
    guard = 1e-4 if prec == 0 else 0.03
    ref = O.search(x, 0.0, 1.0, 8, guard=guard)
    plan = _plan(capi, n, 0.0, 1.0, 1024, 8, precision=prec, correlator=corr)
    assert plan.info.n_z == 1
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 16)
    assert st == capi.FDAS_OK and nf == len(cands) > 0
    assert np.all(cands["iz"] == 0)
    _compare_cands(cands, ref["candidates"], ref["guard"], rel_power=guard)
    plan.close()


def test_power_beyond_fp32_range_reported_as_nonfinite(capi):
    """A finite series whose spectral power does not fit in FP32 (one sample
    of 1e21: |X_k|^2 = 1e42) is reported like a non-finite series; one of
    1e15 (|X_k|^2 = 1e30) is searched.  The plan stays usable."""
    n = 1 << 14
    plan = _plan(capi, n, 16.0, 2.0, 2048, 4)
    x = S.white_noise(n, 3)
    x[5] = 1e21
    with pytest.raises(capi.FdasError) as ei:
        plan.search([torch.from_numpy(x).cuda()])
    assert ei.value.status == capi.FDAS_ERR_NONFINITE
    x[5] = 1e15
    st, _, _ = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 10)
    assert st in (capi.FDAS_OK, capi.FDAS_ERR_CAND_OVERFLOW, capi.FDAS_ERR_CAND_STORE_FULL)
    x[5] = 0.0
    st, _, _ = plan.search([torch.from_numpy(x).cuda()])
    assert st == capi.FDAS_OK
    plan.close()


def test_nonfinite_input_reported(capi):
    n = 1 << 14
    x = S.white_noise(n, 2)
    x[123] = np.nan
    plan = _plan(capi, n, 16.0, 2.0, 2048, 4)
    st, cands, nf = None, None, None
    with pytest.raises(capi.FdasError) as ei:
        plan.search([torch.from_numpy(x).cuda()])
    assert ei.value.status == capi.FDAS_ERR_NONFINITE
    # the plan stays usable
    x[123] = 0.0
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()])
    assert st == capi.FDAS_OK
    plan.close()


def test_minimum_size_and_single_harmonic(capi):
    n = 1 << 10
    x = S.sinusoid_series(n=n, seed=12, r0=100.3, z0=1.0, amp=0.6)
    ref = O.search(x, 2.0, 1.0, 1, norm_block=2048, guard=1e-4)
    plan = _plan(capi, n, 2.0, 1.0, 1024, 1)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()])
    assert st == capi.FDAS_OK and nf > 0
    _compare_cands(cands, ref["candidates"], ref["guard"])
    plan.close()
