"""Full-size parity: 2^23 samples, 193 templates (z in [-96, 96] step 1),
8192-bin segments, 16 harmonics -- the configuration the benchmark times.

* One series with three accelerated pulse trains: the whole FP32 power plane
  is compared with the oracle's direct correlation cell by cell, and the
  candidate lists (FP32: identical outside a 1e-4 guard band; BF16/FP16:
  within 3%) are compared with the oracle's.
* A batch of 4 sinusoid series in one BF16 call (the benchmark's launch
  configuration): each GPU candidate's harmonic sum is recomputed by the
  oracle one cell at a time from the series' own spectrum, and must be
  within 3% and above the oracle threshold minus 3%.
* FP32 storage on the tensor cores (split BF16 operands) at full size:
  sampled plane cells within the FP32 bound, the oracle's candidates.
* Interbinning at full size (BF16, the tensor-core epilogue that writes the
  half-bin plane): sampled cells of the 193 x 2^23-column plane, every kind of
  half bin (inside a warp's rows, at a warp edge, at a tile edge, the last
  column) against the oracle's cell-by-cell direct sums on the spectrum as
  stored; and each candidate of a two-series search recomputed from cells.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 1 << 23
Z_MAX, Z_STEP, L, H = 96.0, 1.0, 8192, 16


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    O.build()
    return c


@pytest.fixture(scope="module")
def pulsar_case():
    x, params = S.pulsar_series(N, seed=2)
    ref = O.search(x, Z_MAX, Z_STEP, H, guard=0.03)
    return x, params, ref


def _keyset(c, tf):
    return {(int(t), int(h), int(z), int(r)) for t, h, z, r in zip(c[tf], c["harm"], c["iz"], c["ir"])}


def test_fullsize_fp32_plane_and_candidates(capi, pulsar_case):
    x, params, ref = pulsar_case
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H)
    xd = torch.from_numpy(x).cuda()
    # the whole plane through the stage entry points
    spec = plan.spectrum(xd)
    plane, stats = plan.power_plane(spec)
    torch.cuda.synchronize()
    P = ref["P"]
    got = plane.cpu().numpy()
    tol = 1e-4 * np.maximum(P, ref["mean"])
    bad = np.abs(got - P) > tol
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])
    s = stats.cpu().numpy()
    assert abs(s[0] / ref["mean"] - 1) < 1e-6 and abs(s[1] / ref["std"] - 1) < 1e-5
    del got, plane
    # the search: identical candidates outside the 1e-4 guard band
    st, cands, nf = plan.search([xd], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands) > 0
    T = ref["T"]
    guard = {(0, int(h), int(z), int(r)) for h, z, r, p in
             zip(ref["guard"]["harm"], ref["guard"]["iz"], ref["guard"]["ir"], ref["guard"]["power"])
             if abs(p - T[int(np.log2(h))]) <= 1e-4 * T[int(np.log2(h))]}
    g, r = _keyset(cands, "trial_id"), _keyset(ref["candidates"], "trial")
    assert not ((g ^ r) - guard), sorted((g ^ r) - guard)[:10]
    gp = {(int(h), int(z), int(i)): float(p) for h, z, i, p in
          zip(cands["harm"], cands["iz"], cands["ir"], cands["power"])}
    worst = max(abs(gp[(int(h), int(z), int(i))] / p - 1)
                for h, z, i, p in zip(ref["candidates"]["harm"], ref["candidates"]["iz"],
                                      ref["candidates"]["ir"], ref["candidates"]["power"])
                if (int(h), int(z), int(i)) in gp)
    assert worst < 1e-4, worst
    plan.close()


@pytest.mark.parametrize("corr", [1, 2])
@pytest.mark.parametrize("prec", [1, 2])
def test_fullsize_low_precision_power_error(capi, pulsar_case, prec, corr):
    x, params, ref = pulsar_case
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, precision=prec, correlator=corr)
    assert plan.info.correlator == corr
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf > 0
    g, r = _keyset(cands, "trial_id"), _keyset(ref["candidates"], "trial")
    assert not ((g ^ r) - _keyset(ref["guard"], "trial")), sorted((g ^ r) - _keyset(ref["guard"], "trial"))[:10]
    gp = {(int(h), int(z), int(i)): float(p) for h, z, i, p in
          zip(cands["harm"], cands["iz"], cands["ir"], cands["power"])}
    errs = [abs(gp[(int(h), int(z), int(i))] / p - 1)
            for h, z, i, p in zip(ref["candidates"]["harm"], ref["candidates"]["iz"],
                                  ref["candidates"]["ir"], ref["candidates"]["power"])
            if (int(h), int(z), int(i)) in gp]
    assert len(errs) > 0 and max(errs) <= 0.03, max(errs)
    plan.close()


def test_fullsize_fp32_tensor_split(capi, pulsar_case):
    """FP32 storage on the tensor cores (BF16 hi + lo operands) at full size:
    sampled plane cells within the FP32 bound of the FP64 direct sum on the
    spectrum as stored, and the oracle's candidates outside the 1e-4 guard."""
    x, params, ref = pulsar_case
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, correlator=capi.FDAS_CORR_TENSOR_SPLIT)
    assert plan.info.correlator == capi.FDAS_CORR_TENSOR_SPLIT
    xd = torch.from_numpy(x).cuda()
    spec = plan.spectrum(xd)
    plane, stats = plan.power_plane(spec)
    torch.cuda.synchronize()
    a = spec.cpu().numpy().astype(np.float64)
    Xs = a[0::2] + 1j * a[1::2]
    g = O.geometry(N, Z_MAX, Z_STEP, H)
    rng = np.random.default_rng(8)
    iz = rng.integers(0, g.n_z, 8000)
    r = rng.integers(0, g.n_r, 8000)
    want = O.cell_powers(Xs, O.template_bank(g), iz, r)
    got = plane[torch.from_numpy(iz).cuda(), torch.from_numpy(r).cuda()].cpu().numpy()
    err = np.abs(got - want) / np.maximum(want, ref["mean"])
    assert err.max() < 1e-4, err.max()
    s = stats.cpu().numpy()
    assert abs(s[0] / ref["mean"] - 1) < 1e-5 and abs(s[1] / ref["std"] - 1) < 1e-4
    del plane
    st, cands, nf = plan.search([xd], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands) > 0
    T = ref["T"]
    guard = {(0, int(h), int(z), int(i)) for h, z, i, p in
             zip(ref["guard"]["harm"], ref["guard"]["iz"], ref["guard"]["ir"], ref["guard"]["power"])
             if abs(p - T[int(np.log2(h))]) <= 1e-4 * T[int(np.log2(h))]}
    gk, rk = _keyset(cands, "trial_id"), _keyset(ref["candidates"], "trial")
    assert not ((gk ^ rk) - guard), sorted((gk ^ rk) - guard)[:10]
    plan.close()


def test_fullsize_bf16_batch_candidates_recomputed_by_oracle(capi):
    xs, params = S.torch_batch_series(4, N, base_seed=1000, device="cuda")
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, precision=capi.FDAS_BF16)
    st, cands, nf = plan.search(xs, capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands)
    g = O.geometry(N, Z_MAX, Z_STEP, H)
    bank = O.template_bank(g)
    G = O.gamma_tail_factors(H, 6.0)
    for t, x in enumerate(xs):
        c = cands[cands["trial_id"] == t]
        assert len(c) > 0, f"series {t}: the injected signal was not found"
        Xn, _ = O.normalise(O.spectrum(x.cpu().numpy()), 2048)
        # every gather cell of every candidate, one direct sum each
        cells, owners = [], []
        for n, (h, iz, ir) in enumerate(zip(c["harm"], c["iz"], c["ir"])):
            for k in range(1, int(h) + 1):
                j = k * (H // int(h))
                cells.append(O.harmonic_indices(int(ir), int(iz), g.iz0, H, j))
                owners.append(n)
        cells = np.array(cells)
        pw = O.cell_powers(Xn, bank, cells[:, 0], cells[:, 1])
        s_ora = np.bincount(np.array(owners), weights=pw, minlength=len(c))
        rel = np.abs(c["power"] / s_ora - 1)
        assert rel.max() <= 0.03, (t, rel.max())
        # each candidate is at least near the oracle threshold (mean of the
        # GPU plane agrees with the oracle's to far better than 3%)
        st_ = int(np.log2(c["harm"].max()))
        assert np.all(s_ora >= 0.97 * np.array([G[int(np.log2(h))] for h in c["harm"]]) * 0.98)
    plan.close()


def test_fullsize_interbin_cells_and_candidates(capi):
    xs, params = S.torch_batch_series(2, N, base_seed=2000, device="cuda")
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, precision=capi.FDAS_BF16, interbin=True)
    assert plan.info.correlator == capi.FDAS_CORR_TENSOR and plan.info.plane_cols == N
    g = O.geometry(N, Z_MAX, Z_STEP, H)
    bank = O.template_bank(g)
    # sampled plane cells, from the spectrum exactly as the GPU stored it
    spec = plan.spectrum(xs[0])
    plane, stats = plan.power_plane(spec)
    torch.cuda.synchronize()
    a = spec.float().cpu().numpy().astype(np.float64)
    Xs = a[0::2] + 1j * a[1::2]
    rng = np.random.default_rng(5)
    n_r = N // 2
    iz = rng.integers(0, g.n_z, 6000)
    col = rng.integers(0, 2 * n_r, 6000)
    m = rng.integers(0, n_r // 128, 2000)          # half bins after a warp's last row
    iz = np.concatenate([iz, rng.integers(0, g.n_z, 2000), np.arange(g.n_z)])
    col = np.concatenate([col, 2 * (128 * m + 127) + 1, np.full(g.n_z, 2 * n_r - 1)])
    ref = O.half_bin_cells(Xs, bank, iz, col)
    got = plane[torch.from_numpy(iz).cuda(), torch.from_numpy(col).cuda()].float().cpu().numpy()
    mean = float(stats[0])
    # neighbouring bins bound the error of a half bin (see test_gpu_interbin)
    nb = np.maximum(O.half_bin_cells(Xs, bank, iz, col - col % 2),
                    O.half_bin_cells(Xs, bank, iz, np.minimum(col - col % 2 + 2, 2 * n_r - 2)))
    scale = np.where(col % 2 == 0, np.maximum(ref, mean), np.maximum(np.maximum(ref, nb), mean))
    tol = np.where(col % 2 == 0, 0.03, 0.06)
    err = np.abs(got - ref) / scale
    assert np.all(err < tol), (err.max(), iz[np.argmax(err)], col[np.argmax(err)])
    assert 0.9 < mean < 1.4
    del plane
    # every candidate of a two-series search, each recomputed from oracle
    # cells: the detection strength stays within the paper's 3% (measured on
    # this case: at most 0.54%)
    st, cands, nf = plan.search(xs, capacity=1 << 20)
    assert st == capi.FDAS_OK and nf == len(cands)
    for t, x in enumerate(xs):
        c = cands[cands["trial_id"] == t]
        assert len(c) > 0
        Xn, _ = O.normalise(O.spectrum(x.cpu().numpy()), 2048)
        cells, owners = [], []
        for n, (h, izc, ir) in enumerate(zip(c["harm"], c["iz"], c["ir"])):
            for k in range(1, int(h) + 1):
                cells.append(O.harmonic_indices(int(ir), int(izc), g.iz0, H, k * (H // int(h))))
                owners.append(n)
        cells = np.array(cells)
        pw = O.half_bin_cells(Xn, bank, cells[:, 0], cells[:, 1])
        s_ora = np.bincount(np.array(owners), weights=pw, minlength=len(c))
        rel = np.abs(c["power"] / s_ora - 1)
        assert rel.max() <= 0.03, (t, rel.max())
    plan.close()
