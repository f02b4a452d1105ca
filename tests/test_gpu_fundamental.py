"""The fundamental-indexed harmonic sum (FDAS_HARM_FUNDAMENTAL) against the
FP64 oracle: stage sums on a random plane (2e-6 relative, FP32 sums of FP32
values, 0 outside each stage's domain), the threshold on the oracle's own
plane (every candidate outside a 1e-4 guard band), and whole searches at FP32
(1e-4 guard) and BF16/FP16 storage (3% guard and power)."""
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


def _keys(rec, field):
    return {(int(t), int(h), int(z), int(r)): float(p)
            for t, h, z, r, p in zip(rec[field], rec["harm"], rec["iz"], rec["ir"], rec["power"])}


def _compare(got, ref, guard, rel):
    gk, rk = _keys(got, "trial_id"), _keys(ref, "trial")
    gd = set(_keys(guard, "trial"))
    diff = (set(gk) ^ set(rk)) - gd
    assert not diff, sorted(diff)[:10]
    common = set(gk) & set(rk)
    assert common
    assert max(abs(gk[k] / rk[k] - 1) for k in common) <= rel
    key = list(zip(got["trial_id"], got["harm"], got["iz"], got["ir"]))
    assert key == sorted(key)


@pytest.mark.parametrize("H", [1, 2, 4, 8, 16, 32])
def test_fundamental_sums_match_oracle(capi, H):
    n, z_max = 1 << 12, 40.0
    g = O.geometry(n, z_max, 1.0, H)
    rng = np.random.default_rng(100 + H)
    P = rng.exponential(size=(g.n_z, g.n_r)).astype(np.float32)
    plan = capi.Plan(n, 64e-6, z_max, 1.0, 1024, H, harmonic_mode=capi.FDAS_HARM_FUNDAMENTAL)
    assert plan.info.harmonic_mode == capi.FDAS_HARM_FUNDAMENTAL
    got = plan.harmonic_sums(torch.from_numpy(P).cuda()).cpu().numpy()
    ref = O.fund_planes(P.astype(np.float64), g)
    assert got.shape == ref.shape
    inside = ref > 0
    assert np.all(got[~inside] == 0)
    assert np.max(np.abs(got[inside] - ref[inside]) / ref[inside]) < 2e-6
    plan.close()


def test_fundamental_threshold_on_oracle_plane(capi):
    n = 1 << 15
    x = S.sinusoid_series(n=n, seed=3, r0=3000.3, z0=-5.0, amp=0.15)
    ref = O.search(x, 16.0, 2.0, 4, guard=1e-4, harmonic_mode=O.FUNDAMENTAL)
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4, harmonic_mode=capi.FDAS_HARM_FUNDAMENTAL)
    plane = torch.from_numpy(ref["P"].astype(np.float32)).cuda()
    stats = torch.tensor([ref["mean"], ref["std"]], dtype=torch.float64, device="cuda")
    st, cands, nf = plan.threshold(plane, stats, trial_id=0)
    assert st == capi.FDAS_OK and nf == len(cands) and nf > 0
    _compare(cands, ref["candidates"], ref["guard"], 2e-6)
    # the injected fundamental is found at stage 1 and above
    assert any(int(c["ir"]) == 3000 for c in cands)
    plan.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_fundamental_search_matches_oracle(capi, prec):
    n = 1 << 17
    x, _ = S.pulsar_series(n, seed=9, height=1.0, z_abs=14.0)
    guard = 1e-4 if prec == 0 else 0.03
    ref = O.search(x, 16.0, 2.0, 8, guard=guard, harmonic_mode=O.FUNDAMENTAL)
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 8, precision=prec,
                     harmonic_mode=capi.FDAS_HARM_FUNDAMENTAL)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 18)
    assert st == capi.FDAS_OK and nf == len(cands) and nf > 0
    _compare(cands, ref["candidates"], ref["guard"], 1e-4 if prec == 0 else 0.03)
    plan.close()


def test_harmonic_mode_is_validated(capi):
    with pytest.raises(capi.FdasError) as ei:
        capi.Plan(1 << 14, 64e-6, 16.0, 2.0, 2048, 4, harmonic_mode=7)
    assert ei.value.status == capi.FDAS_ERR_ARG
