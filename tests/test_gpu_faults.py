"""Error paths of the search on the GPU, made on the host.

* A device candidate store smaller than the number of crossings returns
  FDAS_ERR_CAND_STORE_FULL with the true count and no records (the stored
  subset depends on scheduling); a caller buffer smaller than the count but a
  store large enough returns FDAS_ERR_CAND_OVERFLOW with the first records in
  the documented order, equal to the oracle's first records.
* FDAS_FAULT (host-side fault injection): every device allocation of a plan
  failing in turn gives FDAS_ERR_OOM and leaves the device's free memory as it
  was (nothing leaked); `capacity` and `nan_input` give their statuses and the
  plan stays usable.  Nothing here faults, traps or hangs the GPU.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, Z_MAX, Z_STEP, L, H = 1 << 14, 16.0, 2.0, 2048, 4


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    O.build()
    return c


def _series():
    # a strong drifting tone at a low threshold: several hundred crossings
    return S.sinusoid_series(n=N, seed=9, r0=1500.2, z0=2.0, amp=0.3)


def _keys(c, field="trial_id"):
    return [(int(t), int(h), int(z), int(r))
            for t, h, z, r in zip(c[field], c["harm"], c["iz"], c["ir"])]


def test_store_full_is_not_ok_and_reports_the_true_count(capi):
    x = torch.from_numpy(_series()).cuda()
    big = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, threshold_sigma=3.0)
    st, ref, total = big.search([x], capacity=1 << 14)
    big.close()
    assert st == capi.FDAS_OK and total > 300
    small = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, threshold_sigma=3.0, max_candidates=64)
    st, cands, nf = small.search([x], capacity=4096)
    assert st == capi.FDAS_ERR_CAND_STORE_FULL
    assert nf == total and len(cands) == 0
    assert "store" in capi.fdas_last_error()
    # the same plane through fdas_threshold reports the full store too
    spec = small.spectrum(x)
    plane, stats = small.power_plane(spec)
    st, c2, nf2 = small.threshold(plane, stats, capacity=4096)
    assert st == capi.FDAS_ERR_CAND_STORE_FULL and nf2 == total and len(c2) == 0
    small.close()


def test_caller_overflow_gives_the_oracles_first_records(capi):
    """capacity < crossings <= max_candidates: FDAS_ERR_CAND_OVERFLOW, the true
    count, and the first `capacity` records in (trial, h, iz, ir) order equal
    the oracle's first records (compared where the oracle's list is decided
    outside its FP32 guard band)."""
    xn = _series()
    ref = O.search(xn, Z_MAX, Z_STEP, H, sigma=3.0, guard=1e-4)
    want = [(0, int(h), int(z), int(r)) for h, z, r in
            zip(ref["candidates"]["harm"], ref["candidates"]["iz"], ref["candidates"]["ir"])]
    guard = {(0, int(h), int(z), int(r)) for h, z, r in
             zip(ref["guard"]["harm"], ref["guard"]["iz"], ref["guard"]["ir"])}
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, threshold_sigma=3.0)
    x = torch.from_numpy(xn).cuda()
    st, full, total = plan.search([x], capacity=1 << 14)
    assert st == capi.FDAS_OK
    cap = 40
    st, part, nf = plan.search([x], capacity=cap)
    assert st == capi.FDAS_ERR_CAND_OVERFLOW and nf == total and len(part) == cap
    got = _keys(part)
    assert got == _keys(full)[:cap]
    # the oracle's first records, skipping guard-band cells on both sides
    want_clean = [k for k in want if k not in guard]
    got_clean = [k for k in got if k not in guard]
    assert got_clean == want_clean[:len(got_clean)]
    assert len(got_clean) >= cap - len(guard)
    plan.close()


def test_fault_capacity_and_nan_input(capi, monkeypatch):
    x = torch.from_numpy(_series()).cuda()
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H)
    st, ref, total = plan.search([x])
    assert st == capi.FDAS_OK and total >= 2
    monkeypatch.setenv("FDAS_FAULT", "capacity")
    st, c, nf = plan.search([x])
    assert st == capi.FDAS_ERR_CAND_STORE_FULL and nf == total and len(c) == 0
    monkeypatch.setenv("FDAS_FAULT", "nan_input")
    with pytest.raises(capi.FdasError) as ei:
        plan.search([x])
    assert ei.value.status == capi.FDAS_ERR_NONFINITE
    monkeypatch.setenv("FDAS_FAULT", "bad_args")
    with pytest.raises(capi.FdasError) as ei:
        plan.search([x])
    assert ei.value.status == capi.FDAS_ERR_ARG
    monkeypatch.delenv("FDAS_FAULT")
    st, c, nf = plan.search([x])
    assert st == capi.FDAS_OK and nf == total and _keys(c) == _keys(ref)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_every_failed_allocation_frees_the_plan(capi, monkeypatch, prec):
    """FDAS_FAULT=alloc:k for every allocation k of a plan: fdas_plan_create
    returns FDAS_ERR_OOM and the device's free memory is what it was before
    (a leaked plane, spectrum, FFT scratch or staging buffer, 4 MB or more at
    this size, would show; small buffers share pages and cannot be seen)."""
    p = capi.FDAS_FP32 if prec == "fp32" else capi.FDAS_BF16
    n = 1 << 20
    # one plan first, so that lazily loaded kernels are resident before the
    # free memory is read
    capi.Plan(n, 64e-6, 96.0, 1.0, 8192, 16, precision=p).close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for k in range(1, 64):
        monkeypatch.setenv("FDAS_FAULT", f"alloc:{k}")
        try:
            plan = capi.Plan(n, 64e-6, 96.0, 1.0, 8192, 16, precision=p)
        except capi.FdasError as e:
            assert e.status == capi.FDAS_ERR_OOM, e
            assert "injected" in str(e)
            failed += 1
            torch.cuda.synchronize()
            free = torch.cuda.mem_get_info()[0]
            assert abs(free - free0) < (4 << 20), (k, free0 - free)
            continue
        # k is past the plan's last allocation: it was created normally
        plan.close()
        break
    else:
        pytest.fail("the plan never got past its allocations")
    assert failed >= 15
    monkeypatch.delenv("FDAS_FAULT")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (4 << 20)
