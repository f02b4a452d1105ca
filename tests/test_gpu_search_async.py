"""The stream-ordered search (fdas_search_async) and the candidate ordering.

fdas_search_async must give what fdas_search gives: the same records in the
same order (byte for byte), the same n_found and, as `status`, the code
fdas_search returns.  It decides the count and the status on the device and
queues the whole sort network, so these tests run it beside the blocking
call on the same batches: plain, overflowing the caller's buffer, filling the
plan's store, with a non-finite series, and with more than one shared-memory
chunk of records (8192) to order, where the result is also checked to be
sorted by (trial_id, harm, iz, ir) and, for a single trial, to be the
oracle's list.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REC = 20   # bytes per fdas_candidate


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    O.build()
    return c


def _outputs(capacity, pinned):
    if pinned:
        cands = torch.zeros(max(1, capacity) * REC, dtype=torch.uint8).pin_memory()
        nf = torch.full((1,), -1, dtype=torch.int64).pin_memory()
        st = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    else:
        cands = torch.zeros(max(1, capacity) * REC, dtype=torch.uint8, device="cuda")
        nf = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    return cands, nf, st


def _run_async(capi, plan, series, ids, capacity, pinned=False):
    cands, nf, st = _outputs(capacity, pinned)
    if capacity == 0:
        cands = cands[:0]
    plan.search_async(series, cands, nf, st, trial_ids=ids)
    torch.cuda.synchronize()
    n_found, status = int(nf.cpu()[0]), int(st.cpu()[0])
    k = 0 if status == capi.FDAS_ERR_CAND_STORE_FULL else min(n_found, capacity)
    return status, capi.Plan.candidates(cands, k), n_found


def _batch(n, k, seed=0):
    xs = []
    for i in range(k):
        x, _ = S.batch_series(seed + i, n=n)
        x = (x + S.inject_sinusoid(np.zeros(n, np.float32), 900.0 + 350 * i, 3.0, 0.1)).astype(np.float32)
        xs.append(x)
    return xs


@pytest.mark.parametrize("prec,pinned", [(0, False), (1, True)])
def test_async_equals_blocking(capi, prec, pinned):
    n = 1 << 15
    xs = _batch(n, 5)
    ids = [7, 3, 9, 1, 5]
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4, precision=prec)
    dev = [torch.from_numpy(x).cuda() for x in xs]
    host = [torch.from_numpy(x).pin_memory() for x in xs]
    for series in (dev, host):
        st_b, c_b, nf_b = plan.search(series, trial_ids=ids, capacity=1 << 14)
        st_a, c_a, nf_a = _run_async(capi, plan, series, ids, 1 << 14, pinned)
        assert st_b == st_a == capi.FDAS_OK
        assert nf_a == nf_b == len(c_b) > 0
        assert c_a.tobytes() == c_b.tobytes()
    plan.close()


def test_async_overflow_and_store_full(capi):
    n = 1 << 15
    xs = [torch.from_numpy(x).cuda() for x in _batch(n, 3, seed=10)]
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4)
    st_b, c_b, nf_b = plan.search(xs, capacity=1 << 14)
    assert st_b == capi.FDAS_OK and nf_b > 8
    # the caller's buffer holds only the first 5 records
    st_a, c_a, nf_a = _run_async(capi, plan, xs, None, 5)
    assert st_a == capi.FDAS_ERR_CAND_OVERFLOW and nf_a == nf_b
    assert c_a.tobytes() == c_b[:5].tobytes()
    # no buffer at all
    st0, c0, nf0 = _run_async(capi, plan, xs, None, 0)
    assert st0 == capi.FDAS_ERR_CAND_OVERFLOW and nf0 == nf_b and len(c0) == 0
    plan.close()
    # a device store smaller than the crossings
    small = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4, max_candidates=8)
    st_s, _, nf_s = _run_async(capi, small, xs, None, 1 << 10)
    st_bs, _, nf_bs = small.search(xs, capacity=1 << 10)
    assert st_s == st_bs == capi.FDAS_ERR_CAND_STORE_FULL
    assert nf_s == nf_bs == nf_b
    small.close()


def test_async_nonfinite_series(capi):
    n = 1 << 14
    x = S.white_noise(n, 4)
    x[77] = np.nan
    plan = capi.Plan(n, 64e-6, 8.0, 2.0, 2048, 2)
    st, c, nf = _run_async(capi, plan, [torch.from_numpy(x).cuda()], None, 64)
    assert st == capi.FDAS_ERR_NONFINITE and nf == 0 and len(c) == 0
    # the plan is usable afterwards
    y = torch.from_numpy(S.white_noise(n, 5)).cuda()
    st2, _, _ = _run_async(capi, plan, [y], None, 64)
    assert st2 == capi.FDAS_OK
    plan.close()


def test_ordering_of_many_candidates_matches_oracle(capi):
    """More than 8192 records (several shared-memory chunks, global merge
    steps): a low mean-plus-k-sigma threshold on one series.  Both calls give
    the oracle's candidate list (outside the FP32 guard band), sorted."""
    n = 1 << 16
    x = S.sinusoid_series(n=n, seed=8, r0=7000.4, z0=4.0, amp=0.1)
    ref = O.search(x, 16.0, 2.0, 4, sigma=2.0, mode=O.MEAN_PLUS_KSIGMA, guard=1e-4)
    assert len(ref["candidates"]) > 3 * 8192
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4, threshold_sigma=2.0,
                     threshold_mode=capi.FDAS_THRESH_MEAN_PLUS_KSIGMA)
    xd = torch.from_numpy(x).cuda()
    st_b, c_b, nf_b = plan.search([xd], capacity=1 << 17)
    st_a, c_a, nf_a = _run_async(capi, plan, [xd], None, 1 << 17)
    assert st_b == st_a == capi.FDAS_OK and nf_a == nf_b == len(c_b)
    assert c_a.tobytes() == c_b.tobytes()
    keys = np.stack([c_b["trial_id"].astype(np.int64), c_b["harm"], c_b["iz"], c_b["ir"]])
    order = np.lexsort(keys[::-1])
    assert np.array_equal(order, np.arange(len(c_b)))
    got = {(int(h), int(z), int(r)) for h, z, r in zip(c_b["harm"], c_b["iz"], c_b["ir"])}
    want = {(int(h), int(z), int(r)) for h, z, r in zip(ref["candidates"]["harm"],
                                                       ref["candidates"]["iz"],
                                                       ref["candidates"]["ir"])}
    guard = {(int(h), int(z), int(r)) for h, z, r in zip(ref["guard"]["harm"], ref["guard"]["iz"],
                                                        ref["guard"]["ir"])}
    assert (got ^ want) <= guard
    plan.close()


def test_async_returns_before_the_work_is_done(capi):
    if capi.fdas_checked_build():
        pytest.skip("the checked build waits for the device after each launch group")
    n = 1 << 23
    plan = capi.Plan(n, 64e-6, 96.0, 1.0, 8192, 16, precision=capi.FDAS_BF16)
    xs = [torch.randn(n, device="cuda") for _ in range(24)]
    cands, nf, st = _outputs(1 << 16, True)
    plan.search_async(xs, cands, nf, st)   # warm-up (plan buffers, kernels)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    plan.search_async(xs, cands, nf, st)
    pending = not s.query()
    torch.cuda.synchronize()
    assert pending
    assert int(st[0]) == capi.FDAS_OK
    plan.close()


def test_async_argument_checks(capi):
    n = 1 << 14
    plan = capi.Plan(n, 64e-6, 8.0, 2.0, 2048, 2)
    x = torch.from_numpy(S.white_noise(n, 1)).cuda()
    cands, nf, st = _outputs(16, False)
    # outputs in pageable host memory
    with pytest.raises(capi.FdasError):
        plan.search_async([x], cands, torch.zeros(1, dtype=torch.int64), st)
    with pytest.raises(capi.FdasError):
        plan.search_async([x], torch.zeros(16 * REC, dtype=torch.uint8), nf, st)
    # tracing enabled
    plan.profile(True)
    with pytest.raises(capi.FdasError):
        plan.search_async([x], cands, nf, st)
    plan.profile(False)
    plan.search_async([x], cands, nf, st)
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == capi.FDAS_OK
    plan.close()


def test_async_with_graph_replay_and_host_series(capi):
    """A plan that replays each batch as a CUDA graph, series in page-locked
    host memory (copied by the library's copy kernel inside the graph): the
    stream-ordered call gives the blocking call's records, twice in a row
    (the second replays the updated graph)."""
    n = 1 << 15
    xs = _batch(n, 4, seed=30)
    ids = [4, 2, 8, 6]
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4, precision=capi.FDAS_BF16, use_graph=True)
    host = [torch.from_numpy(x).pin_memory() for x in xs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st_b, c_b, nf_b = plan.search(host, trial_ids=ids, capacity=1 << 14, stream=stream)
        assert st_b == capi.FDAS_OK and nf_b == len(c_b) > 0
        for _ in range(2):
            cands, nf, st = _outputs(1 << 14, False)
            plan.search_async(host, cands, nf, st, trial_ids=ids, stream=stream)
            stream.synchronize()
            assert int(st.cpu()[0]) == capi.FDAS_OK and int(nf.cpu()[0]) == nf_b
            assert capi.Plan.candidates(cands, nf_b).tobytes() == c_b.tobytes()
    plan.close()


def test_async_under_host_fault_injection(capi, monkeypatch):
    """FDAS_FAULT=capacity (a one-record store) and nan_input reach the
    stream-ordered call's device-side status like the blocking call's."""
    n = 1 << 14
    x = torch.from_numpy(_batch(n, 1, seed=50)[0]).cuda()
    plan = capi.Plan(n, 64e-6, 8.0, 2.0, 2048, 2)
    st0, c0, nf0 = plan.search([x], capacity=256)
    assert st0 == capi.FDAS_OK and nf0 > 1
    monkeypatch.setenv("FDAS_FAULT", "capacity")
    st, c, nf = _run_async(capi, plan, [x], None, 256)
    assert st == capi.FDAS_ERR_CAND_STORE_FULL and nf == nf0 and len(c) == 0
    monkeypatch.setenv("FDAS_FAULT", "nan_input")
    st, c, nf = _run_async(capi, plan, [x], None, 256)
    assert st == capi.FDAS_ERR_NONFINITE and nf == 0
    monkeypatch.delenv("FDAS_FAULT")
    st, c, nf = _run_async(capi, plan, [x], None, 256)
    assert st == capi.FDAS_OK and c.tobytes() == c0.tobytes()
    plan.close()
