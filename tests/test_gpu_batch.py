"""Uneven batches (series decimated by powers of two in one call), CUDA-graph
replay of a batch, and the autotuned plan, against the FP64 oracle.

A series decimated by 2^d covers the same observation with N/2^d samples, so
it is searched over the same z grid with N/2^(d+1) bins; every series' list
must equal the oracle's for that series (FP32: outside a 1e-4 guard band;
BF16/FP16: outside a 3% guard band, powers within 3%).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NMAX = 1 << 16
ZMAX, ZSTEP, L, H = 16.0, 2.0, 2048, 4


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    O.build()
    return c


def _series(n, i):
    r0 = 0.21 * n / 2 + 0.3 + 17 * i
    return S.sinusoid_series(n=n, seed=40 + i, r0=r0, z0=5.0 - 2 * i, amp=0.25 * np.sqrt(NMAX / n))


@pytest.fixture(scope="module")
def uneven():
    lengths = [NMAX, NMAX // 8, NMAX // 2, NMAX, NMAX // 4, NMAX // 2, NMAX // 8]
    xs = [_series(n, i) for i, n in enumerate(lengths)]
    ids = [10 * i + 3 for i in range(len(xs))]
    refs = {}
    for g in (1e-4, 0.03):
        refs[g] = [O.search(x, ZMAX, ZSTEP, H, trial=t, guard=g) for x, t in zip(xs, ids)]
    return lengths, xs, ids, refs


def _check(got, refs, guard, rel_power):
    ref = np.concatenate([r["candidates"] for r in refs])
    gd = {(int(t), int(h), int(z), int(r)) for r in refs
          for t, h, z, r in zip(r["guard"]["trial"], r["guard"]["harm"], r["guard"]["iz"], r["guard"]["ir"])}
    gk = {(int(t), int(h), int(z), int(r)): float(p) for t, h, z, r, p in
          zip(got["trial_id"], got["harm"], got["iz"], got["ir"], got["power"])}
    rk = {(int(t), int(h), int(z), int(r)): float(p) for t, h, z, r, p in
          zip(ref["trial"], ref["harm"], ref["iz"], ref["ir"], ref["power"])}
    assert not ((set(gk) ^ set(rk)) - gd), sorted((set(gk) ^ set(rk)) - gd)[:10]
    common = set(gk) & set(rk)
    assert common and max(abs(gk[k] / rk[k] - 1) for k in common) <= rel_power
    # every series contributes (each holds a strong sinusoid)
    assert {k[0] for k in gk} == {int(r["candidates"]["trial"][0]) for r in refs}


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_uneven_batch_matches_oracle(capi, uneven, prec):
    lengths, xs, ids, refs = uneven
    plan = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, precision=prec)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda() for x in xs], trial_ids=ids)
    assert st == capi.FDAS_OK and nf == len(cands)
    if prec == 0:
        _check(cands, refs[1e-4], 1e-4, 1e-4)
    else:
        _check(cands, refs[0.03], 0.03, 0.03)
    # ordered by (trial_id, harm, iz, ir)
    key = list(zip(cands["trial_id"], cands["harm"], cands["iz"], cands["ir"]))
    assert key == sorted(key)
    plan.close()


def test_batch_rejects_lengths_the_plan_cannot_take(capi):
    plan = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H)
    bad = torch.zeros(NMAX * 2, device="cuda")
    with pytest.raises(capi.FdasError) as ei:
        plan.search([bad])
    assert ei.value.status == capi.FDAS_ERR_ARG
    with pytest.raises(capi.FdasError):
        plan.search([torch.zeros(3 * 1024, device="cuda")])
    plan.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_direct_launches(capi, uneven, prec):
    """FP32 (FFT correlator) and BF16 (tensor-core correlator) batches
    captured into a CUDA graph give the direct launches' candidates."""
    lengths, xs, ids, refs = uneven
    direct = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, precision=prec)
    graph = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, use_graph=True, precision=prec)
    assert graph.info.use_graph == 1
    side = torch.cuda.Stream()
    batches = [[torch.from_numpy(x).cuda() for x in xs],
               [torch.from_numpy(x[::-1].copy()).cuda() for x in xs]]
    for rnd, dev in enumerate(batches * 2):          # capture, then update and replay
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            st_g, cg, nf_g = graph.search(dev, trial_ids=ids, stream=side)
        st_d, cd, nf_d = direct.search(dev, trial_ids=ids)
        assert st_g == st_d == capi.FDAS_OK
        assert nf_g == nf_d and cg.tolist() == cd.tolist(), rnd
    if prec == 0:
        _check(graph.search(batches[0], trial_ids=ids, stream=side)[1], refs[1e-4], 1e-4, 1e-4)
    else:
        _check(graph.search(batches[0], trial_ids=ids, stream=side)[1], refs[0.03], 0.03, 0.03)
    direct.close()
    graph.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_with_interbinning(capi, uneven, prec):
    """The interbinned search (FP32: complex plane + interbinning kernel;
    BF16: the tensor-core epilogue and its fix-up kernel) captured into a
    CUDA graph gives the direct launches' candidates, decimated series
    included."""
    lengths, xs, ids, refs = uneven
    direct = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, precision=prec, interbin=True)
    graph = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, use_graph=True, precision=prec,
                      interbin=True)
    side = torch.cuda.Stream()
    dev = [torch.from_numpy(x).cuda() for x in xs]
    for rnd in range(2):
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            st_g, cg, nf_g = graph.search(dev, trial_ids=ids, stream=side)
        st_d, cd, nf_d = direct.search(dev, trial_ids=ids)
        assert st_g == st_d == capi.FDAS_OK and nf_d > 0
        assert nf_g == nf_d and cg.tolist() == cd.tolist(), rnd
    direct.close()
    graph.close()


def test_uneven_batch_fundamental_harmonic(capi, uneven):
    """The fundamental-indexed harmonic sum on decimated series (each series
    its own N_r and domain), BF16 storage, against the oracle."""
    lengths, xs, ids, _ = uneven
    refs = [O.search(x, ZMAX, ZSTEP, H, trial=t, guard=0.03, harmonic_mode=O.FUNDAMENTAL)
            for x, t in zip(xs, ids)]
    plan = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, precision=capi.FDAS_BF16,
                     harmonic_mode=capi.FDAS_HARM_FUNDAMENTAL)
    st, cands, nf = plan.search([torch.from_numpy(x).cuda() for x in xs], trial_ids=ids)
    assert st == capi.FDAS_OK and nf == len(cands)
    _check(cands, refs, 0.03, 0.03)
    plan.close()


def test_autotuned_plan(capi, uneven):
    lengths, xs, ids, refs = uneven
    plan = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, autotune=True)
    info = plan.info
    assert info.seg_len in (2048, 4096, 8192) and info.tuned_ms > 0 and info.z_chunks >= 1
    st, cands, nf = plan.search([torch.from_numpy(x).cuda() for x in xs], trial_ids=ids)
    _check(cands, refs[1e-4], 1e-4, 1e-4)
    plan.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_uneven_batch_from_host_memory(capi, uneven, prec):
    """The same uneven batch from page-locked host memory (copied by the
    library's copy kernel), from pageable host memory (cudaMemcpyAsync) and
    from device memory: identical records, in both search calls."""
    lengths, xs, ids, refs = uneven
    plan = capi.Plan(NMAX, 64e-6, ZMAX, ZSTEP, L, H, precision=prec)
    dev = [torch.from_numpy(x).cuda() for x in xs]
    pinned = [torch.from_numpy(x).pin_memory() for x in xs]
    pageable = [torch.from_numpy(x).clone() for x in xs]
    st0, c0, n0 = plan.search(dev, trial_ids=ids, capacity=1 << 15)
    assert st0 == capi.FDAS_OK and n0 == len(c0) > 0
    for host in (pinned, pageable):
        st, c, n = plan.search(host, trial_ids=ids, capacity=1 << 15)
        assert st == capi.FDAS_OK and c.tobytes() == c0.tobytes()
        cands = torch.zeros((1 << 15) * 20, dtype=torch.uint8, device="cuda")
        nf = torch.zeros(1, dtype=torch.int64, device="cuda")
        sa = torch.zeros(1, dtype=torch.int32, device="cuda")
        plan.search_async(host, cands, nf, sa, trial_ids=ids)
        torch.cuda.synchronize()
        assert int(sa.cpu()[0]) == capi.FDAS_OK and int(nf.cpu()[0]) == n0
        assert capi.Plan.candidates(cands, n0).tobytes() == c0.tobytes()
    guard, rel = (1e-4, 1e-4) if prec == 0 else (0.03, 0.03)
    _check(c0, refs[guard], guard, rel)
    plan.close()
