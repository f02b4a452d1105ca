"""Search cases run on both builds of the library.

`run_cases` runs a set of searches and stage calls through whatever library
capi has loaded and returns their outputs as bytes: the ordinary build in the
test process (tests/test_gpu_checked.py), the checked build
(libfdas_checked.so, FDAS_CHECKED=1) in a child process that runs this file as
a script.  The cases cover every checked kernel: the FFT correlator (FP32,
BF16 interbinning), the tensor-core correlation (BF16 in both template
orders, FP16 with interbinning, the FP32 hi/lo split), the top- and the
fundamental-indexed harmonic sums, a decimated series, page-locked host
series replayed as a CUDA graph, the stream-ordered search, more than 8192
records to order, and the stage entry points.

As a script (argument: an output path) it also runs the checked build's fault
injections, FDAS_FAULT=canary and FDAS_FAULT=bounds (blocking, graph replay
and stream-ordered), each followed by a clean search on the same plan, and
saves everything to <path>.npz and <path>.json.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import synthetic as S  # noqa: E402

# (n_samples, Plan keyword arguments, number of series)
CASES = {
    "fp32_fft": (1 << 15, dict(z_max=16.0, z_step=2.0, seg_len=2048, n_harm=4), 3),
    "bf16_tc_paired": (1 << 16, dict(z_max=32.0, z_step=1.0, seg_len=2048, n_harm=16,
                                     precision=1, correlator=2, template_order=2), 3),
    "bf16_tc_z": (1 << 16, dict(z_max=32.0, z_step=1.0, seg_len=2048, n_harm=16,
                                precision=1, correlator=2, template_order=1), 2),
    "fp16_tc_interbin": (1 << 15, dict(z_max=24.0, z_step=2.0, seg_len=2048, n_harm=8,
                                       precision=2, correlator=2, interbin=True), 2),
    "fp32_tc_split": (1 << 15, dict(z_max=16.0, z_step=1.0, seg_len=2048, n_harm=8,
                                    precision=0, correlator=3), 2),
    "bf16_fft_interbin": (1 << 15, dict(z_max=16.0, z_step=2.0, seg_len=2048, n_harm=4,
                                        precision=1, correlator=1, interbin=True), 2),
    "bf16_fundamental": (1 << 16, dict(z_max=32.0, z_step=1.0, seg_len=2048, n_harm=8,
                                       precision=1, harmonic_mode=1), 2),
}


def series(n, k, seed):
    """k seeded series of n samples, each with a bright sinusoid."""
    xs = []
    for i in range(k):
        x, _ = S.batch_series(seed + i, n=n)
        x = (x + S.inject_sinusoid(np.zeros(n, np.float32), 900.0 + 350 * i, 3.0, 0.1))
        xs.append(x.astype(np.float32))
    return xs


def _rec(capi, st, c, nf):
    assert st == capi.FDAS_OK and nf == len(c) and nf > 0, (st, nf)
    return np.frombuffer(c.tobytes(), dtype=np.uint8)


def _u8(t):
    import torch
    return t.contiguous().reshape(-1).view(torch.uint8).cpu().numpy().copy()


def run_cases(capi, torch):
    """name -> uint8 array of the outputs of each search or stage call."""
    out = {}
    for ci, (name, (n, kw, k)) in enumerate(CASES.items()):
        plan = capi.Plan(n, 64e-6, **kw)
        xs = [torch.from_numpy(x).cuda() for x in series(n, k, seed=10 * ci)]
        ids = [5 * i + 1 for i in range(k)][::-1]
        out[name] = _rec(capi, *plan.search(xs, trial_ids=ids, capacity=1 << 15))
        plan.close()
    # a decimated series beside a full one, and the stage entry points
    n = 1 << 16
    plan = capi.Plan(n, 64e-6, 32.0, 1.0, 2048, 16, precision=capi.FDAS_BF16)
    full, = series(n, 1, seed=70)
    half, = series(n // 2, 1, seed=71)
    xs = [torch.from_numpy(full).cuda(), torch.from_numpy(half).cuda()]
    out["decimated"] = _rec(capi, *plan.search(xs, capacity=1 << 15))
    spec = plan.spectrum(xs[0])
    plane, stats = plan.power_plane(spec)
    out["stage_spectrum"] = _u8(spec)
    out["stage_plane"] = _u8(plane)
    out["stage_sums"] = _u8(plan.harmonic_sums(plane))
    out["stage_threshold"] = _rec(capi, *plan.threshold(plane, stats, trial_id=4))
    plan.close()
    # page-locked host series, replayed as a CUDA graph on a side stream
    plan = capi.Plan(1 << 15, 64e-6, 16.0, 2.0, 2048, 4, precision=capi.FDAS_BF16,
                     use_graph=True)
    host = [torch.from_numpy(x).pin_memory() for x in series(1 << 15, 3, seed=80)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for rep in range(2):
            r = plan.search(host, capacity=1 << 15, stream=stream)
            out[f"graph_host_{rep}"] = _rec(capi, *r)
    stream.synchronize()
    plan.close()
    # more than 8192 records (global merge steps of the ordering), blocking
    # and stream-ordered
    n = 1 << 16
    x = S.sinusoid_series(n=n, seed=8, r0=7000.4, z0=4.0, amp=0.1)
    plan = capi.Plan(n, 64e-6, 16.0, 2.0, 2048, 4, threshold_sigma=2.0,
                     threshold_mode=capi.FDAS_THRESH_MEAN_PLUS_KSIGMA)
    xd = torch.from_numpy(x).cuda()
    st, c, nf = plan.search([xd], capacity=1 << 17)
    assert nf > 3 * 8192
    out["many_records"] = _rec(capi, st, c, nf)
    cands = torch.zeros((1 << 17) * 20, dtype=torch.uint8, device="cuda")
    nfd = torch.zeros(1, dtype=torch.int64, device="cuda")
    std = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan.search_async([xd], cands, nfd, std)
    torch.cuda.synchronize()
    assert int(std[0]) == capi.FDAS_OK
    out["many_records_async"] = _u8(cands[:int(nfd[0]) * 20])
    plan.close()
    return out


def _fault(capi, fn):
    """(status, message) of a call made under an injected fault."""
    try:
        fn()
    except capi.FdasError as e:
        return e.status, str(e)
    return capi.FDAS_OK, ""


def run_faults(capi, torch):
    """The checked build's fault injections, each followed by a clean call."""
    res = {}
    n = 1 << 16
    xs = [torch.from_numpy(x).cuda() for x in series(n, 2, seed=90)]
    plan = capi.Plan(n, 64e-6, 32.0, 1.0, 2048, 16, precision=capi.FDAS_BF16, correlator=2)
    clean = _rec(capi, *plan.search(xs, capacity=1 << 15))
    for fault in ("canary", "bounds"):
        os.environ["FDAS_FAULT"] = fault
        res[fault] = _fault(capi, lambda: plan.search(xs, capacity=1 << 15))
        del os.environ["FDAS_FAULT"]
        again = _rec(capi, *plan.search(xs, capacity=1 << 15))
        res[fault + "_then_clean"] = bool(np.array_equal(again, clean))
    # stream-ordered search under the bounds fault
    cands = torch.zeros((1 << 15) * 20, dtype=torch.uint8, device="cuda")
    nfd = torch.zeros(1, dtype=torch.int64, device="cuda")
    std = torch.zeros(1, dtype=torch.int32, device="cuda")
    os.environ["FDAS_FAULT"] = "bounds"
    res["bounds_async"] = _fault(capi, lambda: plan.search_async(xs, cands, nfd, std))
    del os.environ["FDAS_FAULT"]
    torch.cuda.synchronize()
    plan.close()
    # graph replay: the canary written inside the graph is found after it
    plan = capi.Plan(1 << 15, 64e-6, 16.0, 2.0, 2048, 4, precision=capi.FDAS_BF16,
                     use_graph=True)
    xs = [torch.from_numpy(x).cuda() for x in series(1 << 15, 2, seed=95)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        clean = _rec(capi, *plan.search(xs, capacity=1 << 15, stream=stream))
        os.environ["FDAS_FAULT"] = "canary"
        res["canary_graph"] = _fault(capi, lambda: plan.search(xs, capacity=1 << 15,
                                                               stream=stream))
        del os.environ["FDAS_FAULT"]
        again = _rec(capi, *plan.search(xs, capacity=1 << 15, stream=stream))
        res["canary_graph_then_clean"] = bool(np.array_equal(again, clean))
    stream.synchronize()
    plan.close()
    return res


def main(path):
    import importlib

    import torch
    os.environ.pop("FDAS_FAULT", None)
    assert os.environ.get("FDAS_CHECKED") == "1"
    importlib.import_module("paper_2211_13517_gb300.build").build(checked=True)
    from paper_2211_13517_gb300 import capi
    assert capi.fdas_checked_build() and "checked" in capi.fdas_version()
    out = run_cases(capi, torch)
    np.savez(path + ".npz", **out)
    with open(path + ".json", "w") as f:
        json.dump(run_faults(capi, torch), f)


if __name__ == "__main__":
    main(sys.argv[1])
