"""fdas_spectrum_static: the spectrum entry point that allocates nothing.

It exists for callers that may not allocate device memory when they call in
(a real-time pipeline that reserves all of its GPU memory up front and
forbids allocation afterwards, or a host whose device memory is handed out by
another allocator that must not be bypassed).  Its FFT intermediates live in
a fixed array inside the library, so its output must equal what the planned
entry point fdas_spectrum produces, and what the FP64 oracle computes from the
definition, call after call, even though every call reuses the same array;
and the device's free memory must not change across calls.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
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
    return c


def _cplx(t):
    a = t.float().cpu().numpy().astype(np.float64)
    return a[0::2] + 1j * a[1::2]


@pytest.mark.parametrize("n,prec", [(1 << 20, 0), (1 << 14, 1)])
def test_static_spectrum_matches_planned_spectrum_on_consecutive_calls(capi, n, prec):
    plan = capi.Plan(n, 64e-6, 8.0, 1.0, 1024, 4, precision=prec)
    dtype = plan.spec_dtype
    nb = max(1, (n // 2) // min(2048, n // 2))
    for call, seed in enumerate((101, 202)):
        x = torch.from_numpy(S.sinusoid_series(n=n, seed=seed, r0=0.2 * n / 2 + 0.3,
                                               z0=3.0, amp=0.1)).cuda()
        ref, ref_med = plan.spectrum(x, medians=True)
        out = torch.empty(n, dtype=dtype, device="cuda")
        med = torch.empty(nb, dtype=torch.float32, device="cuda")
        capi.fdas_spectrum_static(ctypes.c_void_p(x.data_ptr()), n, prec, capi.FDAS_NORM_MEDIAN,
                                  2048, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(med.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        a, b = _cplx(out), _cplx(ref)
        rms = math.sqrt(np.mean(np.abs(b) ** 2))
        # the tolerance the spectrum parity tests use
        assert np.max(np.abs(a - b)) <= 3e-5 * rms + 2e-6 * np.max(np.abs(b)), call
        assert np.allclose(med.cpu().numpy(), ref_med.cpu().numpy(), rtol=2e-5, atol=0), call
        # and against the FP64 oracle directly: FP32 butterflies as in the
        # spectrum parity test, plus the 16-bit rounding of each component
        # (relative 2^-9) when the output is BF16
        Xn, meds = O.normalise(O.spectrum(x.cpu().numpy()), 2048)
        rms_o = math.sqrt(np.mean(np.abs(Xn) ** 2))
        bound = 3e-5 * rms_o + 2e-6 * np.max(np.abs(Xn))
        if prec != 0:
            bound = bound + 2.0 ** -8 * np.abs(Xn)
        assert np.all(np.abs(a - Xn) <= bound), call
        assert np.max(np.abs(med.cpu().numpy() / meds - 1)) < 2e-5, call
    plan.close()


def test_static_spectrum_allocates_no_device_memory(capi):
    """After the first call (which looks up the fixed array's address), calls
    leave the device's free memory exactly as it was."""
    n = 1 << 18
    x = torch.from_numpy(S.white_noise(n, 7)).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        capi.fdas_spectrum_static(ctypes.c_void_p(x.data_ptr()), n, 0, capi.FDAS_NORM_MEDIAN,
                                  2048, ctypes.c_void_p(out.data_ptr()), None, stream)

    call()
    first = out.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        call()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)   # the same input gives the same bits


def test_static_spectrum_rejects_series_beyond_its_limit(capi):
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_spectrum_static(ctypes.c_void_p(16), 1 << 21, 0, 0, 2048, ctypes.c_void_p(16))
    assert ei.value.status == capi.FDAS_ERR_ARG
    assert "2^20" in str(ei.value)
