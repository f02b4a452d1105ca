"""fdas_spectrum_static: the spectrum entry point that allocates nothing.

It exists for callers that may not allocate device memory when they call in
(code running while a stream is captured into a CUDA graph, or a real-time
pipeline that reserves all of its GPU memory up front).  Its FFT
intermediates live in a fixed array inside the library, so its output must
equal what the planned entry point fdas_spectrum produces, call after call,
even though every call reuses the same array.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

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
    plan.close()


def test_static_spectrum_rejects_series_beyond_its_limit(capi):
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_spectrum_static(ctypes.c_void_p(16), 1 << 21, 0, 0, 2048, ctypes.c_void_p(16))
    assert ei.value.status == capi.FDAS_ERR_ARG
    assert "2^20" in str(ei.value)
