"""The bounded-wait failure path on the GPU, without a fault: a barrier
armed for bytes no copy delivers is waited on with a short limit; the wait
gives up, the kernel records it and returns, the call reports
FDAS_ERR_TIMEOUT, and the same plan then searches normally."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 1 << 16


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    return c


def test_wait_gives_up_and_the_plan_stays_usable(capi):
    plan = capi.Plan(N, 64e-6, 16.0, 2.0, 2048, 4)
    x = torch.from_numpy(S.sinusoid_series(n=N, seed=3, r0=4000.3, z0=3.0, amp=0.3)).cuda()
    st0, c0, nf0 = plan.search([x])
    assert st0 == capi.FDAS_OK and nf0 > 0
    for _ in range(2):
        st = capi.fdas_selftest_wait_timeout(plan.handle, 2_000_000)   # about 1 ms
        assert st == capi.FDAS_ERR_TIMEOUT
        assert "gave up" in capi.fdas_last_error()
        torch.cuda.synchronize()                     # the context is intact
        st1, c1, nf1 = plan.search([x])              # flags are reset per call
        assert st1 == capi.FDAS_OK and nf1 == nf0 and c1.tolist() == c0.tolist()
    plan.close()


def test_wait_limit_is_validated(capi):
    plan = capi.Plan(N, 64e-6, 16.0, 2.0, 2048, 4)
    for bad in (0, -5, 3_000_000_000):
        with pytest.raises(capi.FdasError) as ei:
            capi.fdas_selftest_wait_timeout(plan.handle, bad)
        assert ei.value.status == capi.FDAS_ERR_ARG
    plan.close()
