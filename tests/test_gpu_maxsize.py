"""The largest series a plan takes: 2^24 samples (2^23 bins), 193 templates
(z in [-96, 96] step 1), 8192-bin segments, 16 harmonics.

* The FP32 spectrum and its block medians against the FP64 oracle over all
  2^23 bins (the FFT bound of the spectrum tests).
* A BF16 search (tensor-core correlation, the benchmark's path) of one series
  with an injected sinusoid: the signal is found, and every candidate's
  harmonic sum is recomputed by the oracle one gathered cell at a time from
  the series' own spectrum, within the paper's 3%.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 1 << 24
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
def series():
    x, (r0, z0) = S.batch_series(3, n=N)
    return x, r0, z0


def _cplx(t):
    a = t.float().cpu().numpy().astype(np.float64)
    return a[0::2] + 1j * a[1::2]


def test_maxsize_spectrum_matches_oracle(capi, series):
    x, _, _ = series
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, precision=capi.FDAS_FP32)
    spec, med = plan.spectrum(torch.from_numpy(x).cuda(), medians=True)
    got = _cplx(spec)
    Xn, meds = O.normalise(O.spectrum(x), 2048)
    rms = math.sqrt(np.mean(np.abs(Xn) ** 2))
    err = np.max(np.abs(got - Xn))
    assert err <= 3e-5 * rms + 2e-6 * np.max(np.abs(Xn)), (err, rms)
    assert np.max(np.abs(med.cpu().numpy() / meds - 1)) < 2e-5
    plan.close()


def test_maxsize_bf16_candidates_recomputed_by_oracle(capi, series):
    x, r0, z0 = series
    plan = capi.Plan(N, 64e-6, Z_MAX, Z_STEP, L, H, precision=capi.FDAS_BF16)
    assert plan.info.n_r == N // 2 and plan.info.n_z == 193
    st, c, nf = plan.search([torch.from_numpy(x).cuda()], capacity=1 << 16)
    assert st == capi.FDAS_OK and nf == len(c) and nf > 0
    g = O.geometry(N, Z_MAX, Z_STEP, H)
    # the injected sinusoid: a stage-1 candidate within a bin and a drift step
    iz_sig = g.iz0 + int(round(z0 / Z_STEP))
    one = c[c["harm"] == 1]
    assert np.any((np.abs(one["ir"].astype(np.int64) - int(round(r0))) <= 1) &
                  (np.abs(one["iz"].astype(np.int64) - iz_sig) <= 1)), (r0, z0)
    # every candidate's harmonic sum from its gathered cells, one direct sum each
    bank = O.template_bank(g)
    Xn, _ = O.normalise(O.spectrum(x), 2048)
    cells, owners = [], []
    for n, (h, iz, ir) in enumerate(zip(c["harm"], c["iz"], c["ir"])):
        for k in range(1, int(h) + 1):
            cells.append(O.harmonic_indices(int(ir), int(iz), g.iz0, H, k * (H // int(h))))
            owners.append(n)
    cells = np.array(cells)
    pw = O.cell_powers(Xn, bank, cells[:, 0], cells[:, 1])
    s_ora = np.bincount(np.array(owners), weights=pw, minlength=len(c))
    rel = np.abs(c["power"] / s_ora - 1)
    assert rel.max() <= 0.03, rel.max()
    plan.close()
