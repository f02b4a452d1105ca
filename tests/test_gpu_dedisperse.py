"""Dedispersion (upstream of the search) through the C ABI against the oracle.

* delay table: bit-exact (both sides evaluate the same FP64 expression with
  one IEEE rounding per operation, then floor(x + 1/2)).
* dedispersed series: FP32 sums of n_chan terms in channel order against the
  FP64 sum: |out - ref| <= (n_chan - 1) 2^-24 sum_c |in| (the recursive-
  summation bound), checked per sample with the oracle's sum of |in|.
* 8-bit filterbanks: integer sums, so the series equal the oracle's exactly.
"""
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


@pytest.mark.parametrize("n_chan,f_top,df,tsamp,dm_lo,dm_step,n_dm", [
    (64, 1500.0, 4.0, 64e-6, 0.0, 2.0, 37),
    (4096, 1670.0, 0.125, 64e-6, 0.0, 0.5, 128),     # a wide band in fine channels
    (300, 350.0, 0.2, 256e-6, 10.0, 0.25, 16),      # low frequency, large delays
    (1, 1400.0, 1.0, 64e-6, 0.0, 1.0, 5),           # one channel: no delays
])
def test_delay_table_is_bit_exact(capi, n_chan, f_top, df, tsamp, dm_lo, dm_step, n_dm):
    n_t = 1 << 22
    plan = capi.DedispPlan(n_chan, n_t, f_top, df, tsamp, dm_lo, dm_step, n_dm, 1 << 20)
    got = plan.delays()
    ref = O.dm_delays(n_chan, f_top, df, tsamp, dm_lo, dm_step, n_dm)
    assert got.shape == ref.shape
    assert np.array_equal(got.astype(np.int64), ref)
    assert plan.info.max_delay == ref.max()
    plan.close()


def _case(capi, n_chan, n_t, n_out, f_top, df, tsamp, dm_lo, dm_step, n_dm, seed, pulse_dm=None,
          t0=100):
    delays = O.dm_delays(n_chan, f_top, df, tsamp, dm_lo, dm_step, n_dm)
    fb = S.filterbank_noise(n_chan, n_t, seed)
    if pulse_dm is not None:
        fb = S.add_at_samples(fb, t0 + delays[pulse_dm], 8.0)
    plan = capi.DedispPlan(n_chan, n_t, f_top, df, tsamp, dm_lo, dm_step, n_dm, n_out)
    out = plan.dedisperse(torch.from_numpy(fb).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = O.dedisperse(fb.astype(np.float64), delays, n_out)
    bound = O.dedisperse(np.abs(fb.astype(np.float64)), delays, n_out) * (n_chan - 1) * 2.0 ** -24
    plan.close()
    return got, ref, bound


@pytest.mark.parametrize("n_chan,n_t,n_out,f_top,df,tsamp,dm_lo,dm_step,n_dm", [
    (64, 20000, 17000, 1500.0, 4.0, 64e-6, 0.0, 2.0, 37),     # ragged DM tile and time tile
    (96, 8192, 8192, 1400.0, 2.0, 64e-6, 0.0, 5.0, 16),       # n_out = n_t: zeros past the end
    (1, 3000, 2999, 1400.0, 1.0, 64e-6, 0.0, 1.0, 3),         # one channel
    (40, 60000, 4096, 400.0, 1.0, 64e-6, 0.0, 10.0, 20),      # wide delay spread (1 channel/batch)
    (512, 1 << 15, 1 << 14, 1530.0, 0.5, 64e-6, 3.0, 1.0, 48),
])
def test_dedisperse_matches_oracle(capi, n_chan, n_t, n_out, f_top, df, tsamp, dm_lo, dm_step,
                                   n_dm):
    got, ref, bound = _case(capi, n_chan, n_t, n_out, f_top, df, tsamp, dm_lo, dm_step, n_dm, 17)
    assert got.shape == ref.shape == (n_dm, n_out)
    excess = np.abs(got - ref) - bound
    assert excess.max() <= 1e-6, (excess.max(), np.unravel_index(np.argmax(excess), excess.shape))


def test_dispersed_pulse_lands_at_its_dm(capi):
    n_chan, k, t0 = 256, 29, 777
    got, ref, _ = _case(capi, n_chan, 1 << 15, 1 << 14, 1450.0, 1.0, 64e-6, 0.0, 3.0, 48, 23,
                        pulse_dm=k, t0=t0)
    assert np.unravel_index(np.argmax(got), got.shape) == (k, t0)
    assert got[k, t0] > 8.0 * n_chan - 6.0 * np.sqrt(n_chan)


def test_dedispersed_rows_feed_the_search(capi):
    """Rows of the dedispersion output are searched in place (device views)
    and give the oracle's candidates."""
    n_chan, n_out = 16, 1 << 14
    dd = capi.DedispPlan(n_chan, n_out + 4096, 1400.0, 2.0, 64e-6, 0.0, 10.0, 4, n_out)
    fb = S.filterbank_noise(n_chan, n_out + 4096, 5)
    # a sinusoid common to every channel survives dedispersion at DM 0
    u = np.arange(n_out + 4096) / n_out
    fb += (0.05 * np.cos(2 * np.pi * 3000.3 * u)).astype(np.float32)[None, :]
    out = dd.dedisperse(torch.from_numpy(fb).cuda())
    plan = capi.Plan(n_out, 64e-6, 8.0, 2.0, 1024, 4)
    st, cands, nf = plan.search([out[d] for d in range(4)], capacity=1 << 16)
    assert st == capi.FDAS_OK
    rows = out.cpu().numpy()
    for d in range(4):
        ref = O.search(rows[d], 8.0, 2.0, 4, guard=1e-4)
        mine = cands[cands["trial_id"] == d]
        keys = {(int(h), int(z), int(r)) for h, z, r in zip(mine["harm"], mine["iz"], mine["ir"])}
        rkeys = {(int(h), int(z), int(r)) for h, z, r in
                 zip(ref["candidates"]["harm"], ref["candidates"]["iz"], ref["candidates"]["ir"])}
        gd = {(int(h), int(z), int(r)) for h, z, r in
              zip(ref["guard"]["harm"], ref["guard"]["iz"], ref["guard"]["ir"])}
        assert not ((keys ^ rkeys) - gd)
    assert any(int(r) == 3000 for r in cands["ir"][cands["trial_id"] == 0])
    plan.close()
    dd.close()


@pytest.mark.parametrize("n_chan,n_t,n_out,f_top,df,tsamp,dm_lo,dm_step,n_dm", [
    (64, 20000, 17000, 1500.0, 4.0, 64e-6, 0.0, 2.0, 37),     # ragged DM tile and time tile
    (96, 8192, 8192, 1400.0, 2.0, 64e-6, 0.0, 5.0, 16),       # n_out = n_t: zeros past the end
    (40, 60000, 4096, 400.0, 1.0, 64e-6, 0.0, 10.0, 20),      # wide delay spread (1 channel/batch)
    (1024, 1 << 15, 1 << 14, 1670.0, 0.25, 64e-6, 0.0, 0.25, 70),
])
def test_dedisperse_u8_is_exact(capi, n_chan, n_t, n_out, f_top, df, tsamp, dm_lo, dm_step, n_dm):
    delays = O.dm_delays(n_chan, f_top, df, tsamp, dm_lo, dm_step, n_dm)
    fb = S.filterbank_u8(n_chan, n_t, 29)
    plan = capi.DedispPlan(n_chan, n_t, f_top, df, tsamp, dm_lo, dm_step, n_dm, n_out)
    got = plan.dedisperse(torch.from_numpy(fb).cuda()).cpu().numpy().astype(np.float64)
    ref = O.dedisperse(fb.astype(np.float64), delays, n_out)
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    plan.close()


def test_dedisperse_u8_pulse_and_validation(capi):
    n_chan, k, t0 = 128, 11, 555
    delays = O.dm_delays(n_chan, 1450.0, 2.0, 64e-6, 0.0, 4.0, 32)
    fb = S.add_at_samples(S.filterbank_u8(n_chan, 1 << 14, 3), t0 + delays[k], 100)
    plan = capi.DedispPlan(n_chan, 1 << 14, 1450.0, 2.0, 64e-6, 0.0, 4.0, 32, 1 << 13)
    out = plan.dedisperse(torch.from_numpy(fb).cuda()).cpu().numpy()
    assert np.unravel_index(np.argmax(out), out.shape) == (k, t0)
    plan.close()
    # 8-bit rows must be 16-byte aligned: n_t a multiple of 16
    odd = capi.DedispPlan(4, 1000, 1400.0, 1.0, 64e-6, 0.0, 1.0, 2, 500)
    with pytest.raises(capi.FdasError) as ei:
        odd.dedisperse(torch.zeros((4, 1000), dtype=torch.uint8, device="cuda"))
    assert ei.value.status == capi.FDAS_ERR_ARG
    odd.close()
