"""Refinement: the Fourier-interpolated power P(r, z), its gradients and the
ascent, against the FP64 oracle.

Tolerances: P in FP32 with 512-node quadrature -> 2e-4 relative to
max(P, 1); dP/dr and dP/dz against central differences of the FP64 oracle
(step 1e-4, away from window changes) -> 2e-3 relative to max(|g|, P);
dP/dX (PyTorch convention dP/dRe + i dP/dIm) against central differences
in Re/Im X_k -> 2e-3 relative to max |grad|; the ascent lands within 0.02 bin
in r and 0.2 in z of a noise-free injected signal (config: 50 steps).
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 1 << 15   # N_r = 16384 bins


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    O.build()
    return c


@pytest.fixture(scope="module")
def plan(capi):
    p = capi.Plan(N, 64e-6, 16.0, 1.0, 1024, 4)
    yield p
    p.close()


def _injected(signals, noise_seed=None):
    """Spectrum c rho(r0 - k, z0) summed over signals (+ normalised noise)."""
    n_r = N // 2
    X = np.zeros(n_r, dtype=np.complex128)
    for r0, z0, c in signals:
        w = np.arange(max(0, int(r0) - 200), min(n_r, int(r0) + 200))
        X[w] += c * O.rho(r0 - w, z0)
    if noise_seed is not None:
        Xn, _ = O.normalise(O.spectrum(S.white_noise(N, noise_seed)), 2048)
        X = X + Xn
    X[0] = 0
    return X


def _dev(X):
    return torch.from_numpy(X.astype(np.complex64)).cuda()


def _points(rng, n, n_r, avoid_jumps=False):
    pts = []
    while len(pts) < n:
        r = rng.uniform(1.0, n_r - 2.0)
        z = rng.uniform(-90.0, 90.0)
        if avoid_jumps:
            fr = r - math.floor(r)
            hz = abs(z) / 2 - math.floor(abs(z) / 2)
            if not (0.1 < fr < 0.4 or 0.6 < fr < 0.9) or not (0.05 < hz < 0.95):
                continue
        pts.append((r, z))
    return np.array(pts)


def test_fourier_power_matches_oracle(plan):
    X = _injected([(3000.4, 20.3, 6.0), (9000.7, -55.1, 4.0)], noise_seed=5)
    rng = np.random.default_rng(0)
    pts = np.concatenate([_points(rng, 40, N // 2),
                          [[3000.4, 20.3], [9000.7, -55.1], [3.2, 10.0], [N // 2 - 3.4, -30.0]]])
    P, _ = plan.fourier_power(_dev(X), torch.from_numpy(pts).cuda())
    P = P.cpu().numpy()
    for (r, z), p in zip(pts, P):
        ref, _ = O.fourier_power(X, r, z)
        assert abs(p - ref) <= 2e-4 * max(ref, 1.0), (r, z, p, ref)


def test_rz_gradients_match_fp64_finite_differences(plan):
    X = _injected([(3000.4, 20.3, 6.0)], noise_seed=6)
    rng = np.random.default_rng(1)
    pts = np.concatenate([_points(rng, 12, N // 2, avoid_jumps=True),
                          [[3000.25, 20.3], [3000.7, 21.1], [2999.8, 19.4]]])
    _, g = plan.fourier_power(_dev(X), torch.from_numpy(pts).cuda())
    g = g.cpu().numpy()
    h = 1e-4
    for (r, z), (gr, gz) in zip(pts, g):
        P0, _ = O.fourier_power(X, r, z)
        fr = (O.fourier_power(X, r + h, z)[0] - O.fourier_power(X, r - h, z)[0]) / (2 * h)
        fz = (O.fourier_power(X, r, z + h)[0] - O.fourier_power(X, r, z - h)[0]) / (2 * h)
        assert abs(gr - fr) <= 2e-3 * max(abs(fr), P0, 1.0), (r, z, gr, fr)
        assert abs(gz - fz) <= 2e-3 * max(abs(fz), P0, 1.0), (r, z, gz, fz)


def test_spectrum_gradient_matches_finite_differences(capi, plan):
    X = _injected([(5000.3, -12.7, 5.0)], noise_seed=7)
    pts = np.array([[5000.3, -12.7], [5000.9, -13.3]])
    Xd = _dev(X)
    spec = torch.view_as_real(Xd)
    gP = torch.tensor([1.0, 0.5], dtype=torch.float32, device="cuda")
    grad = torch.zeros_like(Xd)
    grz = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    rz = torch.from_numpy(pts).cuda()
    import ctypes
    capi.fdas_fourier_power_backward(
        plan.handle, ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(rz.data_ptr()), 2,
        ctypes.c_void_p(gP.data_ptr()), ctypes.c_void_p(torch.view_as_real(grad).data_ptr()),
        ctypes.c_void_p(grz.data_ptr()))
    torch.cuda.synchronize()
    grad = grad.cpu().numpy().astype(np.complex128)
    X32 = X.astype(np.complex64).astype(np.complex128)

    def loss(Xv):
        return O.fourier_power(Xv, *pts[0])[0] + 0.5 * O.fourier_power(Xv, *pts[1])[0]

    scale = np.max(np.abs(grad))
    eps = 1e-3
    for k in (4960, 4990, 5000, 5001, 5012, 5040):
        Xp, Xm = X32.copy(), X32.copy()
        Xp[k] += eps
        Xm[k] -= eps
        d_re = (loss(Xp) - loss(Xm)) / (2 * eps)
        Xp, Xm = X32.copy(), X32.copy()
        Xp[k] += 1j * eps
        Xm[k] -= 1j * eps
        d_im = (loss(Xp) - loss(Xm)) / (2 * eps)
        assert abs(grad[k] - (d_re + 1j * d_im)) <= 2e-3 * scale, (k, grad[k], d_re, d_im)
    # outside both windows nothing is added
    assert np.all(grad[:4000] == 0) and np.all(grad[6000:] == 0)
    # grad_rz = gP * (dP/dr, dP/dz)
    _, g = plan.fourier_power(Xd, rz)
    assert np.allclose(grz.cpu().numpy(), gP.cpu().numpy()[:, None] * g.cpu().numpy(), rtol=1e-5)


def test_autograd_function(capi, plan):
    X = _injected([(7000.6, 33.2, 5.0)], noise_seed=8)
    Xd = _dev(X).requires_grad_(True)
    rz = torch.tensor([[7000.6, 33.2], [7001.2, 32.0]], dtype=torch.float64, device="cuda",
                      requires_grad=True)
    P = capi.FourierPower().apply(plan, Xd, rz)
    (P * torch.tensor([1.0, 2.0], device="cuda")).sum().backward()
    assert Xd.grad is not None and rz.grad is not None
    _, g = plan.fourier_power(Xd.detach(), rz.detach())
    want = torch.tensor([1.0, 2.0], device="cuda", dtype=torch.float64)[:, None] * g.double()
    assert torch.allclose(rz.grad, want, rtol=1e-5)
    # the spectrum gradient of P_0 at its centre bin against a finite difference
    k = 7001
    X32 = X.astype(np.complex64).astype(np.complex128)

    def loss(Xv):
        return (O.fourier_power(Xv, 7000.6, 33.2)[0] + 2 * O.fourier_power(Xv, 7001.2, 32.0)[0])

    eps = 1e-3
    Xp, Xm = X32.copy(), X32.copy()
    Xp[k] += eps
    Xm[k] -= eps
    d_re = (loss(Xp) - loss(Xm)) / (2 * eps)
    g_k = Xd.grad[k].item()
    assert abs(g_k.real - d_re) <= 2e-3 * Xd.grad.abs().max().item()


def test_refine_converges_to_injected_signals(capi, plan):
    sig = [(1200.37, 17.6), (4100.81, -48.3), (8300.12, 71.9), (12000.55, -3.4)]
    X = _injected([(r, z, 8.0) for r, z in sig])
    seeds = np.zeros(len(sig), dtype=capi.SEED_DTYPE)
    seeds["r"] = [round(r) for r, _ in sig]
    seeds["z"] = [round(z) for _, z in sig]
    seeds["trial_id"] = np.arange(len(sig))
    P0, _ = plan.fourier_power(_dev(X), torch.from_numpy(
        np.stack([seeds["r"], seeds["z"]], 1)).cuda())
    out = plan.refine(_dev(X), seeds, n_steps=50)
    for (r0, z0), o, p0 in zip(sig, out, P0.cpu().numpy()):
        assert abs(o["r"] - r0) < 0.02 and abs(o["z"] - z0) < 0.2, (r0, z0, o)
        assert o["power"] >= p0 and o["steps"] > 0
        ref, _ = O.fourier_power(X, o["r"], o["z"])
        assert abs(o["power"] - ref) <= 2e-4 * ref
    assert list(out["trial_id"]) == [0, 1, 2, 3]


def test_refine_4096_seeds_from_search_candidates(capi):
    """Seeds: the distinct candidate cells of the 2^23-sample, 193-template
    pulsar search (any stage), up to 4096."""
    n = 1 << 23
    x, params = S.pulsar_series(n, seed=2)
    plan = capi.Plan(n, 64e-6, 96.0, 1.0, 8192, 16)
    xd = torch.from_numpy(x).cuda()
    st, cands, nf = plan.search([xd], capacity=1 << 18)
    cells = np.unique(np.stack([cands["ir"], cands["iz"]], 1), axis=0)[:4096]
    assert len(cells) > 100
    seeds = np.zeros(len(cells), dtype=capi.SEED_DTYPE)
    seeds["r"] = cells[:, 0].astype(np.float64)
    seeds["z"] = (cells[:, 1].astype(np.float64) - plan.info.iz0) * plan.info.z_step
    spec = plan.spectrum(xd)                       # FP32 plan: float pairs
    X = torch.view_as_complex(spec.view(-1, 2))
    P0, _ = plan.fourier_power(X, torch.from_numpy(np.stack([seeds["r"], seeds["z"]], 1)).cuda())
    out = plan.refine(X, seeds, n_steps=50)
    assert np.all(np.isfinite(out["power"]))
    assert np.all(out["power"] >= P0.cpu().numpy())
    Xh = X.cpu().numpy().astype(np.complex128)
    for o in out[:: max(1, len(out) // 8)]:
        ref, _ = O.fourier_power(Xh, o["r"], o["z"])
        assert abs(o["power"] - ref) <= 2e-4 * max(ref, 1.0)
    plan.close()
