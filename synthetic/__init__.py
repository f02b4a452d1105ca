"""Seeded synthetic inputs for FDAS (dedispersed time series).

This module only *makes data*: white noise plus injected accelerated signals.
It holds none of the search's arithmetic (no FFT, no templates, no
correlation, no harmonic sums), so both the CUDA path and the FP64 oracle may
draw their inputs from it.

Signal model (the accelerated sinusoid that FDAS is matched to, paper §2.1):
with u = n/N in [0, 1) the phase in cycles is

    phi(u) = r0 * u + z0 * (u - 1/2)^2 / 2

so the instantaneous frequency is r0 + z0 (u - 1/2) Fourier bins: r0 is the
mid-observation frequency and z0 the drift over the observation.

Workload recipes (the SKA-like shapes of paper §3: 600 s at 64 us, 193
acceleration trials; the batch sizes and signal strengths are readings, since
the paper prints none):

* ``sinusoid_series``   -- 2^17 samples, N(0,1) noise seed 1, one sinusoid
                           r0=5000.3, z0=+7.5, amplitude 0.05.
* ``pulsar_series``     -- 2^23 samples, N(0,1) noise, 3 top-hat pulse trains
                           (duty 0.05, height 0.054), r0 ~ U[1e4, 4e6],
                           z0 ~ U[-90, 90], all drawn from the series seed.
* ``filterbank_noise``  -- the input of dedispersion: N(0,1) channels x
                           samples (``filterbank_u8``: 8-bit, N(128, 16^2)
                           rounded and clipped); ``add_at_samples`` plants a
                           pulse at caller-given samples per channel.
* ``batch_series``      -- series i of a batch: seed base+i, one sinusoid of
                           amplitude 0.05*sqrt(2^17/N) (keeps the expected
                           matched-filter power near 82 at any N), r0, z0 drawn
                           as for the pulse trains.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "white_noise",
    "inject_sinusoid",
    "inject_pulse_train",
    "sinusoid_series",
    "pulsar_series",
    "batch_series",
    "draw_signal_params",
    "filterbank_noise",
    "filterbank_u8",
    "add_at_samples",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def white_noise(n: int, seed: int) -> np.ndarray:
    """N(0,1) float32 noise of length n from numpy PCG64(seed)."""
    return _rng(seed).standard_normal(n, dtype=np.float64).astype(np.float32)


def _phase_cycles(n: int, r0: float, z0: float) -> np.ndarray:
    u = np.arange(n, dtype=np.float64) / n
    return r0 * u + z0 * (u - 0.5) ** 2 / 2.0


def inject_sinusoid(x: np.ndarray, r0: float, z0: float, amp: float,
                    phase: float = 0.0) -> np.ndarray:
    """Return x + amp*cos(2*pi*phi(u) + phase) as float32 (phi in FP64)."""
    ph = _phase_cycles(x.shape[0], r0, z0)
    sig = amp * np.cos(2.0 * np.pi * ph + phase)
    return (x.astype(np.float64) + sig).astype(np.float32)


def inject_pulse_train(x: np.ndarray, r0: float, z0: float, duty: float,
                       height: float) -> np.ndarray:
    """Return x + height wherever frac(phi(u)) < duty (top-hat pulses)."""
    ph = _phase_cycles(x.shape[0], r0, z0)
    on = (ph - np.floor(ph)) < duty
    return (x.astype(np.float64) + height * on).astype(np.float32)


def draw_signal_params(seed: int, count: int, r_lo: float = 1e4,
                       r_hi: float = 4e6, z_abs: float = 90.0):
    """Draw `count` (r0, z0) pairs, r0 ~ U[r_lo, r_hi], z0 ~ U[-z_abs, z_abs].

    Uses a generator derived from `seed` but distinct from the noise stream.
    """
    g = _rng(seed + 0x5EED)
    r = g.uniform(r_lo, r_hi, size=count)
    z = g.uniform(-z_abs, z_abs, size=count)
    return list(zip(r.tolist(), z.tolist()))


def sinusoid_series(n: int = 1 << 17, seed: int = 1, r0: float = 5000.3,
                    z0: float = 7.5, amp: float = 0.05) -> np.ndarray:
    """Noise plus one accelerated sinusoid (the 2^17-sample FP32 workload)."""
    return inject_sinusoid(white_noise(n, seed), r0, z0, amp)


def pulsar_series(n: int = 1 << 23, seed: int = 2, n_pulsars: int = 3,
                  duty: float = 0.05, height: float = 0.054,
                  r_lo: float = 1e4, r_hi: float = 4e6, z_abs: float = 90.0):
    """Noise plus `n_pulsars` accelerated top-hat pulse trains.

    Returns (series float32[n], [(r0, z0), ...]).  r_hi is clipped to the
    spectrum length so that small test sizes stay meaningful.
    """
    r_hi = min(r_hi, 0.45 * n)
    r_lo = min(r_lo, 0.1 * r_hi)
    x = white_noise(n, seed)
    params = draw_signal_params(seed, n_pulsars, r_lo, r_hi, z_abs)
    for r0, z0 in params:
        x = inject_pulse_train(x, r0, z0, duty, height)
    return x, params


def batch_series(i: int, n: int = 1 << 23, base_seed: int = 1000,
                 z_abs: float = 90.0):
    """Series i of a DM-trial batch: noise (seed base+i) plus one sinusoid.

    Returns (series float32[n], (r0, z0)).
    """
    seed = base_seed + i
    r_hi = min(4e6, 0.45 * n)
    (r0, z0), = draw_signal_params(seed, 1, min(1e4, 0.1 * r_hi), r_hi, z_abs)
    amp = 0.05 * np.sqrt((1 << 17) / n)
    return inject_sinusoid(white_noise(n, seed), r0, z0, amp), (r0, z0)


def torch_batch_series(count: int, n: int = 1 << 23, base_seed: int = 1000,
                       device="cuda", z_abs: float = 90.0):
    """Device-side batch with the recipe of `batch_series` (for large batches).

    Series i: N(0,1) noise from torch's generator seeded base_seed+i plus one
    sinusoid of amplitude 0.05*sqrt(2^17/n), (r0, z0) drawn by
    draw_signal_params(base_seed+i).  Returns (list of float32 tensors,
    [(r0, z0), ...]).
    """
    import math as _m

    import torch
    out, params = [], []
    r_hi = min(4e6, 0.45 * n)
    amp = 0.05 * _m.sqrt((1 << 17) / n)
    u = torch.arange(n, device=device, dtype=torch.float64) / n
    for i in range(count):
        seed = base_seed + i
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        x = torch.randn(n, generator=g, device=device, dtype=torch.float32)
        (r0, z0), = draw_signal_params(seed, 1, min(1e4, 0.1 * r_hi), r_hi, z_abs)
        ph = r0 * u + z0 * (u - 0.5) ** 2 / 2.0
        x += (amp * torch.cos(2.0 * _m.pi * ph)).to(torch.float32)
        out.append(x)
        params.append((r0, z0))
    return out, params


def filterbank_noise(n_chan: int, n_t: int, seed: int) -> np.ndarray:
    """N(0,1) float32 filterbank [n_chan][n_t] (channel-major) from PCG64(seed)."""
    return _rng(seed).standard_normal((n_chan, n_t), dtype=np.float64).astype(np.float32)


def filterbank_u8(n_chan: int, n_t: int, seed: int, mean: float = 128.0,
                  std: float = 16.0) -> np.ndarray:
    """8-bit filterbank [n_chan][n_t]: rounded N(mean, std^2) from PCG64(seed),
    clipped to [0, 255]."""
    x = _rng(seed).standard_normal((n_chan, n_t), dtype=np.float64) * std + mean
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def add_at_samples(fb: np.ndarray, samples, amp: float) -> np.ndarray:
    """Add `amp` to fb[c, samples[c]] for every channel c (indices given by the
    caller; samples outside [0, n_t) are skipped).  Returns a new array."""
    out = np.array(fb, copy=True)
    for c, t in enumerate(samples):
        if 0 <= int(t) < out.shape[1]:
            if out.dtype == np.uint8:
                out[c, int(t)] = min(255, int(out[c, int(t)]) + int(amp))
            else:
                out[c, int(t)] += out.dtype.type(amp)
    return out
