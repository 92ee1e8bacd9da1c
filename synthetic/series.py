"""Seeded synthetic de-dispersed time series.

Signal convention (the paper prints none; this is the reading the project
uses throughout): an accelerated sinusoid whose *mean* Fourier frequency over
the observation is r0 bins and whose frequency drift is z0 bins,

    x_n += A * cos(2*pi*((r0 - z0/2) * n/N + z0 * n^2 / (2 N^2)) + phi),

so the instantaneous frequency runs linearly from r0 - z0/2 to r0 + z0/2
(z = fdot * T^2, Section 2). Harmonic k of a signal has frequency k*r0,
drift k*z0 and amplitude A/k. "Single-bin SNR s" means that the expected
whitened power at the peak is s^2 for unit-variance noise, i.e.
A = 2 s / sqrt(N).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Chirp:
    r0: float          # mean frequency in bins
    z0: float          # drift in bins over the observation
    snr: float         # single-bin amplitude SNR of the fundamental
    phase: float       # radians
    nharm: int = 1     # number of harmonics injected (amplitude A/k)


def make_series(n: int, seed: int, chirps=(), noise_sigma: float = 1.0,
                dtype=np.float32, noise: bool = True, device=None) -> np.ndarray:
    """Gaussian noise (sigma = noise_sigma) plus the given chirps; with
    noise=False only the chirps (amplitudes still scaled by noise_sigma).

    The noise always comes from numpy's seeded generator; with ``device``
    (a torch device) the float64 chirp sum is evaluated there, which only
    changes the last bits of the float64 sum and is far faster for 2^23
    samples. The returned array is what both the CUDA path and the oracle use.
    """
    rng = np.random.default_rng(seed)
    if noise:
        x = rng.standard_normal(n) * noise_sigma
    else:
        x = np.zeros(n)
    if not chirps:
        return x.astype(dtype)
    if device is not None:
        import torch
        u = torch.arange(n, dtype=torch.float64, device=device) / n
        acc = torch.zeros(n, dtype=torch.float64, device=device)
        for c in chirps:
            amp = 2.0 * c.snr * noise_sigma / math.sqrt(n)
            for k in range(1, c.nharm + 1):
                rk, zk = k * c.r0, k * c.z0
                cyc = (rk - zk / 2.0) * u + zk * u * u / 2.0
                cyc = cyc - torch.floor(cyc)
                acc += (amp / k) * torch.cos(2.0 * math.pi * cyc + c.phase)
        x = x + acc.cpu().numpy()
        return x.astype(dtype)
    idx = np.arange(n, dtype=np.float64)
    u = idx / n
    for c in chirps:
        amp = 2.0 * c.snr * noise_sigma / math.sqrt(n)
        for k in range(1, c.nharm + 1):
            rk, zk = k * c.r0, k * c.z0
            # cycles, reduced mod 1 before scaling by 2*pi
            cyc = (rk - zk / 2.0) * u + zk * u * u / 2.0
            cyc -= np.floor(cyc)
            x += (amp / k) * np.cos(2.0 * np.pi * cyc + c.phase)
    return x.astype(dtype)


def random_chirps(rng: np.random.Generator, count: int, n: int, zmax: float,
                  snr_range=(8.0, 20.0), max_harm: int = 8,
                  r_range=(1.0e4, 4.0e6)) -> list:
    r_hi = min(r_range[1], 0.45 * n)
    out = []
    for _ in range(count):
        out.append(Chirp(r0=float(rng.uniform(r_range[0], r_hi)),
                         z0=float(rng.uniform(-zmax, zmax)),
                         snr=float(rng.uniform(*snr_range)),
                         phase=float(rng.uniform(0.0, 2.0 * np.pi)),
                         nharm=int(rng.integers(1, max_harm + 1))))
    return out


def snap_235(n: float, min_pow2: int = 12) -> int:
    """Largest 2^a 3^b 5^c <= n with a >= min_pow2 (uneven series lengths)."""
    best = 1 << min_pow2
    limit = int(n)
    p2 = 1 << min_pow2
    while p2 <= limit:
        p3 = p2
        while p3 <= limit:
            p5 = p3
            while p5 <= limit:
                best = max(best, p5)
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best


# Workloads. Sizes follow the SKA-shaped configurations: 2^17 and 2^23
# samples; templates every dz = 2 drift bins out to |z| <= zmax; template
# width m and segment length L as listed.
WORKLOADS = {
    "cfg1_n2e17_z50": dict(N=1 << 17, zmax=50, dz=2, m=128, L=2048, nharm=1,
                           sigma=6.0, seed=1),
    "cfg2_n2e23_z200": dict(N=1 << 23, zmax=200, dz=2, m=512, L=8192, nharm=16,
                            sigma=6.0, seed=2),
}


def workload(name: str, seed: int | None = None, device=None):
    """(series float32, params dict) for a named workload."""
    p = dict(WORKLOADS[name])
    if seed is not None:
        p["seed"] = seed
    n = p["N"]
    if name.startswith("cfg1"):
        rng = np.random.default_rng(p["seed"] + 1000)
        chirps = [Chirp(r0=10000.3, z0=35.0, snr=8.0,
                        phase=float(rng.uniform(0.0, 2.0 * np.pi)), nharm=1)]
    else:
        rng = np.random.default_rng(p["seed"] + 1000)
        chirps = random_chirps(rng, 20, n, p["zmax"])
    x = make_series(n, p["seed"], chirps, device=device)
    p["chirps"] = chirps
    return x, p
