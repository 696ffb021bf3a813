"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method: it only draws seeded random
grid functions, evaluates the problem's initial condition and builds the
request stream of the serving workload.  Both the CUDA path and the oracle
receive these arrays as inputs.

Layout: numpy float64, C order ``[z][y][x]`` over the N^3 interior points of
the unit cube, h = 1/(N+1), x_i = i*h (zero Dirichlet boundary).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def grid(N: int) -> np.ndarray:
    """Interior coordinates x_i = i/(N+1), i = 1..N."""
    return np.arange(1, N + 1, dtype=np.float64) / (N + 1)


def sine_mode(N: int, k1: int = 1, k2: int = 1, k3: int = 1) -> np.ndarray:
    """sin(k1 pi x) sin(k2 pi y) sin(k3 pi z); (1,1,1) is the initial value of Eq. 4 at t=0."""
    x = grid(N)
    sx, sy, sz = np.sin(k1 * np.pi * x), np.sin(k2 * np.pi * x), np.sin(k3 * np.pi * x)
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def random_field(N: int, seed: int, batch: int | None = None, scale: float = 1.0) -> np.ndarray:
    """Uniform[-scale, scale) values on the interior (a rough, all-frequency field)."""
    rng = np.random.default_rng(seed)
    shape = (N, N, N) if batch is None else (batch, N, N, N)
    return scale * (2.0 * rng.random(shape) - 1.0)


def smooth_random_field(N: int, seed: int, nmodes: int = 8, kmax: int = 8) -> np.ndarray:
    """Seeded sum of sine modes with N(0,1) amplitudes and mode numbers 1..kmax."""
    rng = np.random.default_rng(seed)
    u = np.zeros((N, N, N))
    for _ in range(nmodes):
        k = rng.integers(1, kmax + 1, size=3)
        u += rng.standard_normal() * sine_mode(N, int(k[0]), int(k[1]), int(k[2]))
    return u


@dataclass
class Request:
    """One heat-equation solve of the serving workload (zero forcing)."""
    rid: int
    arrival: float            # seconds after the stream starts
    N: int
    nu: float
    T: float
    dt: float
    modes: list = field(default_factory=list)   # [(k1, k2, k3, amplitude)] * 8

    def initial_value(self) -> np.ndarray:
        u = np.zeros((self.N, self.N, self.N))
        for k1, k2, k3, a in self.modes:
            u += a * sine_mode(self.N, k1, k2, k3)
        return u


def request_stream(n: int, rate: float, seed: int = 1307, sizes=(63, 127, 255),
                   horizons=(0.25, 0.5, 1.0), dt: float = 1.0 / 32.0) -> list[Request]:
    """Poisson arrivals at `rate` per second; N uniform in `sizes`, nu ~ U[0.05, 0.2],
    T uniform in `horizons`, 8 modes with (k1,k2,k3) uniform in 1..8 and N(0,1) amplitudes."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        gap = rng.exponential(1.0)  # drawn at every rate, so the requests do not depend on it
        t += gap / rate if rate > 0 else 0.0
        N = int(rng.choice(sizes))
        nu = float(rng.uniform(0.05, 0.2))
        T = float(rng.choice(horizons))
        modes = []
        for _ in range(8):
            k = rng.integers(1, 9, size=3)
            modes.append((int(k[0]), int(k[1]), int(k[2]), float(rng.standard_normal())))
        out.append(Request(rid, t, N, nu, T, dt, modes))
    return out
