"""Seeded synthetic inputs shaped like the workloads of arXiv 2205.09070.

This module only draws random numbers and packs them; it holds none of the
method's arithmetic, so both the CUDA path (tests, bench) and the CPU oracle
can use it.  The paper's own data (NOAA GHCN-Daily station-day points, Sec. 3)
is not available; these generators stand in for it:

* ``small_2d``     : N = 2,000 uniform points in [0,1]^2, 2 functions x 3 bumps
                     (radii U(0.15, 0.3)), stationary radius 0.05, noise 1e-4.
* ``uniform_3d``   : N = 200,000 uniform points in [0,1]^3, 4 x 8 bumps
                     (radii U(0.02, 0.05)), stationary radius 0.02.
* ``grad_3d``      : N = 5,000 uniform points in [0,1]^3 with the 4 x 8 bump
                     layout (163 hyperparameters), radii U(0.15, 0.3), r_s 0.09.
* ``batch_2d``     : 256 independent 2-D problems, N_i uniform in [1000, 50000],
                     2 x 4 bumps each, stationary radius U(0.02, 0.08).
* ``mixture_3d``   : a 50-component Gaussian mixture (sigma 0.02, 80 %) plus 20 %
                     uniform background in [0,1]^3 -- the clustered station
                     geometry of the climate example -- with 8 x 16 bumps
                     (radii U(0.01, 0.03)) centred on mixture components.

Hyperparameter layout (P = n1*n2*(dim+2) + 3): for each function m and bump b,
[centre (dim), radius, amplitude]; then stationary radius r_s, amplitude A,
noise variance sigma_n^2.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    name: str
    x: np.ndarray          # (N, dim) float64, row-major
    y: np.ndarray          # (N,) float64
    h: np.ndarray          # (P,) float64
    dim: int
    n1: int
    n2: int
    beta: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def pack_h(centres, radii, amps, r_s, A, sigma2) -> np.ndarray:
    """Flatten bump parameters (n1, n2, dim) / (n1, n2) / (n1, n2) and the
    three trailing scalars into the hyperparameter vector."""
    n1, n2, dim = centres.shape
    b = np.concatenate([centres, radii[..., None], amps[..., None]], axis=2)
    return np.concatenate([b.reshape(-1), [r_s, A, sigma2]]).astype(np.float64)


def _gaussian_field(rng, x, n_bumps=5, width=0.1):
    amp = rng.normal(0.0, 1.0, n_bumps)
    cen = rng.uniform(0.0, 1.0, (n_bumps, x.shape[1]))
    y = np.zeros(x.shape[0])
    for a, c in zip(amp, cen):
        y += a * np.exp(-np.sum((x - c) ** 2, axis=1) / (2.0 * width * width))
    return y


def small_2d(seed: int = 1, n: int = 2000) -> Problem:
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, (n, 2))
    y = np.sin(6.0 * x[:, 0]) * np.cos(4.0 * x[:, 1]) + rng.normal(0.0, 0.01, n)
    n1, n2 = 2, 3
    centres = rng.uniform(0.0, 1.0, (n1, n2, 2))
    radii = rng.uniform(0.15, 0.3, (n1, n2))
    amps = rng.normal(0.0, 1.0, (n1, n2))
    h = pack_h(centres, radii, amps, 0.05, 1.0, 1e-4)
    return Problem("small_2d", x, y, h, 2, n1, n2)


def uniform_3d(seed: int = 2, n: int = 200_000, radii_range=(0.02, 0.05), r_s: float = 0.02) -> Problem:
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, (n, 3))
    y = _gaussian_field(rng, x) + rng.normal(0.0, 0.02, n)
    n1, n2 = 4, 8
    centres = rng.uniform(0.0, 1.0, (n1, n2, 3))
    radii = rng.uniform(radii_range[0], radii_range[1], (n1, n2))
    amps = rng.normal(0.0, 1.0, (n1, n2))
    h = pack_h(centres, radii, amps, r_s, 1.0, 4e-4)
    return Problem("uniform_3d", x, y, h, 3, n1, n2)


def grad_3d(seed: int = 3, n: int = 5000) -> Problem:
    p = uniform_3d(seed, n, radii_range=(0.15, 0.3), r_s=0.09)
    p.name = "grad_3d"
    return p


def batch_2d(seed: int = 4, n_inst: int = 256, n_range=(1000, 50_000)) -> list[Problem]:
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_range[0], n_range[1] + 1, n_inst)
    out = []
    for k, n in enumerate(sizes):
        x = rng.uniform(0.0, 1.0, (int(n), 2))
        y = np.sin(6.0 * x[:, 0]) * np.cos(4.0 * x[:, 1]) + rng.normal(0.0, 0.01, int(n))
        centres = rng.uniform(0.0, 1.0, (2, 4, 2))
        radii = rng.uniform(0.15, 0.3, (2, 4))
        amps = rng.normal(0.0, 1.0, (2, 4))
        r_s = rng.uniform(0.02, 0.08)
        out.append(Problem(f"batch_2d[{k}]", x, y, pack_h(centres, radii, amps, r_s, 1.0, 1e-4), 2, 2, 4))
    return out


def mixture_3d(seed: int = 5, n: int = 5_000_000, r_s: float = 0.005, n_comp: int = 50,
               frac_mixture: float = 0.8, sigma: float = 0.02, n1: int = 8, n2: int = 16) -> Problem:
    rng = np.random.default_rng(seed)
    n_mix = int(round(frac_mixture * n))
    means = rng.uniform(0.0, 1.0, (n_comp, 3))
    comp = rng.integers(0, n_comp, n_mix)
    x_mix = means[comp] + rng.normal(0.0, sigma, (n_mix, 3))
    x_bg = rng.uniform(0.0, 1.0, (n - n_mix, 3))
    x = np.concatenate([x_mix, x_bg])
    x = x[rng.permutation(n)]
    y = _gaussian_field(rng, x) + rng.normal(0.0, 0.02, n)
    which = (16 * np.arange(n1)[:, None] + np.arange(n2)[None, :]) % n_comp
    centres = means[which] + rng.normal(0.0, 0.01, (n1, n2, 3))
    radii = rng.uniform(0.01, 0.03, (n1, n2))
    amps = rng.normal(0.0, 1.0, (n1, n2))
    h = pack_h(centres, radii, amps, r_s, 1.0, 4e-4)
    return Problem("mixture_3d", np.ascontiguousarray(x), y, h, 3, n1, n2,
                   meta={"n_comp": n_comp, "sigma": sigma, "r_s": r_s})


def mixture_1m(seed: int = 6, n: int = 1_000_000) -> Problem:
    """The 1M-point measurement workload: the mixture generator at N = 1e6 with
    the stationary radius scaled by 5^(1/3) so that the neighbours per row
    match the 5M-point case."""
    p = mixture_3d(seed, n, r_s=0.005 * 5.0 ** (1.0 / 3.0))
    p.name = "mixture_1m"
    return p
