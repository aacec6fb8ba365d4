"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This module holds no arithmetic of the method: it only samples targets, initial states and
random vectors on the interior grid nodes, with numpy's PCG64 generator. Both the oracle and
the CUDA path receive the same arrays from here.

Grid convention: nx, ny count intervals on (0, Lx) x (0, Ly); the interior nodes are
x_i = i Lx/nx, y_j = j Ly/ny, i = 1..nx-1, j = 1..ny-1; time nodes t_n = n T/Nt, n = 1..Nt.
Arrays are [Nt][ny-1][nx-1] (time slices of [y][x], x fastest), float64.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One problem instance: sizes, coefficients and how to draw its inputs."""

    name: str
    nx: int
    ny: int
    Nt: int
    n_sub: int
    T: float = 1.0
    nu: float = 1.0
    omega: float = 1e-4
    Lx: float = 1.0
    Ly: float = 1.0
    target: str = "cos-mode-noise"       # see make_target
    u0: str = "zero"                     # "zero" or "paper"
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return (self.nx - 1) * (self.ny - 1)

    @property
    def V(self):
        return self.N * self.Nt


def _grid(w: Workload):
    x = w.Lx / w.nx * np.arange(1, w.nx)
    y = w.Ly / w.ny * np.arange(1, w.ny)
    t = w.T / w.Nt * np.arange(1, w.Nt + 1)
    return x, y, t


def make_target(w: Workload) -> np.ndarray:
    """Target u~ sampled at (t_n, y_j, x_i), shape [Nt][ny-1][nx-1].

    * "cos-mode-noise": sin(pi x) sin(pi y) cos(2 pi t) plus N(0, sigma^2) noise,
      sigma = w.extra.get("sigma", 1e-3), PCG64(seed).
    * "sine-series": sum over k, l <= kmax (default 8) of
      (a_kl cos 2 pi t + b_kl sin 2 pi t) sin(k pi x / Lx) sin(l pi y / Ly), a, b ~ N(0, 1).
    * "paper": sin(2 pi t) sin(2 pi x) sin(2 pi y), the experiment of Section 4.
    """
    x, y, t = _grid(w)
    X = x[None, None, :]
    Y = y[None, :, None]
    Tt = t[:, None, None]
    rng = np.random.Generator(np.random.PCG64(w.seed))
    if w.target == "cos-mode-noise":
        sigma = float(w.extra.get("sigma", 1e-3))
        base = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.cos(2 * np.pi * Tt)
        return base + sigma * rng.standard_normal((w.Nt, w.ny - 1, w.nx - 1))
    if w.target == "sine-series":
        kmax = int(w.extra.get("kmax", 8))
        a = rng.standard_normal((kmax, kmax))
        b = rng.standard_normal((kmax, kmax))
        sx = np.sin(np.pi * np.arange(1, kmax + 1)[:, None] * x[None, :] / w.Lx)   # [k][i]
        sy = np.sin(np.pi * np.arange(1, kmax + 1)[:, None] * y[None, :] / w.Ly)   # [l][j]
        ca = sy.T @ a.T @ sx                     # sum_kl a_kl sy_l(j) sx_k(i): [j][i]
        cb = sy.T @ b.T @ sx
        return (np.cos(2 * np.pi * t)[:, None, None] * ca[None]
                + np.sin(2 * np.pi * t)[:, None, None] * cb[None])
    if w.target == "paper":
        return np.sin(2 * np.pi * Tt) * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    raise ValueError(w.target)


def make_u0(w: Workload) -> np.ndarray:
    """Initial state on the interior nodes, shape [ny-1][nx-1]."""
    x, y, _ = _grid(w)
    if w.u0 == "zero":
        return np.zeros((w.ny - 1, w.nx - 1))
    if w.u0 == "paper":
        X, Y = np.meshgrid(x, y, indexing="xy")
        return -X * Y * (X - 1.0) * (Y - 2.0)
    raise ValueError(w.u0)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Standard-normal float64 vector from PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def random_mode_block(w: Workload, modes, seed: int) -> np.ndarray:
    """A space-time block that lives on a few spatial sine modes only.

    Returns (block [Nt][ny-1][nx-1], coeff [Nt][len(modes)]) with
    block = sum_q coeff[:, q] * sin(k_q pi x / Lx) sin(l_q pi y / Ly), (k_q, l_q) = modes[q],
    the coefficients N(0, 1). Such inputs let a test compare full-size outputs mode by mode.
    """
    x, y, _ = _grid(w)
    rng = np.random.Generator(np.random.PCG64(seed))
    coeff = rng.standard_normal((w.Nt, len(modes)))
    blk = np.zeros((w.Nt, w.ny - 1, w.nx - 1))
    for q, (k, l) in enumerate(modes):
        shape = np.sin(np.pi * l * y / w.Ly)[:, None] * np.sin(np.pi * k * x / w.Lx)[None, :]
        blk += coeff[:, q][:, None, None] * shape[None]
    return blk, coeff


# The problem instances the tests and the benchmark use.
CFG_SMALL = Workload("plain-fp64 32x32 Nt=64 ND=4", nx=32, ny=32, Nt=64, n_sub=4,
                     nu=1.0, omega=1e-4, target="cos-mode-noise", seed=0)
CFG_GPU = Workload("plain-fp64 256x256 Nt=1024 ND=64", nx=256, ny=256, Nt=1024, n_sub=64,
                   nu=1.0, omega=1e-4, target="sine-series", seed=1)
CFG_MIXED = Workload("mixed 512x512 Nt=512 ND=64", nx=512, ny=512, Nt=512, n_sub=64,
                     nu=0.1, omega=1e-4, target="sine-series", seed=2)
CFG_LEARNED = Workload("learned-coarse 256x256 Nt=2048 ND=256", nx=256, ny=256, Nt=2048,
                       n_sub=256, nu=1.0, omega=1e-4, target="sine-series", seed=4)
CFG_PAPER = Workload("paper 16x16 on (0,1)x(0,2)", nx=16, ny=16, Nt=200, n_sub=10,
                     Lx=1.0, Ly=2.0, omega=1e-4, target="paper", u0="paper", seed=0)


def batched_instances(count: int = 64, seed: int = 3) -> list[Workload]:
    """Uneven instances: nx=ny in {64,128,256}, Nt in {128..1024}, N_D in {8..64} <= Nt/2,
    nu log-uniform [0.1, 10], omega log-uniform [1e-6, 1e-2], sine-series targets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(count):
        n = int(rng.choice([64, 128, 256]))
        Nt = int(rng.choice([128, 256, 512, 1024]))
        nd = int(rng.choice([8, 16, 32, 64]))
        nd = min(nd, Nt // 2)
        nu = float(10 ** rng.uniform(-1, 1))
        om = float(10 ** rng.uniform(-6, -2))
        out.append(Workload(f"batch{q}", nx=n, ny=n, Nt=Nt, n_sub=nd, nu=nu, omega=om,
                            target="sine-series", seed=1000 + q))
    return out
