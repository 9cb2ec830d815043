"""Seeded synthetic inputs for the collision-operator hot path.

This module only *creates inputs*: velocity grids, distribution functions built
from Maxwellians, the BKW initial datum, a 2D regime mask and a request stream.
It holds none of the collision or moment arithmetic, imports neither the CUDA
library nor the CPU oracle, and is shared by both so that they see identical
bytes.  Every generator takes an explicit seed (numpy PCG64).

Grid convention (velocity setting of section 4.1): N points per axis on the
periodic box [-L, L)^3, v_j = -L + j*dv with dv = 2L/N, so the grid contains 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20250506

# Box geometry used by every workload unless stated: support S = 6 and the
# no-overlap half-width L = (3 + sqrt 2) S / 2 of the periodised operator.
DEFAULT_S = 6.0
DEFAULT_L = (3.0 + math.sqrt(2.0)) * DEFAULT_S / 2.0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def velocity_axis(N: int, L: float) -> np.ndarray:
    return -L + np.arange(N, dtype=np.float64) * (2.0 * L / N)


def _gauss_1d(x: np.ndarray, mean: float, var: float) -> np.ndarray:
    return np.exp(-((x - mean) ** 2) / (2.0 * var))


def maxwellian_cells(N: int, L: float, rho, u, T) -> np.ndarray:
    """Isotropic Maxwellians rho/(2 pi T)^{3/2} exp(-|v-u|^2/2T), one per cell.

    rho, T: [n]; u: [n, 3].  Returns [n, N, N, N] float64 (separable build).
    """
    x = velocity_axis(N, L)
    rho = np.asarray(rho, np.float64).reshape(-1)
    T = np.asarray(T, np.float64).reshape(-1)
    u = np.asarray(u, np.float64).reshape(-1, 3)
    n = rho.shape[0]
    g = [np.exp(-((x[None, :] - u[:, d:d + 1]) ** 2) / (2.0 * T[:, None])) for d in range(3)]
    amp = rho / (2.0 * np.pi * T) ** 1.5
    return (amp[:, None, None, None] * g[0][:, :, None, None]
            * g[1][:, None, :, None] * g[2][:, None, None, :]).reshape(n, N, N, N)


def bimodal_batch(n_cells: int, N: int, L: float = DEFAULT_L, seed: int = BASE_SEED + 2,
                  dtype=np.float64, chunk: int = 512) -> np.ndarray:
    """Sum of two Maxwellians per cell, shaped like shock-layer bimodality.

    Densities U[0.5, 2], mean velocities U[-1.5, 1.5]^3, temperatures U[0.5, 2]
    (the batch recipe for the 4096-cell N = 32 workload).
    """
    r = rng(seed)
    rho = r.uniform(0.5, 2.0, size=(n_cells, 2))
    u = r.uniform(-1.5, 1.5, size=(n_cells, 2, 3))
    T = r.uniform(0.5, 2.0, size=(n_cells, 2))
    out = np.empty((n_cells, N, N, N), dtype=dtype)
    for s in range(0, n_cells, chunk):
        e = min(n_cells, s + chunk)
        f = maxwellian_cells(N, L, rho[s:e, 0], u[s:e, 0], T[s:e, 0])
        f += maxwellian_cells(N, L, rho[s:e, 1], u[s:e, 1], T[s:e, 1])
        out[s:e] = f
    return out


def bkw_datum(N: int, L: float, K: float = 0.6) -> np.ndarray:
    """BKW self-similar datum for Maxwell molecules at shape parameter K.

    f_K(v) = exp(-|v|^2/2K) / (2 (2 pi K)^{3/2}) * [(5K-3)/K + (1-K)|v|^2/K^2],
    nonnegative for K >= 3/5; density 1 and temperature 1 for every K.
    """
    x = velocity_axis(N, L)
    v2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    g = np.exp(-v2 / (2.0 * K)) / (2.0 * (2.0 * np.pi * K) ** 1.5)
    return g * ((5.0 * K - 3.0) / K + (1.0 - K) * v2 / (K * K))


def _rotation_from_quaternion(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def anisotropic_cell(N: int, L: float, r: np.random.Generator, dtype=np.float32) -> np.ndarray:
    """0.9 * anisotropic Gaussian + 0.1 * Maxwellian (perturbed-equilibrium cell).

    Temperature tensor Theta = T0 Rot diag(1, a2, a3) Rot^T with a2, a3 ~ U[1, 3],
    T0 ~ U[0.5, 1], Rot from a seeded unit quaternion, u ~ U[-1, 1]^3,
    rho ~ U[0.5, 2]; the second Maxwellian is small and nearby.
    """
    x = velocity_axis(N, L)
    rho = r.uniform(0.5, 2.0)
    u = r.uniform(-1.0, 1.0, size=3)
    T0 = r.uniform(0.5, 1.0)
    a = np.array([1.0, r.uniform(1.0, 3.0), r.uniform(1.0, 3.0)])
    Rm = _rotation_from_quaternion(r.normal(size=4))
    Theta = T0 * Rm @ np.diag(a) @ Rm.T
    P = np.linalg.inv(Theta)
    c0 = x[:, None, None] - u[0]
    c1 = x[None, :, None] - u[1]
    c2 = x[None, None, :] - u[2]
    quad = (P[0, 0] * c0 * c0 + P[1, 1] * c1 * c1 + P[2, 2] * c2 * c2
            + 2 * P[0, 1] * c0 * c1 + 2 * P[0, 2] * c0 * c2 + 2 * P[1, 2] * c1 * c2)
    G = rho / math.sqrt(np.linalg.det(2 * np.pi * Theta)) * np.exp(-0.5 * quad)
    rho2 = r.uniform(0.5, 2.0)
    u2 = u + r.uniform(-0.5, 0.5, size=3)
    T2 = r.uniform(0.5, 1.0)
    M = maxwellian_cells(N, L, [rho2], [u2], [T2])[0]
    return (0.9 * G + 0.1 * M).astype(dtype)


def regime_mask_256(seed: int = BASE_SEED + 4, n: int = 256, target: float = 0.15,
                    tol: float = 0.005) -> np.ndarray:
    """Boolean [n, n] mask of ~15% cells forming curved shock bands.

    Cells within distance w of a parabola-like bow shock x = x0 + a (y - y0)^2
    or of a circle of radius r_c ~ U[0.15, 0.3] around an obstacle centre;
    w is bisected until the marked share is within target +- tol.
    """
    r = rng(seed)
    cx, cy = r.uniform(0.45, 0.6), r.uniform(0.4, 0.6)
    rc = r.uniform(0.15, 0.3)
    x0 = cx - rc - r.uniform(0.05, 0.15)
    a = r.uniform(1.0, 3.0)
    h = 1.0 / n
    xs = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    ys = np.linspace(-0.5, 1.5, 8001)
    px = x0 + a * (ys - cy) ** 2
    # distance to the sampled parabola (min over samples), then to the circle
    d_par = np.full(X.shape, np.inf)
    for k in range(0, ys.size, 500):
        dx = X[..., None] - px[None, None, k:k + 500]
        dy = Y[..., None] - ys[None, None, k:k + 500]
        d_par = np.minimum(d_par, np.sqrt(dx * dx + dy * dy).min(axis=-1))
    d_circ = np.abs(np.sqrt((X - cx) ** 2 + (Y - cy) ** 2) - rc)
    d = np.minimum(d_par, d_circ)
    lo, hi = 0.0, 0.5
    for _ in range(100):
        w = 0.5 * (lo + hi)
        share = float((d <= w).mean())
        if abs(share - target) <= tol:
            break
        if share < target:
            lo = w
        else:
            hi = w
    return d <= w


RAGGED_N = (16, 24, 32, 48)


@dataclass
class RaggedBatch:
    mask: np.ndarray              # [256, 256] bool
    cell_N: np.ndarray            # [n_cells] int, velocity points per axis per marked cell
    groups: dict                  # N -> float32 array [cells_of_N, N, N, N]
    order: dict                   # N -> indices into the marked-cell list


def ragged_batch(seed: int = BASE_SEED + 4, L: float = DEFAULT_L, max_cells=None) -> RaggedBatch:
    """Mixed-N FP32 batch from the 256 x 256 regime mask (N iid over {16,24,32,48})."""
    mask = regime_mask_256(seed)
    n_cells = int(mask.sum())
    if max_cells is not None:
        n_cells = min(n_cells, int(max_cells))
    r = rng(seed + 1000)
    cell_N = r.choice(np.array(RAGGED_N), size=n_cells)
    groups, order = {}, {}
    for N in RAGGED_N:
        idx = np.nonzero(cell_N == N)[0]
        order[N] = idx
        rr = rng(seed + 2000 + N)
        groups[N] = np.stack([anisotropic_cell(N, L, rr) for _ in idx]) if idx.size else \
            np.zeros((0, N, N, N), np.float32)
    return RaggedBatch(mask=mask, cell_N=cell_N, groups=groups, order=order)


@dataclass
class Request:
    rid: int
    arrival_s: float
    n_cells: int
    N: int
    lam: float
    precision: str                 # "f32" or "mixed"
    seed: int


def request_stream(n_requests: int = 2000, rate_per_s: float = 200.0,
                   seed: int = BASE_SEED + 5, Ns=(16, 32, 48, 64), max_cells: int = 2048,
                   precisions=("f32", "mixed")) -> list:
    """Poisson arrivals; cells per request floor(exp(U[0, ln(max_cells+1)]))."""
    r = rng(seed)
    gaps = r.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps)
    cells = np.floor(np.exp(r.uniform(0.0, math.log(max_cells + 1), size=n_requests))).astype(int)
    cells = np.clip(cells, 1, max_cells)
    Nsel = r.choice(np.array(Ns), size=n_requests)
    lam = r.choice(np.array([0.0, 1.0]), size=n_requests)
    prec = r.choice(np.array(precisions), size=n_requests)
    return [Request(i, float(t[i]), int(cells[i]), int(Nsel[i]), float(lam[i]), str(prec[i]),
                    seed * 7919 + i) for i in range(n_requests)]


def bimodal_batch_device(n_cells: int, N: int, L: float, seed: int, dtype=None, device="cuda"):
    """The bimodal recipe of ``bimodal_batch`` drawn on the device (torch), for
    large serving workloads where host generation would dominate; parameters
    from a seeded torch generator (not bitwise the numpy stream)."""
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rho = torch.rand((n_cells, 2), generator=g, device=device, dtype=torch.float64) * 1.5 + 0.5
    u = torch.rand((n_cells, 2, 3), generator=g, device=device, dtype=torch.float64) * 3.0 - 1.5
    T = torch.rand((n_cells, 2), generator=g, device=device, dtype=torch.float64) * 1.5 + 0.5
    x = -L + torch.arange(N, device=device, dtype=torch.float64) * (2.0 * L / N)
    out = torch.zeros((n_cells, N, N, N), device=device, dtype=dtype)
    for j in range(2):
        e = [torch.exp(-(x[None, :] - u[:, j, d:d + 1]) ** 2 / (2.0 * T[:, j:j + 1])) for d in range(3)]
        amp = rho[:, j] / (2.0 * math.pi * T[:, j]) ** 1.5
        out += (amp[:, None, None, None] * e[0][:, :, None, None] * e[1][:, None, :, None]
                * e[2][:, None, None, :]).to(dtype)
    return out


def regime_fields(ny: int, nx: int, dx: float, seed: int = BASE_SEED + 6):
    """Macroscopic fields for the regime update on an nx x ny grid with a
    one-cell halo: [4, ny + 2, nx + 2] float64 planes rho, u_x, u_y, T, each a
    constant plus four seeded tanh(8 sin(k . x + phase)) bands (shock-like
    fronts of random orientation); rho and T are kept >= 0.2.  Also a seeded
    regime map r in {0, 1, 2} [ny, nx] (uint8) and an L1 distance map
    10^U[-5, -3] [ny, nx] (spanning the paper's delta0 = 1e-4)."""
    r = rng(seed)
    y = (np.arange(ny + 2) - 0.5)[:, None] * dx
    x = (np.arange(nx + 2) - 0.5)[None, :] * dx
    out = []
    for q, base in enumerate((1.0, 0.1, -0.2, 0.9)):
        f = np.full((ny + 2, nx + 2), base)
        for _ in range(4):
            kx, ky, ph = r.uniform(1, 12), r.uniform(1, 12), r.uniform(0, 6.3)
            f = f + (0.25 if q in (0, 3) else 0.6) * r.uniform(0.2, 1.0) * np.tanh(8 * np.sin(kx * x + ky * y + ph))
        out.append(f)
    F = np.stack(out)
    F[0] = np.abs(F[0]) + 0.2
    F[3] = np.abs(F[3]) + 0.2
    regimes = r.integers(0, 3, (ny, nx)).astype(np.uint8)
    l1 = 10.0 ** r.uniform(-5, -3, (ny, nx))
    return F, regimes, l1


def bimodal_batch_2d(n_cells: int, N: int, L: float = 8.0, seed: int = BASE_SEED + 7,
                     dtype=np.float64) -> np.ndarray:
    """Two-dimensional cells: sum of two 2D Maxwellians per cell, densities
    U[0.5, 2], mean velocities U[-1.5, 1.5]^2, temperatures U[0.5, 2]."""
    r = rng(seed)
    rho = r.uniform(0.5, 2.0, size=(n_cells, 2))
    u = r.uniform(-1.5, 1.5, size=(n_cells, 2, 2))
    T = r.uniform(0.5, 2.0, size=(n_cells, 2))
    x = velocity_axis(N, L)
    out = np.zeros((n_cells, N, N), dtype=np.float64)
    for m in range(2):
        g0 = np.exp(-(x[None, :] - u[:, m, 0:1]) ** 2 / (2.0 * T[:, m:m + 1]))
        g1 = np.exp(-(x[None, :] - u[:, m, 1:2]) ** 2 / (2.0 * T[:, m:m + 1]))
        amp = rho[:, m] / (2.0 * np.pi * T[:, m])
        out += amp[:, None, None] * g0[:, :, None] * g1[:, None, :]
    return out.astype(dtype)


def bkw_datum_2d(N: int, L: float, S: float) -> np.ndarray:
    """2D BKW datum for Maxwell molecules at shape parameter S >= 1/2:
    exp(-|v|^2/(2S)) / (2 pi S^2) (2S - 1 + (1 - S)/(2S) |v|^2) (density 1)."""
    x = velocity_axis(N, L)
    v2 = x[:, None] ** 2 + x[None, :] ** 2
    return np.exp(-v2 / (2.0 * S)) / (2.0 * np.pi * S * S) * (2.0 * S - 1.0 + (1.0 - S) / (2.0 * S) * v2)
