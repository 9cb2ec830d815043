"""Regime indicator on the 2D spatial grid and the regime update (Algorithm 1).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, shares
nothing with the CUDA path.

Restated from arxiv 2505.03360:
  * first and second spatial derivatives by central differences on the
    one-cell stencil (sec. 4.5, eq. for d xi/dx, d xi/dy, Delta rho,
    Delta u_x, Delta u_y), for xi in {rho, u_x, u_y, T};
  * the 2D matrix V_eps^1 and its closed-form eigenvalues (sec. 4.5, eq. for
    V_eps^1 and lambda^{a,b,c}; the 2D case of sec. 3.3, eq. for V_eps^1):
    a1 = 4/3 du_x/dx - 2/3 du_y/dy, a2 = (dT/dx)^2, b1 = du_x/dy + du_y/dx, b2 = dT/dx dT/dy,
    c1 = 4/3 du_y/dy - 2/3 du_x/dx, c2 = (dT/dy)^2,
    h1 = -2/3 (du_x/dx + du_y/dy), xi1 = eps mu / (rho T),
    xi2 = eps^2 2 kappa^2 / (3 rho^2 T^3), d = xi1 b1 + xi2 b2;
  * the Burnett-type indicator (sec. 3.3, eq. for lambda_B):
    lambda_B = eps^2 (|grad T|^2 / T + |grad u|^2
                      + sqrt((|Delta u|^2 + |Delta rho / rho|^2)(1 + T^2)));
  * viscosity and conductivity of hard spheres (sec. 3.1, first order):
    mu = mu0 sqrt(T), kappa = kappa0 sqrt(T);
  * Algorithm 1 (sec. 4.5, regime update r^n -> r^{n+1}, with the thresholds
    eta0, eta1, delta0 and the L1 distance of a layer-1 cell to its Maxwellian).

Readings where the paper is silent:
  * the fields are given on (ny + 2) x (nx + 2) cells with a one-cell halo
    that the caller fills with its boundary conditions (problem dependent);
  * Delta u is the vector (Delta u_x, Delta u_y): the printed "Delta u =
    Delta u_x + Delta u_y" drops the unit vectors that the next line writes
    for grad T, and lambda_B takes its squared modulus (a plain sum of the two
    Laplacians would change under the reflection x -> -x); |grad u|^2 is the
    sum of the squares of the four first derivatives of (u_x, u_y);
  * the Laplacian divides by dx dy, as printed;
  * a cell whose stencil holds a non-finite value, or with rho <= 0 or T <= 0,
    or a regime outside {0, 1, 2}, keeps its regime with bit 7 set (invalid).

Bit-exactness: the regime is an integer decided by floating point, so the
indicators follow one fixed sequence of IEEE double operations (no fused
multiply-add), with the reciprocals 1/(2 dx), 1/(2 dy), 1/(dx dy) and 1/3
rounded once; the GPU kernel takes the same sequence, so its indicators and
decisions equal these bit for bit.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

INVALID = 0x80


@dataclass(frozen=True)
class RegimeParams:
    """Knudsen number, transport constants, grid spacing and thresholds (sec. 5)."""
    eps: float
    mu0: float
    kappa0: float
    dx: float
    dy: float
    eta0: float
    eta1: float
    delta0: float


def indicators(fields: np.ndarray, p: RegimeParams):
    """lambda^a, lambda^b, lambda^c (eigenvalues of V_eps^1) and lambda_B per cell.

    fields: [4, ny + 2, nx + 2] float64 (rho, u_x, u_y, T with a one-cell halo).
    Returns four [ny, nx] arrays (sec. 4.5 eigenvalues; sec. 3.3 lambda_B).
    """
    F = np.asarray(fields, dtype=np.float64)
    i2dx = 1.0 / (2.0 * p.dx)
    i2dy = 1.0 / (2.0 * p.dy)
    ilap = 1.0 / (p.dx * p.dy)
    third = 1.0 / 3.0

    def c(q):
        return F[q, 1:-1, 1:-1]

    def e(q):
        return F[q, 1:-1, 2:]

    def w(q):
        return F[q, 1:-1, :-2]

    def n(q):
        return F[q, 2:, 1:-1]

    def s(q):
        return F[q, :-2, 1:-1]

    def ddx(q):                     # (xi_{i+1,j} - xi_{i-1,j}) / (2 dx)
        return (e(q) - w(q)) * i2dx

    def ddy(q):                     # (xi_{i,j+1} - xi_{i,j-1}) / (2 dy)
        return (n(q) - s(q)) * i2dy

    def lap(q):                     # 5-point Laplacian over dx dy
        return ((((w(q) + e(q)) + s(q)) + n(q)) - 4.0 * c(q)) * ilap

    RHO, UX, UY, T = 0, 1, 2, 3
    ux_x, ux_y, uy_x, uy_y = ddx(UX), ddy(UX), ddx(UY), ddy(UY)
    T_x, T_y = ddx(T), ddy(T)
    rho, Tc = c(RHO), c(T)
    lux, luy = lap(UX), lap(UY)
    rr = lap(RHO) / rho
    gT2 = T_x * T_x + T_y * T_y
    gu2 = ((ux_x * ux_x + ux_y * ux_y) + uy_x * uy_x) + uy_y * uy_y
    eps2 = p.eps * p.eps
    inner = ((lux * lux + luy * luy) + rr * rr) * (1.0 + Tc * Tc)
    lam_B = eps2 * ((gT2 / Tc + gu2) + np.sqrt(inner))

    sT = np.sqrt(Tc)
    mu = p.mu0 * sT
    kap = p.kappa0 * sT
    xi1 = (p.eps * mu) / (rho * Tc)
    xi2 = eps2 * ((2.0 * (kap * kap)) / (3.0 * ((rho * rho) * ((Tc * Tc) * Tc))))
    a1 = (4.0 * ux_x - 2.0 * uy_y) * third
    c1 = (4.0 * uy_y - 2.0 * ux_x) * third
    h1 = -((2.0 * (ux_x + uy_y)) * third)
    a2 = T_x * T_x
    b1 = ux_y + uy_x
    b2 = T_x * T_y
    c2 = T_y * T_y
    d = xi1 * b1 + xi2 * b2
    P = xi1 * (a1 - c1) + xi2 * (a2 - c2)
    S = ((xi1 * a1 + xi2 * a2) + xi1 * c1) + xi2 * c2
    root = np.sqrt(P * P + 4.0 * (d * d))
    lam_a = ((root - S) + 2.0) * 0.5
    lam_b = ((-root - S) + 2.0) * 0.5
    lam_c = 1.0 - xi1 * h1
    return lam_a, lam_b, lam_c, lam_B


def decide(r: np.ndarray, lam_a, lam_b, lam_c, lam_B, l1: np.ndarray, p: RegimeParams) -> np.ndarray:
    """Algorithm 1 (sec. 4.5, regime update) on valid cells.

    r = 2: stay 2 if |lambda_B| > eta1, else 1.
    r = 1: 2 if |lambda_B| > eta1; else 0 if every |lambda^k - 1| <= eta0 and
           the L1 distance to the Maxwellian is <= delta0; else 1.
    r = 0: 1 if some |lambda^k - 1| > eta0, else 0.
    """
    r = np.asarray(r, dtype=np.uint8)
    close = ((np.abs(lam_a - 1.0) <= p.eta0) & (np.abs(lam_b - 1.0) <= p.eta0)
             & (np.abs(lam_c - 1.0) <= p.eta0))
    burnett = np.abs(lam_B) > p.eta1
    out = np.empty_like(r)
    out[r == 2] = np.where(burnett[r == 2], 2, 1)
    one = r == 1
    to0 = close & (np.asarray(l1) <= p.delta0)
    out[one] = np.where(burnett[one], 2, np.where(to0[one], 0, 1))
    out[r == 0] = np.where(close[r == 0], 0, 1)
    return out


def valid_cells(fields: np.ndarray, r: np.ndarray, l1: np.ndarray) -> np.ndarray:
    """Cells whose stencil values are finite, with rho > 0, T > 0, a regime in
    {0, 1, 2} and, for a layer-1 cell, a finite L1 distance."""
    F = np.asarray(fields, dtype=np.float64)
    fin = np.isfinite(F).all(axis=0)
    ok = (fin[1:-1, 1:-1] & fin[1:-1, 2:] & fin[1:-1, :-2] & fin[2:, 1:-1] & fin[:-2, 1:-1])
    ok &= (F[0, 1:-1, 1:-1] > 0.0) & (F[3, 1:-1, 1:-1] > 0.0)
    r = np.asarray(r)
    ok &= r <= 2
    ok &= (r != 1) | np.isfinite(np.asarray(l1, dtype=np.float64))
    return ok


def regime_update(fields: np.ndarray, r: np.ndarray, l1: np.ndarray, p: RegimeParams):
    """r^{n+1} and the indicators [4, ny, nx] (lambda^a, lambda^b, lambda^c, lambda_B).
    Invalid cells keep their regime with bit 7 set."""
    with np.errstate(all="ignore"):
        lam = indicators(fields, p)
        ok = valid_cells(fields, r, l1)
        rn = decide(np.where(ok, r, 0).astype(np.uint8), *lam, l1, p)
    out = np.where(ok, rn, np.asarray(r, dtype=np.uint8) | INVALID).astype(np.uint8)
    return out, np.stack(lam)
