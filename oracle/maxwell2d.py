"""Fast spectral collision operator for Maxwell molecules in two velocity
dimensions (arxiv 2505.03360, sec. 4.4.1, "The 2d case").

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, numpy's
FFT as the transform step.

Kernel.  For d = 2 and gamma = 0 the Carleman weight is constant (sec. 4.4.1,
Bt = 2^{d-1} C_gamma (|x|^2 + |y|^2)^{-(d-gamma-2)/2}), Bt = 2 b0 for the
collision kernel B = b0 (b0 = 1/(2 pi) gives int_{S^1} b dsigma = 1, the BKW
normalisation).  With x = rho e_theta, y = rho' e_theta', theta, theta' in
[0, pi), rho, rho' in [-R, R], delta(x.y) leaves theta' = theta + pi/2 and
  K(l, m) = Bt int_0^pi phi(xi_l . e_theta) phi(xi_m . e_theta^perp) dtheta,
  phi(s) = int_{-R}^{R} exp(i rho s) drho = 2 R sinc(R s),
discretised on the A equally spaced angles theta_p = p pi / A, p = 1..A, with
weight pi / A (the integrand has period pi, so the rule is spectrally
accurate):
  alpha_p(xi)  = phi(xi . e_p),  alpha'_p(xi) = phi(xi . e_p^perp),
  c = Bt pi / A,  K(l, m) = sum_p c alpha_p(xi_l) alpha'_p(xi_m).

Operator (same conventions as the 3D path): fh = DFT(f) on the N x N grid
v_j = -L + j 2L/N with every |k_d| = N/2 mode dropped, xi_k = pi k / L,
  Q = sum_p c IDFT(alpha_p fh) IDFT(alpha'_p fh) - IDFT(fh) IDFT(Lambda fh),
  Lambda = sum_p c alpha_p alpha'_p  (the loss on the same directions),
R = 2 S with S the support (default 2L/(3 + sqrt 2), the no-overlap bound).

BKW solution (2D Maxwell molecules, b0 = 1/(2 pi)):
  f_S(v) = exp(-|v|^2/(2S)) / (2 pi S^2) (2S - 1 + (1 - S)/(2S) |v|^2),
  S(t) = 1 - exp(-t/8)/2,  Q(f_S, f_S) = d/dt f_S = (1 - S)/8 d/dS f_S.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Params2D:
    N: int
    L: float
    S: float = 0.0            # support; 0 -> 2L/(3 + sqrt 2); truncation R = 2S
    A: int = 16               # directions theta_p = p pi / A
    b0: float = -1.0          # collision kernel constant; <= 0 -> 1/(2 pi)

    @property
    def support(self) -> float:
        return self.S if self.S > 0 else 2.0 * self.L / (3.0 + math.sqrt(2.0))

    @property
    def R(self) -> float:
        return 2.0 * self.support

    @property
    def kernel_b0(self) -> float:
        return self.b0 if self.b0 > 0 else 1.0 / (2.0 * math.pi)


def modes(N: int) -> np.ndarray:
    """Signed integer frequencies in FFT order."""
    return np.fft.fftfreq(N, 1.0 / N).round().astype(np.int64)


def nyquist_mask(N: int) -> np.ndarray:
    nyq = modes(N) == -(N // 2)
    return nyq[:, None] | nyq[None, :]


def _phase(N: int) -> np.ndarray:
    """(-1)^(k0 + k1): the grid starts at v_0 = -L."""
    s = np.where(modes(N) % 2 == 0, 1.0, -1.0)
    return s[:, None] * s[None, :]


def dft(f: np.ndarray) -> np.ndarray:
    """fh_k = N^-2 sum_j f(v_j) exp(-i xi_k . v_j), Nyquist modes zeroed."""
    N = f.shape[-1]
    fh = np.fft.fft2(f) / N ** 2 * _phase(N)
    fh[nyquist_mask(N)] = 0.0
    return fh


def idft(gh: np.ndarray) -> np.ndarray:
    N = gh.shape[-1]
    return np.fft.ifft2(gh * _phase(N)) * N ** 2


def phi(s: np.ndarray, R: float) -> np.ndarray:
    """int_{-R}^{R} exp(i rho s) drho = 2 R sinc(R s) (sinc(x) = sin x / x)."""
    return 2.0 * R * np.sinc(R * np.asarray(s) / math.pi)


def multipliers(p: Params2D):
    """(c, alpha [A, N, N], alpha' [A, N, N], Lambda [N, N]) on the FFT-ordered grid."""
    xi = modes(p.N) * (math.pi / p.L)
    X0, X1 = np.meshgrid(xi, xi, indexing="ij")
    c = 2.0 * p.kernel_b0 * math.pi / p.A
    al, alp = [], []
    for q in range(1, p.A + 1):
        th = math.pi * q / p.A
        e, ep = (math.cos(th), math.sin(th)), (-math.sin(th), math.cos(th))
        al.append(phi(X0 * e[0] + X1 * e[1], p.R))
        alp.append(phi(X0 * ep[0] + X1 * ep[1], p.R))
    al, alp = np.stack(al), np.stack(alp)
    return c, al, alp, c * np.einsum("p...,p...->...", al, alp)


def q_fast(f: np.ndarray, p: Params2D, m=None) -> np.ndarray:
    """Q(f, f) on the N x N grid for one cell, fast algorithm (FP64)."""
    c, al, alp, lam = multipliers(p) if m is None else m
    fh = dft(np.asarray(f, dtype=np.float64))
    G = np.zeros(f.shape)
    for q in range(al.shape[0]):
        G += c * idft(al[q] * fh).real * idft(alp[q] * fh).real
    return G - idft(fh).real * idft(lam * fh).real


def q_direct(f: np.ndarray, p: Params2D, m=None) -> np.ndarray:
    """O(N^4) spectral sum Qh_k = sum_{l+m=k mod N} fh_l fh_m [K(l,m) - K(m,m)]."""
    c, al, alp, _ = multipliers(p) if m is None else m
    N = p.N
    fh = dft(np.asarray(f, dtype=np.float64))
    keep = ~nyquist_mask(N)
    k = modes(N)
    K0, K1 = np.meshgrid(k, k, indexing="ij")
    kv = np.stack([K0[keep], K1[keep]], axis=1)
    fv = fh[keep]
    K = c * (al[:, keep].T @ alp[:, keep])          # K[l, m]
    Kmm = np.diag(K).copy()
    Qh = np.zeros((N, N), dtype=complex)
    for li in range(kv.shape[0]):
        idx = np.mod(kv[li][None, :] + kv, N)
        np.add.at(Qh, (idx[:, 0], idx[:, 1]), fv[li] * fv * (K[li] - Kmm))
    return idft(Qh).real


def kernel_quad(l, m, p: Params2D) -> float:
    """K(l, m) by adaptive quadrature of the theta integral (scipy), l, m wave vectors."""
    from scipy import integrate
    Bt = 2.0 * p.kernel_b0

    def g(th):
        e = (math.cos(th), math.sin(th))
        ep = (-math.sin(th), math.cos(th))
        return float(phi(l[0] * e[0] + l[1] * e[1], p.R) * phi(m[0] * ep[0] + m[1] * ep[1], p.R))

    val, _ = integrate.quad(g, 0.0, math.pi, limit=400, epsabs=1e-13, epsrel=1e-13)
    return Bt * val


def grid(p: Params2D) -> np.ndarray:
    return -p.L + np.arange(p.N) * (2.0 * p.L / p.N)


def conserved_moments(Q: np.ndarray, p: Params2D) -> np.ndarray:
    """(int Q, int Q v_x, int Q v_y, int Q |v|^2) by the grid sum."""
    x = grid(p)
    V0, V1 = np.meshgrid(x, x, indexing="ij")
    w = (2.0 * p.L / p.N) ** 2
    return np.array([Q.sum(), (Q * V0).sum(), (Q * V1).sum(), (Q * (V0 ** 2 + V1 ** 2)).sum()]) * w


def bkw(p: Params2D, S: float):
    """(f_S, d f_S / dS) on the grid."""
    x = grid(p)
    v2 = x[:, None] ** 2 + x[None, :] ** 2
    g = np.exp(-v2 / (2.0 * S)) / (2.0 * math.pi * S * S)
    P = 2.0 * S - 1.0 + (1.0 - S) / (2.0 * S) * v2
    dg = g * (v2 / (2.0 * S * S) - 2.0 / S)
    dP = 2.0 - v2 / (2.0 * S * S)
    return g * P, dg * P + g * dP


def bkw_S(t: float) -> float:
    return 1.0 - 0.5 * math.exp(-t / 8.0)


def bkw_Q(p: Params2D, S: float) -> np.ndarray:
    """Q(f_S, f_S) = (1 - S)/8 d f_S / dS."""
    return (1.0 - S) / 8.0 * bkw(p, S)[1]


def maxwellian(p: Params2D, rho: float, u, T: float) -> np.ndarray:
    x = grid(p)
    g0 = np.exp(-((x - u[0]) ** 2) / (2.0 * T))
    g1 = np.exp(-((x - u[1]) ** 2) / (2.0 * T))
    return rho / (2.0 * math.pi * T) * g0[:, None] * g1[None, :]
