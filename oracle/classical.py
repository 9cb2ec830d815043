"""Classical Fourier-Galerkin kernel in closed form (sec. 4.4.1, eq. Q_k).

The classical spectral method writes
  Qh_k = sum_{l+m=k} fh_l fh_m [B^(l,m) - B^(m,m)],
  B^(l,m) = int_{|q| <= R_g} int_{S^2} B(|q|) exp(-i(xi_l.q^- + xi_m.q^+)) dsigma dq,
with q^+- = (q +- |q| sigma)/2.  For the VHS kernel B = b0 |q|^lam the sigma
integral is 4 pi sinc(|q| |xi_m - xi_l|/2) and the q integral reduces to
  B^(l,m) = 16 pi^2 b0 I_lam(a, b),  a = |xi_l+xi_m|/2, b = |xi_l-xi_m|/2,
  I_lam(a, b) = int_0^{R_g} r^{2+lam} sinc(a r) sinc(b r) dr,
which has the closed forms below.  R_g = 2S is the classical |g| truncation
(Proposition of sec. 4.4.1: supp Q within B(sqrt 2 S) for supp f in B(S)).
For f supported in B(S) this kernel and the Carleman form agree; it is used
only as an independent check of the Carleman normalisation.
"""
from __future__ import annotations

import math

import numpy as np

from .collision import dft, idft
from .kernel import Params, fft_modes, nyquist_mask


def _C1(c: np.ndarray, R: float) -> np.ndarray:
    """int_0^R r cos(c r) dr (series for small |c R|)."""
    c = np.asarray(c, dtype=np.float64)
    out = np.empty_like(c)
    small = np.abs(c * R) < 1e-2
    cs = c[~small]
    out[~small] = R * np.sin(cs * R) / cs + (np.cos(cs * R) - 1.0) / (cs * cs)
    x = c[small]
    acc = np.zeros_like(x)
    for n in range(8):
        acc += (-1) ** n * x ** (2 * n) * R ** (2 * n + 2) / (math.factorial(2 * n) * (2 * n + 2))
    out[small] = acc
    return out


def _C0(c: np.ndarray, R: float) -> np.ndarray:
    """int_0^R cos(c r) dr = sin(c R)/c (series for small |c R|)."""
    c = np.asarray(c, dtype=np.float64)
    out = np.empty_like(c)
    small = np.abs(c * R) < 1e-2
    cs = c[~small]
    out[~small] = np.sin(cs * R) / cs
    x = c[small]
    acc = np.zeros_like(x)
    for n in range(8):
        acc += (-1) ** n * x ** (2 * n) * R ** (2 * n + 1) / (math.factorial(2 * n) * (2 * n + 1))
    out[small] = acc
    return out


def _one_zero(b: np.ndarray, R: float, lam: float) -> np.ndarray:
    """I_lam(0, b) = (1/b) int_0^R r^{1+lam} sin(b r) dr for b > 0."""
    bR = b * R
    if lam == 1.0:
        val = -R * R * np.cos(bR) / b + 2 * R * np.sin(bR) / b ** 2 + 2 * (np.cos(bR) - 1.0) / b ** 3
    else:
        val = np.sin(bR) / b ** 2 - R * np.cos(bR) / b
    return val / b


def I_lam(a: np.ndarray, b: np.ndarray, R: float, lam: float) -> np.ndarray:
    """I_lam(a, b) for lam in {0, 1}, closed form with exact a=0 / b=0 branches."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.empty(np.broadcast(a, b).shape)
    a, b = np.broadcast_to(a, out.shape), np.broadcast_to(b, out.shape)
    za, zb = (a == 0.0), (b == 0.0)
    both = za & zb
    out[both] = R ** (3 + lam) / (3 + lam)
    ao = za & ~zb
    out[ao] = _one_zero(b[ao], R, lam)
    bo = zb & ~za
    out[bo] = _one_zero(a[bo], R, lam)
    gen = ~za & ~zb
    ag, bg = a[gen], b[gen]
    if lam == 1.0:
        out[gen] = (_C1(ag - bg, R) - _C1(ag + bg, R)) / (2.0 * ag * bg)
    elif lam == 0.0:
        out[gen] = (_C0(ag - bg, R) - _C0(ag + bg, R)) / (2.0 * ag * bg)
    else:
        raise ValueError("closed form only for lam in {0, 1}")
    return out


def I_lam_quadrature(a, b, R, lam, n=256):
    """Same integral by n-point Gauss-Legendre (cross-check of the closed form)."""
    x, w = np.polynomial.legendre.leggauss(n)
    r = 0.5 * R * (x + 1.0)
    w = 0.5 * R * w
    a = np.asarray(a, dtype=np.float64)[..., None]
    b = np.asarray(b, dtype=np.float64)[..., None]
    return np.sum(w * r ** (2 + lam) * np.sinc(a * r / np.pi) * np.sinc(b * r / np.pi), axis=-1)


def q_classical(f: np.ndarray, p: Params, Rg: float = None) -> np.ndarray:
    """O(N^6) classical spectral sum with the closed-form kernel (circular l+m)."""
    N = p.N
    Rg = p.R if Rg is None else Rg
    b0 = p.kernel_b0
    fh = dft(np.asarray(f, dtype=np.float64))
    keep = ~nyquist_mask(N)
    kk = fft_modes(N)
    K0, K1, K2 = np.meshgrid(kk, kk, kk, indexing="ij")
    kv = np.stack([K0[keep], K1[keep], K2[keep]], axis=1)
    xv = kv * (math.pi / p.L)
    fv = fh[keep]
    nm = np.linalg.norm(xv, axis=1)
    Bmm = 16 * math.pi ** 2 * b0 * I_lam(nm, np.zeros_like(nm), Rg, p.lam)   # B^(m,m)
    Qh = np.zeros((N, N, N), dtype=complex)
    for li in range(kv.shape[0]):
        a = 0.5 * np.linalg.norm(xv[li][None, :] + xv, axis=1)
        b = 0.5 * np.linalg.norm(xv[li][None, :] - xv, axis=1)
        Blm = 16 * math.pi ** 2 * b0 * I_lam(a, b, Rg, p.lam)
        idx = np.mod(kv[li][None, :] + kv, N)
        np.add.at(Qh, (idx[:, 0], idx[:, 1], idx[:, 2]), fv[li] * fv * (Blm - Bmm))
    return idft(Qh).real
