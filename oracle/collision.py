"""Collision operator Q^R(f,f) on the periodic velocity grid (sec. 4.4.1).

Fourier convention (sec. 4.4.1, truncated Fourier series f_N, rescaled from
[-pi, pi] to [-L, L]): f(v) = sum_k fh_k exp(i xi_k . v), xi_k = pi k / L,
k_d in {-N/2, ..., N/2-1}.  Every mode with some |k_d| = N/2 is set to zero
on input so that the real, even multipliers map real functions to real
functions and the k = 0 bin receives no wrapped contribution (mass exact).

q_fast   the fast algorithm: one FFT of f, then for every term t of the
         separated kernel (sec. 4.4.1, eq. for beta_F as a sum over
         directions) two inverse FFTs and a pointwise product, plus the loss
         term f_p * IDFT(Lambda fh).  N-point circular products by default;
         dealias=1 pads the products to 3N/2 (Galerkin).
q_direct the O(N^6) spectral sum (sec. 4.4.1, eq. Q_k):
         Qh_k = sum_{l+m=k} fh_l fh_m [K(l,m) - K(l,l)],
         K(l,m) = sum_t c_t alpha_t(xi_l) alpha'_t(xi_m),
         with l + m taken modulo N (circular) or exactly (dealias).
Both use numpy's FFT as the transform step; nothing is blocked or fused.
"""
from __future__ import annotations

import numpy as np

from .kernel import Params, fft_modes, multipliers, nyquist_mask, Multipliers, iter_terms


def _phase(N: int) -> np.ndarray:
    """prod_d (-1)^{k_d}: the grid starts at v_0 = -L, so exp(i xi_k v_j) = (-1)^k w^{kj}."""
    s = np.where(fft_modes(N) % 2 == 0, 1.0, -1.0)
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


def dft(f: np.ndarray) -> np.ndarray:
    """fh_k = N^-3 sum_j f(v_j) exp(-i xi_k . v_j), FFT-ordered, Nyquist modes zeroed."""
    N = f.shape[-1]
    fh = np.fft.fftn(f, axes=(-3, -2, -1)) / N ** 3 * _phase(N)
    fh[..., nyquist_mask(N)] = 0.0
    return fh


def idft(gh: np.ndarray) -> np.ndarray:
    """g(v_j) = sum_k gh_k exp(i xi_k . v_j) (complex result)."""
    N = gh.shape[-1]
    return np.fft.ifftn(gh * _phase(N), axes=(-3, -2, -1)) * N ** 3


def _real(z: np.ndarray) -> np.ndarray:
    return z.real


def q_fast(f: np.ndarray, p: Params, m: Multipliers = None) -> np.ndarray:
    """Q^R(f,f) on the grid for one cell f [N,N,N] (FP64), fast algorithm."""
    if m is None:
        m = multipliers(p)
    if p.dealias:
        return _q_fast_galerkin(f, p, m)
    fh = dft(np.asarray(f, dtype=np.float64))
    G = np.zeros(f.shape)
    for t in range(m.n_terms):
        a = _real(idft(m.alpha[t] * fh))
        b = _real(idft(m.alphap[t] * fh))
        G += m.coef[t] * a * b
    ell = _real(idft(m.lam_loss * fh))
    fp = _real(idft(fh))
    return G - fp * ell


def q_fast_streaming(f: np.ndarray, p: Params, psi_method: str = "cheb") -> np.ndarray:
    """Same sum as q_fast with the multipliers generated one direction at a time
    (large grids, where storing every alpha_t would not fit in memory)."""
    fh = dft(np.asarray(f, dtype=np.float64))
    G = np.zeros(f.shape)
    Lam = np.zeros(f.shape)
    for c, a_t, b_t in iter_terms(p, psi_method=psi_method):
        G += c * _real(idft(a_t * fh)) * _real(idft(b_t * fh))
        Lam += c * a_t * b_t
    return G - _real(idft(fh)) * _real(idft(Lam * fh))


def q_gain_loss(f: np.ndarray, p: Params, m: Multipliers = None):
    """Gain Q+ and loss Q- = f_p * L(f) separately (sec. 2.1, split Q = Q+ - L(f) f)."""
    if m is None:
        m = multipliers(p)
    fh = dft(np.asarray(f, dtype=np.float64))
    G = np.zeros(f.shape)
    for t in range(m.n_terms):
        G += m.coef[t] * _real(idft(m.alpha[t] * fh)) * _real(idft(m.alphap[t] * fh))
    return G, _real(idft(fh)) * _real(idft(m.lam_loss * fh))


def _pad(gh: np.ndarray, N: int, Mpad: int) -> np.ndarray:
    """Embed FFT-ordered N-modes (Nyquist already zero) into an Mpad grid."""
    out = np.zeros((Mpad, Mpad, Mpad), dtype=complex)
    k = fft_modes(N)
    idx = np.where(k < 0, k + Mpad, k)
    out[np.ix_(idx, idx, idx)] = gh
    return out


def _truncate(Gh: np.ndarray, N: int, Mpad: int) -> np.ndarray:
    k = fft_modes(N)
    idx = np.where(k < 0, k + Mpad, k)
    out = Gh[np.ix_(idx, idx, idx)].copy()
    out[nyquist_mask(N)] = 0.0
    return out


def _q_fast_galerkin(f: np.ndarray, p: Params, m: Multipliers) -> np.ndarray:
    """Products evaluated on a 3N/2 grid (no aliasing of quadratic terms), result
    projected back onto the modes |k_d| < N/2."""
    N = p.N
    Mpad = 3 * N // 2
    fh = dft(np.asarray(f, dtype=np.float64))

    def to_phys(gh):
        return np.fft.ifftn(_pad(gh, N, Mpad)) * Mpad ** 3

    Gp = np.zeros((Mpad, Mpad, Mpad))
    for t in range(m.n_terms):
        Gp += m.coef[t] * to_phys(m.alpha[t] * fh).real * to_phys(m.alphap[t] * fh).real
    Gp -= to_phys(fh).real * to_phys(m.lam_loss * fh).real
    Qh = _truncate(np.fft.fftn(Gp) / Mpad ** 3, N, Mpad)
    return idft(Qh).real


def q_direct(f: np.ndarray, p: Params, m: Multipliers = None) -> np.ndarray:
    """O(N^6) spectral sum Qh_k = sum_{l+m=k} fh_l fh_m [K(l,m) - K(l,l)]."""
    if m is None:
        m = multipliers(p)
    N = p.N
    fh = dft(np.asarray(f, dtype=np.float64))
    keep = ~nyquist_mask(N)
    kk = fft_modes(N)
    K0, K1, K2 = np.meshgrid(kk, kk, kk, indexing="ij")
    kv = np.stack([K0[keep], K1[keep], K2[keep]], axis=1)          # [n, 3]
    fv = fh[keep]                                                  # [n]
    A = (m.coef[:, None] * m.alpha[:, keep])                       # [T, n]
    B = m.alphap[:, keep]                                          # [T, n]
    K = A.T @ B                                                    # K[l, m]
    Kll = np.diag(K).copy()
    Qh = np.zeros((N, N, N), dtype=complex)
    for li in range(kv.shape[0]):
        ksum = kv[li][None, :] + kv                                # l + m for all m
        contrib = fv[li] * fv * (K[li] - Kll[li])
        if p.dealias:
            ok = np.all(np.abs(ksum) <= N // 2 - 1, axis=1)
            idx = np.where(ksum[ok] < 0, ksum[ok] + N, ksum[ok])
            np.add.at(Qh, (idx[:, 0], idx[:, 1], idx[:, 2]), contrib[ok])
        else:
            idx = np.mod(ksum, N)
            np.add.at(Qh, (idx[:, 0], idx[:, 1], idx[:, 2]), contrib)
    return idft(Qh).real


def grid_weight(p: Params) -> float:
    """Delta v^3, the weight of each grid point in velocity integrals."""
    dv = 2.0 * p.L / p.N
    return dv ** 3


def conserved_moments(Q: np.ndarray, p: Params) -> np.ndarray:
    """(int Q, int Q v, int Q |v|^2) by the grid sum (hypothesis H1, sec. 2)."""
    x = -p.L + np.arange(p.N) * (2.0 * p.L / p.N)
    V0, V1, V2 = np.meshgrid(x, x, x, indexing="ij")
    w = grid_weight(p)
    return np.array([Q.sum(), (Q * V0).sum(), (Q * V1).sum(), (Q * V2).sum(),
                     (Q * (V0 ** 2 + V1 ** 2 + V2 ** 2)).sum()]) * w
