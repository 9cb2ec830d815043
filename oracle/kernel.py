"""Carleman multipliers of the fast spectral method (sec. 4.4.1).

Starting point: the truncated Carleman operator (sec. 4.4.1, eq. for Q^R),
  Q^R(f,f)(v) = int_{B_R} int_{B_R} Bt(x,y) delta(x.y) [f(v+y) f(v+x) - f(v+x+y) f(v)] dx dy,
with Bt = 2^{d-1} B(sqrt(|x|^2+|y|^2)) (|x|^2+|y|^2)^{-(d-2)/2} (Carleman lemma);
for the VHS kernel B = b0 |g|^lam in 3D, Bt = 4 b0 (|x|^2+|y|^2)^{(lam-1)/2}.

Writing x = rho e and resolving delta(x.y) leaves y in the plane e-perp:
  int int delta(x.y) F = int_{S^2} de int_0^R rho drho int_{disk_R(e-perp)} F dA(y).
Fourier modes e^{i xi.x}, e^{i xi'.y} then factor, and pairing e with -e over
the hemisphere gives, per direction e_p (weight w_p) and radial GL node
(rho_i, W_i) on [0, R]:
  alpha_{p,i}(xi)  = 2 W_i rho_i cos(rho_i xi.e_p)              (x integral)
  alpha'_{p,i}(xi) = Psi_{rho_i}(|xi - (xi.e_p) e_p|)          (y integral)
  Psi_rho(s) = 2 pi int_0^R r (rho^2 + r^2)^{(lam-1)/2} J0(r s) dr
with coefficient c_p = 4 b0 w_p.  For lam = 1 (hard spheres) Psi does not
depend on rho, Psi(s) = 2 pi R J1(R s)/s, and the i-sum collapses to one
multiplier per direction, alpha_p = sum_i alpha_{p,i}.  The loss multiplier
is Lambda(xi) = sum_t c_t alpha_t(xi) alpha'_t(xi) (same nodes as the gain).

The paper's printed psi (sec. 4.4.1, 3D case) integrates over a sphere with a
sin(theta) weight; the y integral of the Carleman form is over the circle in
e-perp, which is what Psi above computes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import special

from .quadrature import gauss_legendre, hemisphere_rule


@dataclass(frozen=True)
class Params:
    """Operator and grid parameters (names follow the paper's notation, sec. 2.1 and 4.4.1)."""
    N: int
    L: float
    S: float = 0.0            # support radius; 0 -> 2L/(3+sqrt 2); truncation R = 2S
    lam: float = 1.0          # VHS exponent (gamma of sec. 2.1)
    b0: float = -1.0          # kernel constant C_gamma; <0 -> 1/(4 pi) if lam==0 else 1
    M: int = 48               # full-sphere directions
    Mtheta: int = 4           # GL nodes in cos(theta) (rule 0) / A1 (rule 1)
    Mr: int = 16              # radial GL nodes on [0, R]
    sphere_rule: int = 0
    dealias: int = 0
    rank: int = 0             # lam != 1: radial terms per direction (0: the Mr node terms; see radial_factors)

    @property
    def support(self) -> float:
        return self.S if self.S > 0 else 2.0 * self.L / (3.0 + math.sqrt(2.0))

    @property
    def R(self) -> float:
        return 2.0 * self.support

    @property
    def kernel_b0(self) -> float:
        if self.b0 > 0:
            return self.b0
        return 1.0 / (4.0 * math.pi) if self.lam == 0.0 else 1.0


def fft_modes(N: int) -> np.ndarray:
    """Signed integer frequencies in FFT order: 0..N/2-1, -N/2..-1."""
    return np.fft.fftfreq(N, 1.0 / N).round().astype(np.int64)


def xi_grid(N: int, L: float):
    """Wave vectors xi_k = pi k / L on the full N^3 FFT-ordered grid, [N,N,N,3]."""
    k = fft_modes(N) * (math.pi / L)
    X = np.empty((N, N, N, 3))
    X[..., 0] = k[:, None, None]
    X[..., 1] = k[None, :, None]
    X[..., 2] = k[None, None, :]
    return X


def nyquist_mask(N: int) -> np.ndarray:
    """True where any |k_d| = N/2 (modes dropped so multipliers stay real/even)."""
    k = fft_modes(N)
    nyq = (k == -N // 2)
    return nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :]


def psi_hs(s: np.ndarray, R: float) -> np.ndarray:
    """Disk transform for lam = 1: 2 pi int_0^R r J0(r s) dr = 2 pi R J1(R s)/s."""
    s = np.asarray(s, dtype=np.float64)
    out = np.empty_like(s)
    small = s * R < 1e-8
    out[small] = math.pi * R * R
    ss = s[~small]
    out[~small] = 2.0 * math.pi * R * special.j1(R * ss) / ss
    return out


def _psi_nodes(rho_min: float, R: float, n_per_panel: int = 16, width: float = 0.5):
    """Composite GL nodes on [0, R]: geometric panels from rho_min, then <= width."""
    edges = [0.0]
    a = min(rho_min, R)
    edges.append(a)
    while a < R and a < width:
        a = min(2.0 * a, R)
        edges.append(a)
    while a < R:
        a = min(a + width, R)
        edges.append(a)
    xs, ws = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        if hi > lo:
            x, w = gauss_legendre(n_per_panel, lo, hi)
            xs.append(x)
            ws.append(w)
    return np.concatenate(xs), np.concatenate(ws)


def psi_general(s: np.ndarray, rhos: np.ndarray, R: float, lam: float) -> np.ndarray:
    """Psi_rho(s) = 2 pi int_0^R r (rho^2 + r^2)^{(lam-1)/2} J0(r s) dr for each rho.

    Returns [len(s), len(rhos)].  Composite Gauss-Legendre in r (graded panels
    near r = 0, where the integrand varies on the scale rho); the integrand is
    analytic on [0, R] because rho > 0.
    """
    s = np.asarray(s, dtype=np.float64).reshape(-1)
    r, w = _psi_nodes(float(np.min(rhos)), R)
    g = (2.0 * math.pi) * w[:, None] * r[:, None] * \
        (rhos[None, :] ** 2 + r[:, None] ** 2) ** ((lam - 1.0) / 2.0)      # [nr, Mr]
    out = np.empty((s.size, rhos.size))
    chunk = 4096
    for a in range(0, s.size, chunk):
        J = special.j0(s[a:a + chunk, None] * r[None, :])                   # [c, nr]
        out[a:a + chunk] = J @ g
    return out


def psi_general_cheb(s: np.ndarray, rhos: np.ndarray, R: float, lam: float,
                     width: float = 1.0, deg: int = 47) -> np.ndarray:
    """Psi_rho(s) through piecewise Chebyshev interpolation in s.

    On each s-panel of the given width, Psi is sampled by ``psi_general`` at
    deg+1 Chebyshev points and interpolated (numpy's Chebyshev basis as the
    library step).  Psi is entire in s with bandwidth R, so deg = 47 on unit
    panels resolves it to rounding for R up to ~25 (pinned against direct
    quadrature by the oracle tests).  Used only for large grids.
    """
    s = np.asarray(s, dtype=np.float64).reshape(-1)
    out = np.empty((s.size, rhos.size))
    if s.size == 0:
        return out
    x = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))     # Chebyshev points, (-1,1)
    Vinv = np.linalg.inv(np.polynomial.chebyshev.chebvander(x, deg))
    panel = np.floor(s / width).astype(np.int64)
    for pnl in np.unique(panel):
        lo = pnl * width
        sel = panel == pnl
        nodes = lo + 0.5 * width * (x + 1.0)
        coef = Vinv @ psi_general(nodes, rhos, R, lam)               # [deg+1, Mr]
        t = 2.0 * (s[sel] - lo) / width - 1.0
        out[sel] = np.polynomial.chebyshev.chebvander(t, deg) @ coef
    return out


@dataclass
class Multipliers:
    """Terms t of the separated kernel: K(l,m) = sum_t c_t alpha_t(xi_l) alpha'_t(xi_m)."""
    coef: np.ndarray          # [T]   c_t = 4 b0 w_p
    alpha: np.ndarray         # [T, N, N, N] on the FFT-ordered xi grid
    alphap: np.ndarray        # [T, N, N, N]
    directions: np.ndarray    # [Mh, 3]
    weights: np.ndarray       # [Mh]
    rho: np.ndarray           # radial nodes
    W: np.ndarray             # radial weights
    lam_loss: np.ndarray = field(default=None)   # Lambda = sum_t c_t alpha_t alpha'_t

    @property
    def n_terms(self) -> int:
        return self.coef.size


def direction_terms(p: Params, xv: np.ndarray, ep: np.ndarray, wp: float,
                    rho: np.ndarray, W: np.ndarray, psi_method: str = "direct"):
    """Terms (c, alpha, alpha') of one hemisphere direction e_p at wave vectors xv [n, 3]."""
    b0 = p.kernel_b0
    proj = xv @ ep                                    # xi . e
    perp = xv - proj[:, None] * ep[None, :]
    s = np.sqrt(np.sum(perp * perp, axis=1))          # |xi - (xi.e) e|
    cosm = np.cos(proj[:, None] * rho[None, :])       # [n, Mr]
    su, inv = np.unique(s, return_inverse=True)
    if p.lam == 1.0:
        a = (cosm * (2.0 * W * rho)[None, :]).sum(axis=1)
        return [(4.0 * b0 * wp, a, psi_hs(su, p.R)[inv])]
    if psi_method == "cheb":
        Psi = psi_general_cheb(su, rho, p.R, p.lam)[inv]
    else:
        Psi = psi_general(su, rho, p.R, p.lam)[inv]   # [n, Mr]
    full = [(4.0 * b0 * wp, 2.0 * W[i] * rho[i] * cosm[:, i], Psi[:, i]) for i in range(p.Mr)]
    fac = radial_factors(p, rho, W)
    if fac is None:
        return full
    P, Rm = fac
    A = np.stack([t[1] for t in full], axis=1)         # [n, Mr]: a_i cos(rho_i t)
    return [(4.0 * b0 * wp, A @ P[q], Psi @ Rm[q]) for q in range(P.shape[0])]


def radial_factors(p: Params, rho: np.ndarray, W: np.ndarray):
    """Low-rank separable approximation of the radial kernel (lam != 1).

    Per direction the Mr radial terms sum to
        sum_i a_i cos(rho_i t) Psi_{rho_i}(s),   a_i = 2 W_i rho_i,
        Psi_rho(s) = int_0^R g_rho(r) J0(r s) dr,  g_rho(r) = 2 pi r (rho^2 + r^2)^{(lam-1)/2},
    a bilinear form in the Mr-vectors c(t) = cos(rho_i t) and a_i Psi_{rho_i}(s)
    through the kernel matrix of B~ on (rho_i, r).  Its singular vectors are the
    eigenvectors U of the Gram matrix G_ii' = a_i a_i' int_0^R g_i g_i' dr (an
    integral, independent of the quadrature that evaluates it); keeping the r
    largest, term q of a direction is
        alpha_q  = sqrt(s_q) sum_i U_iq cos(rho_i t)
        alpha'_q = sum_i U_iq a_i Psi_{rho_i}(s) / sqrt(s_q),   s_q = sqrt(eigenvalue q),
    (U and s_q from the singular value decomposition of the factor
    Y_ik = a_i g_i(r_k) sqrt(w_k), G = Y Y^T, on the radial quadrature of Psi),
    so sum_q alpha_q alpha'_q = c^T U_r U_r^T diag(a) Psi, exact for r = Mr.
    Every term keeps the form alpha(xi . e) alpha'(|xi_perp|) with alpha even,
    so the loss built from the same terms keeps mass exact.
    Returns (P, Rm) with alpha_q = sum_i P[q, i] (a_i cos(rho_i t)) and
    alpha'_q = sum_i Rm[q, i] Psi_{rho_i}(s), or None (rank 0, or lam = 1) for the
    Mr node terms themselves; rank = Mr gives the same operator in the
    rotated basis."""
    if p.lam == 1.0 or p.rank <= 0:
        return None
    r, w = _psi_nodes(float(np.min(rho)), p.R)
    a = 2.0 * W * rho
    g = (2.0 * math.pi) * r[:, None] * (rho[None, :] ** 2 + r[:, None] ** 2) ** ((p.lam - 1.0) / 2.0)   # [nr, Mr]
    # Y Y^T = G with Y_ik = a_i g_i(r_k) sqrt(w_k): the left singular vectors of Y
    # are the eigenvectors of G, computed without squaring its condition number
    Y = a[:, None] * (g * np.sqrt(w)[:, None]).T                       # [Mr, nr]
    U, sv, _ = np.linalg.svd(Y, full_matrices=False)
    k = min(p.rank, p.Mr)
    U, sv = U[:, :k], sv[:k]
    sq = np.sqrt(sv)                                                   # sqrt(s_q)
    P = (sq[:, None] * U.T) / a[None, :]
    Rm = (U.T * a[None, :]) / sq[:, None]
    return P, Rm


def rules(p: Params):
    e, w = hemisphere_rule(p.M, p.Mtheta, p.sphere_rule)
    rho, W = gauss_legendre(p.Mr, 0.0, p.R)
    return e, w, rho, W


def iter_terms(p: Params, xi: np.ndarray = None, psi_method: str = "direct"):
    """Yield (c_t, alpha_t, alpha'_t) on the grid one direction at a time (streaming)."""
    if xi is None:
        xi = xi_grid(p.N, p.L)
    shape = xi.shape[:-1]
    xv = xi.reshape(-1, 3)
    e, w, rho, W = rules(p)
    for pi_ in range(e.shape[0]):
        for c, a, b in direction_terms(p, xv, e[pi_], w[pi_], rho, W, psi_method):
            yield c, a.reshape(shape), b.reshape(shape)


def multipliers(p: Params, xi: np.ndarray = None, psi_method: str = "direct") -> Multipliers:
    """Build alpha, alpha', c and Lambda on the N^3 grid (or on given xi [...,3])."""
    e, w, rho, W = rules(p)
    coefs, alphas, alphaps = [], [], []
    for c, a, b in iter_terms(p, xi, psi_method):
        coefs.append(c)
        alphas.append(a)
        alphaps.append(b)
    m = Multipliers(np.array(coefs), np.stack(alphas), np.stack(alphaps), e, w, rho, W)
    m.lam_loss = np.einsum("t,t...,t...->...", m.coef, m.alpha, m.alphap)
    return m


def lambda0_closed_form(p: Params) -> float:
    """Lambda(0) from the Thales-sphere geometry (exact integral, no quadrature).

    Lambda(0) = 4 b0 * (hemisphere area 2 pi) * int_0^R 2 rho Psi_rho(0) drho with
    Psi_rho(0) = 2 pi int_0^R r (rho^2+r^2)^{(lam-1)/2} dr:
      lam = 1: 8 pi^2 b0 R^4;   lam = 0: 32 pi^2 b0 R^3 (2 sqrt 2 - 2) / 3.
    """
    R, b0 = p.R, p.kernel_b0
    if p.lam == 1.0:
        return 8.0 * math.pi ** 2 * b0 * R ** 4
    if p.lam == 0.0:
        return 32.0 * math.pi ** 2 * b0 * R ** 3 * (2.0 * math.sqrt(2.0) - 2.0) / 3.0
    raise ValueError("closed form only for lam in {0, 1}")
