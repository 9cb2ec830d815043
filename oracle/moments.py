"""Per-cell moments, realizability matrices, L1 distance and mask bits.

Definitions restated from the paper (every integral is a grid sum times dv^3,
c = v - u, V = c / sqrt(T)):
  rho, u, T                       hypothesis H3 (sec. 2)
  rho Theta = int c (x) c f,  T = tr(Theta)/3           stress tensor (sec. 2.2)
  tau = rho Theta - p I, p = rho T;  q = 1/2 int c |c|^2 f        App. A
  Abar = (1/rho) int (V(x)V - |V|^2/3 I) f = Theta/T - I          eq. for Abar (sec. 3.1)
  Bbar = (1/rho) int 1/2 (|V|^2 - 5) V f = q / (rho T^{3/2})      eq. for Bbar (sec. 3.1)
  Cbar = 2/(5 rho) int (|V|^2/2 - 5/2)^2 f                        App. A
  V_eps = I + Abar - 2/3 Bbar Bbar^T                              eq. V_eps (sec. 3.2)
  V_gen = I + Abar - [(2/(5 Cbar)) / (1 - 2/(5 Cbar))] Bbar Bbar^T App. A (general Cbar)
  ||f - M_{rho,u,T}||_L1                                          L1 criterion (sec. 3.3)
Mask bits (uint8 per cell):
  bit0  realizability matrix M not PSD: not(rho > 0, T > 0, Cbar > 2/5, V_gen PSD)
        (Schur-complement argument of App. A)
  bit1  Euler breakdown: some eigenvalue of V_eps with |lambda - 1| > eta0 (sec. 3.3),
        decided as not((1+eta0) I - V_eps PSD and V_eps - (1-eta0) I PSD)
  bit2  ||f - M||_L1 > delta0 (sec. 3.3)
  bit7  invalid input: a non-finite value in the cell (bits 0-2 set as well)
PSD is decided by the signs of the 7 principal minors of a symmetric 3x3 matrix.

Bit-exactness.  The mask is an integer decided by floating point, so both the
oracle and the GPU take the decision from the same numbers:
  * every sum over the grid is an exact integer: f is converted to fixed point
    F = trunc(f * 2^P) (toward zero) with a per-cell scale P = 61 - e, where e is the binary
    exponent with max|f| < 2^e (a max is order-independent too), and F is
    multiplied by integer grid monomials (v = dv k with k_d = j_d - N/2), so
    the sum is independent of order and resolves f to 2^-61 of its peak;
  * each integer sum is rounded once to double (round-half-even);
  * the scalar algebra below is a fixed sequence of IEEE double operations
    with no fused multiply-add (Python float arithmetic);
  * the Maxwellian of the L1 test is separable; each 1D factor uses the
    project's own exponential (Cody-Waite reduction by ln 2 and a degree-13
    Horner Taylor polynomial), is rounded to fixed point E = rint(e 2^31), and
    M_fix = (A_fix E + 2^30) >> 31 with A_fix = rint(rho/(2 pi T)^{3/2} e0 e1 2^P2),
    P2 = 30 - max(e, e_M) (e_M the exponent of the Maxwellian's peak), so
    |F2 - M_fix| with F2 = trunc(f 2^P2) is again an exact integer sum; the L1
    test resolves f and M to 2^-30 of the larger peak (32-bit integers).
Eigenvalues of V_eps are reported (numpy eigvalsh), not bit-exact.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext

import numpy as np

FIX_TOP = 61          # fixed-point values of the moment sums stay below 2^61 in magnitude
L1_TOP = 30           # fixed-point values of the L1 test stay below 2^30
E_BITS = 31

getcontext().prec = 60
_LN2 = Decimal(2).ln()
# Cody-Waite split of ln 2: a head with 32 significant bits (k * head exact for
# |k| < 2^21) and the double nearest to the remainder.
LN2_HI = float(Decimal(round(_LN2 * (Decimal(2) ** 32))) / (Decimal(2) ** 32))
LN2_LO = float(_LN2 - Decimal(LN2_HI))
INV_LN2 = float(1 / _LN2)
EXP_COEF = [1.0 / math.factorial(n) for n in range(14)]   # Taylor coefficients 1/n!


def own_exp(x: float) -> float:
    """exp(x) for x <= 0: k = rint(x / ln2), r = (x - k ln2_hi) - k ln2_lo,
    p(r) = sum_{n<=13} r^n/n! by Horner (no FMA), result p * 2^k.
    Returns 0 for x < -700 (below every value the fixed-point test resolves)."""
    if x < -700.0:
        return 0.0
    k = float(np.rint(x * INV_LN2))
    t1 = k * LN2_HI
    t2 = x - t1
    t3 = k * LN2_LO
    r = t2 - t3
    p = EXP_COEF[13]
    for n in range(12, -1, -1):
        p = p * r
        p = p + EXP_COEF[n]
    return math.ldexp(p, int(k))


def max_exponent(f: np.ndarray) -> int:
    """e with max|f| < 2^e and max|f| >= 2^(e-1) (frexp convention); None if f == 0."""
    mx = float(np.max(np.abs(f)))
    if mx == 0.0:
        return None
    return math.frexp(mx)[1]


def to_fixed(f: np.ndarray, P: int) -> np.ndarray:
    """F = trunc(f * 2^P) (toward zero) as exact Python ints (object array)."""
    return np.trunc(np.ldexp(np.asarray(f, dtype=np.float64), P)).astype(np.int64).astype(object)


def _psd(S) -> bool:
    a, b, c, d, e, f = S
    if not (a >= 0.0 and b >= 0.0 and c >= 0.0):
        return False
    if not (a * b - d * d >= 0.0 and a * c - e * e >= 0.0 and b * c - f * f >= 0.0):
        return False
    det = (a * (b * c - f * f) - d * (d * c - f * e)) + e * (d * f - b * e)
    return det >= 0.0


PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]    # packed xx, yy, zz, xy, xz, yz


def _sym(P6, d, e):
    if d == e:
        return P6[d]
    return P6[{(0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}[(d, e)]]


def integer_sums(f: np.ndarray, P: int):
    """Exact integer sums S0, S_d, S_de, S3_d, S4 over one cell (Python ints)."""
    N = f.shape[-1]
    F = to_fixed(f, P)
    k = (np.arange(N) - N // 2).astype(object)
    k0 = np.broadcast_to(k[:, None, None], F.shape)
    k1 = np.broadcast_to(k[None, :, None], F.shape)
    k2 = np.broadcast_to(k[None, None, :], F.shape)
    kd = [k0, k1, k2]
    kk = k0 * k0 + k1 * k1 + k2 * k2
    S0 = int(F.sum())
    S1 = [int((F * kd[d]).sum()) for d in range(3)]
    S2 = [int((F * kd[d] * kd[e]).sum()) for d, e in PAIRS]
    S3 = [int((F * kd[d] * kk).sum()) for d in range(3)]
    S4 = int((F * kk * kk).sum())
    return F, S0, S1, S2, S3, S4


def cell_moments(f: np.ndarray, L: float, eta0: float, delta0: float):
    """Moments dict and mask byte for one cell f [N,N,N] (float64 or float32)."""
    N = f.shape[-1]
    fd = np.asarray(f, dtype=np.float64)
    nan = float("nan")
    out = {k: nan for k in ("rho", "T", "Cbar", "l1")}
    for k in ("u", "q", "Bbar", "eig"):
        out[k] = [nan] * 3
    for k in ("Theta", "tau", "Abar", "V"):
        out[k] = [nan] * 6
    if not np.all(np.isfinite(fd)):
        return out, 0x87
    ef = max_exponent(fd)
    if ef is None:
        out["rho"] = 0.0
        return out, 0x07
    P1 = FIX_TOP - ef
    F, S0, S1, S2, S3, S4 = integer_sums(fd, P1)
    h = (2.0 * L) / N
    vol = (h * h) * h
    D0 = float(S0)
    rho = math.ldexp(D0, -P1) * vol
    out["rho"] = rho
    if not (D0 > 0.0):
        return out, 0x07
    inv0 = 1.0 / D0
    kap = [float(S1[d]) * inv0 for d in range(3)]
    out["u"] = [kap[d] * h for d in range(3)]
    m2 = [float(S2[i]) * inv0 for i in range(6)]
    C = [m2[i] - kap[d] * kap[e] for i, (d, e) in enumerate(PAIRS)]
    trC = (C[0] + C[1]) + C[2]
    Tg = trC / 3.0
    h2 = h * h
    T = Tg * h2
    out["T"] = T
    if not (Tg > 0.0):
        return out, 0x07
    Theta = [C[i] * h2 for i in range(6)]
    p = rho * T
    tau = [rho * Theta[i] - p if i < 3 else rho * Theta[i] for i in range(6)]
    E3 = [float(S3[d]) * inv0 for d in range(3)]
    kk = (kap[0] * kap[0] + kap[1] * kap[1]) + kap[2] * kap[2]
    sC = [(kap[0] * _sym(C, d, 0) + kap[1] * _sym(C, d, 1)) + kap[2] * _sym(C, d, 2) for d in range(3)]
    m3 = [((E3[d] - 2.0 * sC[d]) - kap[d] * trC) - kap[d] * kk for d in range(3)]
    rv = rho * vol
    q = [0.5 * (rv * m3[d]) for d in range(3)]
    E4 = float(S4) * inv0
    kE3 = (kap[0] * E3[0] + kap[1] * E3[1]) + kap[2] * E3[2]
    trm2 = (m2[0] + m2[1]) + m2[2]
    km2k = ((kap[0] * kap[0] * m2[0] + kap[1] * kap[1] * m2[1]) + kap[2] * kap[2] * m2[2]) + \
        2.0 * ((kap[0] * kap[1] * m2[3] + kap[0] * kap[2] * m2[4]) + kap[1] * kap[2] * m2[5])
    m4 = (((E4 - 4.0 * kE3) + 2.0 * kk * trm2) + 4.0 * km2k) - 3.0 * (kk * kk)
    Cbar = m4 / (10.0 * (Tg * Tg)) - 0.5
    Abar = [C[i] / Tg - 1.0 if i < 3 else C[i] / Tg for i in range(6)]
    sq = Tg * math.sqrt(Tg)
    Bbar = [(0.5 * m3[d]) / sq for d in range(3)]
    c23 = 2.0 / 3.0
    V = [(1.0 + Abar[i]) - c23 * (Bbar[d] * Bbar[e]) if i < 3 else Abar[i] - c23 * (Bbar[d] * Bbar[e])
         for i, (d, e) in enumerate(PAIRS)]
    out.update(Theta=Theta, tau=tau, q=q, Cbar=Cbar, Abar=Abar, Bbar=Bbar, V=V)

    realizable = False
    if Cbar > 0.4:
        gam = 2.0 / (5.0 * Cbar)
        coef = gam / (1.0 - gam)
        Vg = [(1.0 + Abar[i]) - coef * (Bbar[d] * Bbar[e]) if i < 3 else Abar[i] - coef * (Bbar[d] * Bbar[e])
              for i, (d, e) in enumerate(PAIRS)]
        realizable = _psd(Vg)
    up = [(1.0 + eta0) - V[i] if i < 3 else -V[i] for i in range(6)]
    dn = [V[i] - (1.0 - eta0) if i < 3 else V[i] for i in range(6)]
    near_euler = _psd(up) and _psd(dn)
    Vm = np.array([[V[0], V[3], V[4]], [V[3], V[1], V[5]], [V[4], V[5], V[2]]])
    out["eig"] = list(np.linalg.eigvalsh(Vm))

    # L1 distance to the Maxwellian with the same rho, u, T
    s = (2.0 * math.pi) * T
    CM = rho / (s * math.sqrt(s))
    P2 = L1_TOP - max(ef, math.frexp(CM)[1])
    inv2T = 1.0 / (2.0 * T)
    e = []
    for d in range(3):
        row = []
        for j in range(N):
            x = h * float(j - N // 2) - out["u"][d]
            row.append(own_exp(-((x * x) * inv2T)))
        e.append(row)
    E2 = np.array([int(np.rint(e[2][j] * 2.0 ** E_BITS)) for j in range(N)], dtype=object)
    A = np.array([[(CM * e[0][j0]) * e[1][j1] for j1 in range(N)] for j0 in range(N)])
    Afix = np.rint(np.ldexp(A, P2)).astype(np.int64).astype(object)
    Mfix = (Afix[:, :, None] * E2[None, None, :] + (1 << (E_BITS - 1))) >> E_BITS
    F2 = to_fixed(fd, P2)
    S_l1 = int(np.abs(F2 - Mfix).sum())
    l1 = math.ldexp(float(S_l1), -P2) * vol
    out["l1"] = l1
    mask = (0 if realizable else 1) | (0 if near_euler else 2)
    if l1 > delta0:
        mask |= 4
    return out, mask


MOMENT_FIELDS = [("rho", 1), ("u", 3), ("T", 1), ("Theta", 6), ("tau", 6), ("q", 3), ("Abar", 6),
                 ("Bbar", 3), ("Cbar", 1), ("V", 6), ("eig", 3), ("l1", 1)]


def pack(out: dict) -> np.ndarray:
    """Flatten a moments dict into the 40-double record layout of coll_moments."""
    v = []
    for name, n in MOMENT_FIELDS:
        x = out[name]
        v.extend(x if n > 1 else [x])
    return np.array(v, dtype=np.float64)


def batch(f: np.ndarray, L: float, eta0: float, delta0: float):
    """Records [n, 40] and mask bytes [n] for a batch f [n, N, N, N]."""
    recs, masks = [], []
    for c in range(f.shape[0]):
        o, m = cell_moments(f[c], L, eta0, delta0)
        recs.append(pack(o))
        masks.append(m)
    return np.stack(recs), np.array(masks, dtype=np.uint8)
