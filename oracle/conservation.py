"""Collision invariants of Q per cell (hypothesis H1, sec. 2): the operator
preserves mass, momentum and kinetic energy,
    int Q dv = 0,   int Q v dv = 0,   int Q |v|^2 dv = 0.
Test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline use this module.

On the grid (v = h k, k_d = j_d - N/2, h = 2L/N, every integral a grid sum
times h^3) this returns, per cell, eight values:
    m0  = int Q,      m1_d = int Q v_d (d = 0, 1, 2),   m2 = int Q |v|^2,
    a0  = int |Q|,    a1   = int |Q| (|v_0| + |v_1| + |v_2|),   a2 = int |Q| |v|^2,
so that |m0| / a0, max_d |m1_d| / a1 and |m2| / a2 are relative conservation
errors (|int Q v_d| <= a1 and |int Q phi| <= int |Q| |phi|).

Arithmetic (the reading used for the GPU check, which the paper leaves open):
Q is converted to fixed point F = trunc(Q 2^P) (toward zero) with
P = 61 - e, 2^e above max |Q| (the moment sums' convention), the eight sums of
F times integer grid monomials are exact integers, each is rounded once to
double, and the scaling by 2^-P, h^3 and h or h^2 is a fixed sequence of
double operations:  m = ((S 2^-P) h^3) h^p.  The result is independent of
the order of summation, and within N^3 2^-P max|phi| h^3 of the real-number
sum of the grid values.
A non-finite value gives NaN for all eight; an all-zero cell gives zeros.
"""
from __future__ import annotations

import math

import numpy as np

from .moments import FIX_TOP, max_exponent, to_fixed

FIELDS = ("m0", "m1_0", "m1_1", "m1_2", "m2", "a0", "a1", "a2")


def integer_sums(Q: np.ndarray, P: int):
    """The eight exact integer sums of F = trunc(Q 2^P) times grid monomials."""
    N = Q.shape[-1]
    F = to_fixed(Q, P)
    A = np.abs(F)
    k = (np.arange(N) - N // 2).astype(object)
    k0 = np.broadcast_to(k[:, None, None], F.shape)
    k1 = np.broadcast_to(k[None, :, None], F.shape)
    k2 = np.broadcast_to(k[None, None, :], F.shape)
    kk = k0 * k0 + k1 * k1 + k2 * k2
    k1n = np.abs(k0) + np.abs(k1) + np.abs(k2)
    return [int(F.sum()), int((F * k0).sum()), int((F * k1).sum()), int((F * k2).sum()), int((F * kk).sum()),
            int(A.sum()), int((A * k1n).sum()), int((A * kk).sum())]


def cell_invariants(Q: np.ndarray, L: float) -> np.ndarray:
    """The eight values (m0, m1[3], m2, a0, a1, a2) of one cell Q [N, N, N]."""
    N = Q.shape[-1]
    Qd = np.asarray(Q, dtype=np.float64)
    if not np.all(np.isfinite(Qd)):
        return np.full(8, np.nan)
    e = max_exponent(Qd)
    if e is None:
        return np.zeros(8)
    P = FIX_TOP - e
    S = integer_sums(Qd, P)
    h = (2.0 * L) / N
    vol = (h * h) * h
    h2 = h * h
    powers = (0, 1, 1, 1, 2, 0, 1, 2)
    out = []
    for s, p in zip(S, powers):
        v = math.ldexp(float(s), -P) * vol           # float(int) rounds half to even
        if p == 1:
            v = v * h
        elif p == 2:
            v = v * h2
        out.append(v)
    return np.array(out, dtype=np.float64)


def batch(Q: np.ndarray, L: float) -> np.ndarray:
    """[n, 8] invariants of a batch Q [n, N, N, N]."""
    return np.stack([cell_invariants(Q[c], L) for c in range(Q.shape[0])])


def relative_errors(inv: np.ndarray) -> np.ndarray:
    """[n, 3] relative conservation errors |m0|/a0, max_d |m1_d|/a1, |m2|/a2."""
    inv = np.atleast_2d(inv)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.stack([np.abs(inv[:, 0]) / inv[:, 5], np.abs(inv[:, 1:4]).max(1) / inv[:, 6],
                         np.abs(inv[:, 4]) / inv[:, 7]], 1)
