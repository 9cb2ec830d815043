"""The generated twiddle tables of the register FFTs (csrc/twiddles.h, written by
csrc/gen_twiddles.py), checked on the host against high-precision values:
cos/sin correctly rounded, and the FMA-form tables consistent with them.

Where the exact value is 0 (cos at n = 48, 144; sin at n = 96) the table holds
the generator's 50-digit residual (below 1e-50) instead of 0; the transforms
never read those entries (n % 48 == 0 is an exact rotation by 1, i, -1, -i)."""
import math
import os
import re

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2505_03360_gb300", "csrc", "twiddles.h")


def _tables():
    txt = open(HDR).read()
    out = {}
    for name, body in re.findall(r"(kTw\w+)\[192\] = \{(.*?)\};", txt, re.S):
        out[name] = [float.fromhex(v.strip().rstrip("f")) for v in body.split(",")]
    return out


T = _tables()
mpmath.mp.dps = 40


def _exact(n):
    a = 2 * mpmath.pi * n / 192
    c, s = mpmath.cos(a), mpmath.sin(a)
    return (mpmath.mpf(0) if abs(c) < 1e-30 else c), (mpmath.mpf(0) if abs(s) < 1e-30 else s)


def _same(table_value, exact):
    return table_value == float(exact) or (exact == 0 and abs(table_value) < 1e-50)


def _form(n):
    return 0 if (n % 96 <= 24 or n % 96 >= 72) else 1


def test_cos_sin_correctly_rounded():
    for n in range(192):
        c, s = _exact(n)
        assert _same(T["kTwCosD"][n], c) and _same(T["kTwSinD"][n], s), n
        assert _same(T["kTwCosF"][n], np.float32(mpmath.nstr(c, 30))), n


def test_fma_form_tables():
    """w y = m (y + i t y) (form 0) or m (t y + i y) (form 1) with |t| <= 1, |m| >= 1/sqrt 2;
    R3 = m(3n) / m(n) and IM = 1 / m(n), each within half an ulp of the exact value."""
    for n in range(192):
        c, s = _exact(n)
        m, t = (c, s / c) if _form(n) == 0 else (s, c / s)
        assert _same(T["kTwMD"][n], m) and _same(T["kTwTD"][n], t), n
        assert abs(T["kTwTD"][n]) <= 1.0 and abs(T["kTwMD"][n]) >= 1 / math.sqrt(2) - 1e-16, n
        m3 = _exact(3 * n % 192)[0] if _form(3 * n % 192) == 0 else _exact(3 * n % 192)[1]
        assert T["kTwR3D"][n] == float(m3 / m) and T["kTwIMD"][n] == float(1 / m), n
        # the two forms reproduce the twiddle on a test vector to rounding
        w, y = complex(float(c), float(s)), complex(0.37, -1.21)
        tm, tt = T["kTwMD"][n], T["kTwTD"][n]
        got = tm * (y + 1j * tt * y) if _form(n) == 0 else tm * (tt * y + 1j * y)
        assert abs(got - w * y) < 4e-16 * abs(y), n
