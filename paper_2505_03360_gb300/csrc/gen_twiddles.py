"""Writes twiddles.h: cos and sin of 2 pi n / 192, n = 0..191, correctly rounded
(double; float; and float tails for float-pair arithmetic), and the tables of
the FMA form of a twiddle, w y = m (y + i t y) with m = cos, t = tan where
|cos| >= |sin| and w y = m (t y + i y) with m = sin, t = cot elsewhere (so that
|t| <= 1 and |m| >= 1/sqrt 2), the scale ratios m(3n) / m(n) and 1 / m(n).

192 = lcm(16, 24, 32, 48, 64), so every twiddle of the supported FFT lengths
and of their radix-2/3/4 sub-lengths is an entry of this table.  Values are
computed with mpmath at 50 digits and rounded once to double (and from the
exact value once to float).  Run by hand; the output header is committed.
"""
import os

import mpmath
import numpy as np

mpmath.mp.dps = 50
rows_d, rows_f, rows_l = [], [], []
for n in range(192):
    a = 2 * mpmath.pi * n / 192
    c, s = mpmath.cos(a), mpmath.sin(a)
    cd, sd = float(c), float(s)
    cf = float(np.float32(mpmath.nstr(c, 40)))
    sf = float(np.float32(mpmath.nstr(s, 40)))
    rows_d.append((cd.hex(), sd.hex()))
    rows_f.append((cf.hex(), sf.hex()))
    # tails of the float-pair twiddles: the float nearest to (exact - head)
    cl = float(np.float32(mpmath.nstr(c - mpmath.mpf(cf), 40)))
    sl = float(np.float32(mpmath.nstr(s - mpmath.mpf(sf), 40)))
    rows_l.append((cl.hex(), sl.hex()))
def form(n):
    """0: scaled by cos (|cos| >= |sin|), 1: scaled by sin."""
    a = n % 96
    return 0 if (a <= 24 or a >= 72) else 1


def fma_parts(n):
    a = 2 * mpmath.pi * n / 192
    c, s = mpmath.cos(a), mpmath.sin(a)
    return (c, s / c) if form(n) == 0 else (s, c / s)


def rnd_f(x):
    return float(np.float32(mpmath.nstr(x, 40)))


fma_rows = []
for n in range(192):
    m, t = fma_parts(n)
    m3 = fma_parts((3 * n) % 192)[0]
    vals = (m, t, m3 / m, 1 / m)
    fma_rows.append(([float(v).hex() for v in vals], [rnd_f(v).hex() for v in vals]))
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "twiddles.h")
with open(out, "w") as fh:
    fh.write("// Generated by gen_twiddles.py: cos/sin(2 pi n / 192), correctly rounded.\n")
    fh.write("#pragma once\n\n")
    fh.write("static __constant__ double kTwCosD[192] = {\n")
    fh.write(",\n".join("  %s" % c for c, _ in rows_d) + "};\n")
    fh.write("static __constant__ double kTwSinD[192] = {\n")
    fh.write(",\n".join("  %s" % s for _, s in rows_d) + "};\n")
    fh.write("static __constant__ float kTwCosF[192] = {\n")
    fh.write(",\n".join("  %sf" % c for c, _ in rows_f) + "};\n")
    fh.write("static __constant__ float kTwSinF[192] = {\n")
    fh.write(",\n".join("  %sf" % s for _, s in rows_f) + "};\n")
    fh.write("// tails: cos - kTwCosF and sin - kTwSinF rounded to float (float-pair twiddles)\n")
    fh.write("static __constant__ float kTwCosL[192] = {\n")
    fh.write(",\n".join("  %sf" % c for c, _ in rows_l) + "};\n")
    fh.write("static __constant__ float kTwSinL[192] = {\n")
    fh.write(",\n".join("  %sf" % s for _, s in rows_l) + "};\n")
    fh.write("// FMA form: w y = m (y + i t y) (form 0, |cos| >= |sin|) or m (t y + i y) (form 1);\n")
    fh.write("// ratio m(3n mod 192) / m(n) and 1 / m(n), each rounded once from the exact value\n")
    for k, name in enumerate(("M", "T", "R3", "IM")):
        fh.write("static __constant__ double kTw%sD[192] = {\n" % name)
        fh.write(",\n".join("  %s" % r[0][k] for r in fma_rows) + "};\n")
        fh.write("static __constant__ float kTw%sF[192] = {\n" % name)
        fh.write(",\n".join("  %sf" % r[1][k] for r in fma_rows) + "};\n")
