"""Accuracy of the digit arithmetic behind the tensor-core commit (host-side
restatement, exact integers).

The CUDA commit forms D = V^T C and C - V E from 56-bit fixed-point digits:
a value x with |x| < 2^E is Y = round(|x| 2^(56-E)), cut into eight 7-bit
digits; V rows carry a row scale 2^Er, C' = 2^Er C and E carry column
scales; products of digits are summed per level k + l <= 8 exactly, and the
levels are recombined (pass 2 in int64 with levels 7 and 8 rounded down).
This test restates those steps in Python integers and checks that the
result is as close to the exact (rational) product as an FP64 evaluation,
on operands whose rows span 2^-20 .. 2^20.
"""
import math
import struct
from fractions import Fraction as F

import numpy as np

ND = 8


def ebound(x):
    if x == 0 or abs(x) < 2.0 ** -1022:
        return -2000
    return math.frexp(abs(x))[1]  # |x| < 2^e


def fix56(x, sh):
    if x == 0 or abs(x) < 2.0 ** -1022:
        return 0
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    e = (b >> 52) & 0x7FF
    mant = (b & ((1 << 52) - 1)) | (1 << 52)
    s = e - 1075 + sh
    assert s <= 3
    if s >= 0:
        return mant << s
    return (mant + (1 << (-s - 1))) >> (-s) if s > -64 else 0


def digits(x, sh):
    y = fix56(x, sh)
    assert y < 1 << 56
    hi, lo = y >> 28, y & 0x0FFFFFFF
    d = [(hi >> (21 - 7 * k)) & 0x7F for k in range(4)] + [(lo >> (21 - 7 * k)) & 0x7F for k in range(4)]
    sg = -1 if x < 0 else 1
    return [sg * v for v in d]


def levels(a, b):
    """Level sums over k + l <= 8 of digit vectors a[i][k], b[i][l]."""
    lev = [0] * (ND + 1)
    for k in range(ND):
        for l in range(ND):
            if k + l <= ND:
                lev[k + l] += sum(ai[k] * bi[l] for ai, bi in zip(a, b))
    return lev


def commit_digits(V, C, T, kp):
    L, nb = V.shape[0], C.shape[1]
    Er = [max(ebound(v) for v in V[r, :kp]) for r in range(L)]
    a = [[digits(V[r, t], 56 - Er[r]) for t in range(kp)] for r in range(L)]
    Ec = [max([ebound(C[r, c]) + Er[r] for r in range(L) if ebound(C[r, c]) > -2000] or [-8000]) for c in range(nb)]
    bC = [[digits(C[r, c], Er[r] + 56 - Ec[c]) for c in range(nb)] for r in range(L)]
    D = np.zeros((kp, nb))
    for t in range(kp):
        for c in range(nb):
            lev = levels([a[r][t] for r in range(L)], [bC[r][c] for r in range(L)])
            s = float(lev[ND])
            for lam in range(ND - 1, -1, -1):
                s = s * 2.0 ** -7 + lev[lam]
            D[t, c] = math.ldexp(s, Ec[c] - 14)
    E = T[:kp, :kp].T @ D
    Ee = [max(ebound(E[t, c]) for t in range(kp)) for c in range(nb)]
    dE = [[digits(E[t, c], 56 - Ee[c]) for c in range(nb)] for t in range(kp)]
    Cn = C.copy()
    for r in range(L):
        for c in range(nb):
            lev = levels(a[r], [dE[t][c] for t in range(kp)])
            assert all(abs(v) < 2 ** 24 for v in lev)  # exact in FP32 accumulators
            u = sum(lev[l] << (43 - 7 * l) for l in range(7)) + (lev[7] >> 6) + (lev[8] >> 13)
            assert abs(u) < 2 ** 63
            Cn[r, c] = float(F(C[r, c]) - F(float(u)) * F(2) ** (Er[r] + Ee[c] - 57))
    return D, E, Cn


def test_digit_products_as_accurate_as_fp64():
    rng = np.random.default_rng(7)
    L, kp, nb = 36, 7, 3
    for trial in range(2):
        V = rng.standard_normal((L, kp))
        for t in range(kp):
            V[:t, t] = 0.0
        V *= 2.0 ** rng.integers(-20, 21, size=(L, 1))
        C = rng.standard_normal((L, nb))
        C[5, 1] = 0.0
        T = np.triu(rng.standard_normal((kp, kp)))
        D, E, Cn = commit_digits(V, C, T, kp)
        D64 = V.T @ C
        Dx = [[sum(F(V[r, t]) * F(C[r, c]) for r in range(L)) for c in range(nb)] for t in range(kp)]
        scale = np.abs(V).T @ np.abs(C)
        err = max(abs(float(F(D[t, c]) - Dx[t][c])) / scale[t, c] for t in range(kp) for c in range(nb))
        err64 = max(abs(float(F(D64[t, c]) - Dx[t][c])) / scale[t, c] for t in range(kp) for c in range(nb))
        # pass 1 is at least as accurate as the FP64 product, within 2^-53
        # of the magnitude sum (dropping level 8 or truncating digits fails)
        assert err <= min(err64, 2.0 ** -53), (err, err64)
        Cx = [[F(C[r, c]) - sum(F(V[r, t]) * F(E[t, c]) for t in range(kp)) for c in range(nb)] for r in range(L)]
        sc = np.abs(V) @ np.abs(E) + np.abs(C)
        errC = max(abs(float(F(Cn[r, c]) - Cx[r][c])) / sc[r, c] for r in range(L) for c in range(nb))
        # pass 2 (int64 recombination): within 1.26 * 2^-52 of the magnitude
        # sum on these operands (a wrong level shift or truncation fails)
        assert errC <= 2.8e-16, errC


def test_digit_split_is_exact_for_representable_values():
    # a value whose bits fit in the 56-bit window is rebuilt exactly
    for x in [1.0, -0.75, 3.0 * 2.0 ** -30, 0.1, -123456.789]:
        E = ebound(x)
        d = digits(x, 56 - E)
        y = sum(abs(v) << (49 - 7 * k) for k, v in enumerate(d))
        assert F(y) * F(2) ** (E - 56) == abs(F(x))
