"""Accuracy of the digit arithmetic behind the tensor-core commit (host-side
restatement, exact integers).

The CUDA commit forms D = V^T C and C - V E from 56-bit fixed-point digits:
a value x with |x| < 2^E is Y = round(|x| 2^(56-E)), cut into eight 7-bit
digits; reflector t of V is first scaled by 2^-Ft (2^Ft > |v0_t|, its pivot
entry), then V rows carry a row scale 2^Er, C' = 2^Er C and E'' = 2^Ft E
carry column scales; products of digits are summed per level k + l <= 8
exactly, and the levels are recombined (pass 2 in int64 with levels 7 and 8
rounded down).
This test restates those steps in Python integers (with the FP32 and int32
accumulation of the level sums as the kernel does it: 16-row MMA steps,
levels 0-6 moved into int32 every 128 rows, levels 7-8 kept in FP32) and
checks the result against the exact (rational) product.

The fixed point is accurate relative to the scales, not to each term:
where every term of a sum lies far below them (a large entry of C paired
with a zero of V, say), the digits lose bits an FP64 dot product keeps.
The reflector scales remove the common case (reflectors of very different
norms); pass 1's accuracy guard (sum of |leading digit| products, one more
MMA) detects the rest and hands the batch to FP64, so D is within the
worst-case bound of the FP64 evaluation, gamma_L sum |v||c|, element by
element.  Pass 2 has no guard: its error is at most (3k+2) 2^(Er+Ee-57) per
element, within the FP64 bound unless every product of the element lies
far below both its row and its column scale.
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


NEX = 7  # levels moved into int32 sums every 128 rows


def levels_pass1(a, b):
    """Pass-1 level sums as the kernel accumulates them: 16-row MMA steps
    summed in FP32 (exact below 2^24); every 128 rows levels 0 .. NEX-1 are
    moved into int32 (checked for overflow) and restart, levels NEX .. 8 keep
    accumulating in FP32 (rounded)."""
    L = len(a)
    lev_int = [0] * NEX
    lev_f = [np.float32(0.0)] * (ND + 1 - NEX)
    blk = [np.float32(0.0)] * NEX
    for r0 in range(0, L, 16):
        step = levels(a[r0:r0 + 16], b[r0:r0 + 16])
        for lam in range(NEX):
            v = np.float32(blk[lam]) + np.float32(step[lam])
            assert abs(float(v)) < 2 ** 24 and float(v) == float(blk[lam]) + step[lam]  # exact in FP32
            blk[lam] = v
        for lam in range(NEX, ND + 1):
            lev_f[lam - NEX] = np.float32(lev_f[lam - NEX] + np.float32(step[lam]))
        if (r0 // 16) % 8 == 7 or r0 + 16 >= L:
            for lam in range(NEX):
                lev_int[lam] += int(blk[lam])
                assert abs(lev_int[lam]) < 2 ** 31
                blk[lam] = np.float32(0.0)
    return lev_int + [float(v) for v in lev_f]


def guard_pass1(a, bC, kp, nb):
    """Sum of |leading digit| products per (reflector, column): the pass-1
    accuracy guard's quantity (the batch goes to FP64 below 2^11)."""
    L = len(a)
    return np.array([[sum(abs(a[r][t][0]) * abs(bC[r][c][0]) for r in range(L)) for c in range(nb)]
                     for t in range(kp)], dtype=float)


def reflector_scales(V, kp):
    """Ft = exponent bound of reflector t's largest entry (for a Householder
    vector that is its pivot entry v0, |v0| = |x0| + ||x|| >= |x_r|, which
    the kernel uses)."""
    return [max(ebound(v) for v in V[:, t]) for t in range(kp)]


def commit_digits(V, C, T, kp, guard=False):
    """The tensor-core commit restated; with guard=True pass 1's accuracy
    guard too (FP64 for the whole batch when it fires).  The digits cover
    rows [r0d, L); the reflectors' triangle (rows < kp: pivots and the zeros
    above them), rounded up to r0d = a multiple of 8 rows, is summed in
    FP64.  Returns D, E, the updated C and the number of batches sent to FP64
    (0 or 1)."""
    L, nb = V.shape[0], C.shape[1]
    r0d = (kp + 7) & ~7
    Ft = reflector_scales(V, kp)
    Vs = np.array([[math.ldexp(V[r, t], -Ft[t]) for t in range(kp)] for r in range(L)])
    Er = [max(ebound(v) for v in Vs[r, :kp]) for r in range(L)]
    a = [[digits(Vs[r, t], 56 - Er[r]) for t in range(kp)] for r in range(r0d, L)]
    Ec = [max([ebound(C[r, c]) + Er[r] for r in range(r0d, L) if ebound(C[r, c]) > -2000] or [-8000])
          for c in range(nb)]
    bC = [[digits(C[r, c], Er[r] + 56 - Ec[c]) for c in range(nb)] for r in range(r0d, L)]
    fire = False
    if guard:
        S0 = guard_pass1(a, bC, kp, nb)
        for t in range(kp):
            for c in range(nb):
                if Ec[c] == -8000:
                    continue  # no digit rows: no digit error
                tabs = sum(abs(V[r, t]) * abs(C[r, c]) for r in range(t, r0d))
                es = Ec[c] + Ft[t]
                fire |= not (math.ldexp(S0[t, c], es - 14) + tabs >= math.ldexp(2048.0, es - 14))
    if fire:
        D = np.zeros((kp, nb))
        for t in range(kp):
            for c in range(nb):
                acc = 0.0
                for r in range(L):
                    acc = acc + V[r, t] * C[r, c]
                D[t, c] = acc
        E = T[:kp, :kp].T @ D
        Cn = C.copy()
        for r in range(L):
            for c in range(nb):
                x = C[r, c]
                for t in range(kp):
                    x = x - V[r, t] * E[t, c]
                Cn[r, c] = x
        return D, E, Cn, 1
    D = np.zeros((kp, nb))
    for t in range(kp):
        for c in range(nb):
            lev = levels_pass1([a[i][t] for i in range(L - r0d)], [bC[i][c] for i in range(L - r0d)])
            s = float(lev[ND])
            for lam in range(ND - 1, -1, -1):
                s = s * 2.0 ** -7 + lev[lam]
            tri = 0.0
            for r in range(t, r0d):
                tri = tri + V[r, t] * C[r, c]
            D[t, c] = math.ldexp(s, Ec[c] - 14 + Ft[t]) + tri
    E = T[:kp, :kp].T @ D
    return D, E, commit_pass2(V, C, E, kp), 0


def commit_pass2(V, C, E, kp):
    """Pass 2, C - V E: rows [r0d, L) from the digits of V / 2^Ft (row
    scales) and of E'' = 2^Ft E (column scales), the rows below r0d in FP64."""
    L, nb = C.shape
    r0d = (kp + 7) & ~7
    Ft = reflector_scales(V, kp)
    Vs = np.array([[math.ldexp(V[r, t], -Ft[t]) for t in range(kp)] for r in range(L)])
    Er = [max(ebound(v) for v in Vs[r, :kp]) for r in range(L)]
    a = [[digits(Vs[r, t], 56 - Er[r]) for t in range(kp)] for r in range(L)]
    Es = np.array([[math.ldexp(E[t, c], Ft[t]) for c in range(nb)] for t in range(kp)])
    Ee = [max(ebound(Es[t, c]) for t in range(kp)) for c in range(nb)]
    dE = [[digits(Es[t, c], 56 - Ee[c]) for c in range(nb)] for t in range(kp)]
    Cn = C.copy()
    for r in range(L):
        for c in range(nb):
            if r < r0d:
                x = C[r, c]
                for t in range(min(r, kp - 1) + 1):
                    x = x - V[r, t] * E[t, c]
                Cn[r, c] = x
                continue
            lev = levels(a[r], [dE[t][c] for t in range(kp)])
            assert all(abs(v) < 2 ** 24 for v in lev)  # exact in FP32 accumulators
            u = sum(lev[l] << (43 - 7 * l) for l in range(7)) + (lev[7] >> 6) + (lev[8] >> 13)
            assert abs(u) < 2 ** 63
            Cn[r, c] = float(F(C[r, c]) - F(float(u)) * F(2) ** (Er[r] + Ee[c] - 57))
    return Cn


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
        D, E, Cn, _ = commit_digits(V, C, T, kp)
        D64 = V.T @ C
        Dx = [[sum(F(V[r, t]) * F(C[r, c]) for r in range(L)) for c in range(nb)] for t in range(kp)]
        scale = np.abs(V).T @ np.abs(C)
        err = max(abs(float(F(D[t, c]) - Dx[t][c])) / scale[t, c] for t in range(kp) for c in range(nb))
        err64 = max(abs(float(F(D64[t, c]) - Dx[t][c])) / scale[t, c] for t in range(kp) for c in range(nb))
        # pass 1 is within 2^-52 of the magnitude sum, like the FP64 product
        # (the digit part is exact to 2^-56; the triangle rows and the final
        # sum add FP64 roundings; dropping level 8 or truncating digits fails)
        assert err <= 2.0 ** -52 and err <= 2.0 * err64, (err, err64)
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


def gamma(k):
    u = 2.0 ** -53
    return k * u / (1 - k * u)


def bound_ratios(V, C, T, kp, guard):
    """Errors of the digit commit (with or without pass 1's guard) relative
    to the worst-case bounds of the FP64 evaluation, element by element:
    |D - D_exact| / (gamma_L sum |v||c|) and
    |C' - C'_exact| / (gamma_(k+1) (|c| + sum |v||e|) + u |C'|)."""
    L, nb = C.shape
    D, E, Cn, fb = commit_digits(V, C, T, kp, guard=guard)
    Dx = [[sum(F(V[r, t]) * F(C[r, c]) for r in range(L)) for c in range(nb)] for t in range(kp)]
    b1 = gamma(L) * (np.abs(V).T @ np.abs(C))
    r1 = max(abs(float(F(D[t, c]) - Dx[t][c])) / b1[t, c] for t in range(kp) for c in range(nb))
    Cx = [[F(C[r, c]) - sum(F(V[r, t]) * F(E[t, c]) for t in range(kp)) for c in range(nb)] for r in range(L)]
    b2 = gamma(kp + 1) * (np.abs(V) @ np.abs(E) + np.abs(C)) + 2.0 ** -53 * np.abs(Cn)
    r2 = max(abs(float(F(Cn[r, c]) - Cx[r][c])) / b2[r, c] for r in range(L) for c in range(nb))
    return r1, r2, fb


def triangular_V(rng, L, kp):
    V = rng.standard_normal((L, kp))
    for t in range(kp):
        V[:t, t] = 0.0
    return V


def test_triangle_rows_are_exact():
    """C's first row scaled by 2^30 while V(0, t) = 0 for t >= 1 (the zero
    triangle of the reflectors): a fixed point over all rows would let row 0
    set every column scale and lose ~30 bits of D(t >= 1, c); the triangle
    rows are summed in FP64, so both passes stay within the FP64 bounds and
    the guard is not needed."""
    rng = np.random.default_rng(3)
    L, kp, nb = 36, 7, 3
    V = triangular_V(rng, L, kp)
    C = rng.standard_normal((L, nb))
    C[0, :] *= 2.0 ** 30
    T = np.triu(rng.standard_normal((kp, kp)))
    r1, r2, fb = bound_ratios(V, C, T, kp, guard=True)
    assert fb == 0 and r1 <= 1.0 and r2 <= 1.0


def test_guard_catches_large_entry_paired_with_zero():
    """Below the triangle: row 20 of V zero for every reflector but the
    first, and row 20 of C scaled by 2^30.  That row sets the column scale
    of C' while taking no part in D(t >= 1, c), so the unguarded digits lose
    ~30 bits of those sums (far outside the FP64 bound); the guard fires and
    the result is back within the bound."""
    rng = np.random.default_rng(3)
    L, kp, nb = 36, 7, 3
    V = triangular_V(rng, L, kp)
    V[20, 1:] = 0.0
    C = rng.standard_normal((L, nb))
    C[20, :] *= 2.0 ** 30
    T = np.triu(rng.standard_normal((kp, kp)))
    r1, _, _ = bound_ratios(V, C, T, kp, guard=False)
    assert r1 > 1e3
    r1, r2, fb = bound_ratios(V, C, T, kp, guard=True)
    assert fb == 1 and r1 <= 1.0 and r2 <= 1.0


def test_reflectors_of_different_norms():
    """Reflectors whose norms differ by 2^30 (later columns of a correlated
    block keep little of their norm): without the reflector scales the rows
    of V would be set by the large reflectors and the small ones would lose
    30 bits in both passes; with them both passes stay within the FP64
    bounds and the guard stays quiet."""
    rng = np.random.default_rng(4)
    L, kp, nb = 40, 6, 2
    V = triangular_V(rng, L, kp)
    V[:, 1:] *= 2.0 ** -30
    C = rng.standard_normal((L, nb))
    T = np.diag(2.0 / np.sum(V * V, axis=0))  # beta_t = 2 / ||v_t||^2 scales like the reflector
    r1, r2, fb = bound_ratios(V, C, T, kp, guard=True)
    assert fb == 0 and r1 <= 1.0 and r2 <= 1.0


def test_pass2_bound_on_mismatched_scales():
    """The pattern pass 2 does not guard: in every row the largest scaled
    reflector entry meets a tiny D'' entry and the large D'' entries meet
    tiny reflector entries.  The element error then exceeds the FP64 bound,
    but stays within the stated (3k+2) 2^(Er+Ee-57)."""
    rng = np.random.default_rng(6)
    L, kp, nb = 40, 4, 2
    V = triangular_V(rng, L, kp)
    V[kp:, 1:] *= 2.0 ** -20  # rows below the triangle dominated by reflector 0
    E = rng.standard_normal((kp, nb))
    E[0, :] *= 2.0 ** -20     # ... where E is tiny
    C = 2.0 ** -45 * rng.standard_normal((L, nb))
    Cn = commit_pass2(V, C, E, kp)
    Ft = reflector_scales(V, kp)
    Vs = np.array([[math.ldexp(V[r, t], -Ft[t]) for t in range(kp)] for r in range(L)])
    Er = [max(ebound(v) for v in Vs[r]) for r in range(L)]
    Es = np.array([[math.ldexp(E[t, c], Ft[t]) for c in range(nb)] for t in range(kp)])
    Ee = [max(ebound(Es[t, c]) for t in range(kp)) for c in range(nb)]
    worst = 0.0
    for r in range(L):
        for c in range(nb):
            exact = F(C[r, c]) - sum(F(V[r, t]) * F(E[t, c]) for t in range(kp))
            err = abs(float(F(Cn[r, c]) - exact))
            assert err <= (3 * kp + 2) * 2.0 ** (Er[r] + Ee[c] - 57) + 2.0 ** -53 * abs(Cn[r, c])
            fp64 = gamma(kp + 1) * (abs(C[r, c]) + float(np.abs(V[r]) @ np.abs(E[:, c])))
            worst = max(worst, err / fp64)
    assert worst > 1.0  # outside the FP64 bound: the documented limit of pass 2


def test_guard_is_quiet_on_ordinary_operands_long_panel():
    """L = 300 (so pass 1 moves its level sums into int32 twice and keeps
    levels 7-8 in FP32 across the blocks), rows of V and C scaled together
    over 2^-20 .. 2^20: the guard never sends the batch to FP64 and every
    element of both passes is within the FP64 bound."""
    rng = np.random.default_rng(5)
    L, kp, nb = 300, 12, 2
    V = triangular_V(rng, L, kp)
    rs = 2.0 ** rng.integers(-20, 21, size=(L, 1))
    V *= rs
    C = rng.standard_normal((L, nb)) * rs
    T = np.triu(rng.standard_normal((kp, kp))) / 4
    r1, r2, fb = bound_ratios(V, C, T, kp, guard=True)
    assert fb == 0
    assert r1 <= 1.0 and r2 <= 1.0


def test_column_zero_below_the_triangle():
    """A column that left the passive set re-enters with its trailing part
    zero except at the top row (inside the FP64 rows): it has no digit rows,
    so the guard does not send the batch to FP64, and both passes are exact
    to FP64 rounding."""
    rng = np.random.default_rng(9)
    L, kp, nb = 40, 6, 3
    V = triangular_V(rng, L, kp)
    C = rng.standard_normal((L, nb))
    C[1:, 1] = 0.0
    T = np.triu(rng.standard_normal((kp, kp)))
    r1, r2, fb = bound_ratios(V, C, T, kp, guard=True)
    assert fb == 0 and r1 <= 1.0 and r2 <= 1.0
