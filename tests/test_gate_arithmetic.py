"""The arithmetic of the fit kernel's FP64 island, emulated on the CPU.

The kernel decides the outward chi2 gate q - chi2_max det <= 0 in binary32
when the margin exceeds 2^-19 of the magnitudes of its terms, and in FP64
otherwise; it forms the inward chi2 = q / det as q y0 (1 + e) with
e = 1 - det y0 in FP64.  These tests restate that arithmetic with numpy's
binary32 and binary64 operations (each correctly rounded; a binary32 fused
multiply-add is emulated through binary64, whose double rounding differs from
a single rounding with probability of order 2^-29 per operation) and check
the two claims the kernel rests on against exact rational arithmetic:

* whenever the binary32 test is sure, its decision equals the FP64 one;
* the inward chi2 is within 2^-40 of (qh + ql) / det.

No GPU is involved: this pins the reasoning, the GPU parity tests pin the
kernel."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def fma32(a, b, c):
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def fma64(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def two_prod(a, b):
    p = F32(a * b)
    return p, fma32(a, b, -p)


def two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    return s, F32(F32(a - F32(s - bb)) + F32(b - bb))


def quad_form2(S00, S10, S11, r0, r1):
    """r^T adj(S) r as an unevaluated sum qh + ql (compensated dot product)."""
    p1, e1 = two_prod(S11, r0)
    p2, e2 = two_prod(F32(F32(-2.0) * S10), r1)
    uh, ul = two_sum(p1, p2)
    ul = F32(ul + F32(e1 + e2))
    vh = F32(r0 * uh)
    vl = fma32(r0, ul, fma32(r0, uh, -vh))
    t, tl = two_prod(r1, r1)
    wh = F32(S00 * t)
    wl = fma32(S00, tl, fma32(S00, t, -wh))
    qh, ql = two_sum(vh, wh)
    return qh, F32(ql + F32(vl + wl))


def narrow_toward_zero(x: float) -> float:
    """binary64 -> binary32 by truncating the fraction (x in the normal binary32 range)."""
    bits = np.array([x], np.float64).view(np.uint64)[0]
    hi, lo = int(bits >> np.uint64(32)), int(bits & np.uint64(0xFFFFFFFF))
    u = ((((hi - (896 << 20)) << 3) | (lo >> 29)) & 0xFFFFFFFF)
    return np.array([u], np.uint32).view(np.float32)[0]


def cases(n, seed):
    """Innovation matrices of all correlations (up to 0.999) and residuals on or near the gate."""
    rng = np.random.default_rng(seed)
    for _ in range(n):
        a, b = 10.0 ** rng.uniform(-4, 0, 2)
        rho = rng.uniform(-0.999, 0.999)
        c = rho * np.sqrt(a * b)
        S00, S11, S10 = F32(a), F32(b), F32(c)
        L = np.linalg.cholesky(np.array([[a, c], [c, b]]))
        z = rng.normal(size=2)
        z /= np.linalg.norm(z)
        k = 4.0 * (1.0 + rng.normal() * 10.0 ** rng.uniform(-9, -1))
        r = L @ (z * k)
        yield S00, S10, S11, F32(r[0]), F32(r[1])


def test_binary32_gate_is_the_fp64_gate_when_sure():
    g = F32(16.0)
    sure_n = 0
    for S00, S10, S11, r0, r1 in cases(20000, 1):
        qh, ql = quad_form2(S00, S10, S11, r0, r1)
        det = fma64(float(S00), float(S11), -float(S10) * float(S10))  # exact products, one rounding
        d32 = narrow_toward_zero(det)
        m = F32(fma32(-g, d32, qh) + ql)
        mag = F32(fma32(g, d32, abs(qh)) + abs(ql))
        fp64 = fma64(-16.0, det, float(qh)) + float(ql)  # the kernel's FP64 evaluation
        if abs(m) > F32(F32(2.0 ** -19) * mag):
            sure_n += 1
            assert (m < 0) == (fp64 <= 0.0), (S00, S10, S11, r0, r1)
    assert sure_n > 10000  # most cases are decided in binary32 even this close to the boundary


def test_inward_chi2_within_2_to_minus_40():
    worst = 0.0
    for S00, S10, S11, r0, r1 in cases(5000, 2):
        qh, ql = quad_form2(S00, S10, S11, r0, r1)
        det = fma64(float(S00), float(S11), -float(S10) * float(S10))
        y0 = F32(F32(1.0) / narrow_toward_zero(det))
        qn = F32(qh + ql)
        qnl = F32(ql - F32(qn - qh))
        p, pe = two_prod(qn, y0)
        pl = fma32(qnl, y0, pe)
        e = fma64(-det, float(y0), 1.0)
        chi2 = float(p) + fma64(float(p), e, float(pl))
        exact = (Fraction(float(qh)) + Fraction(float(ql))) / Fraction(det)
        worst = max(worst, abs(float((Fraction(chi2) - exact) / exact)))
    assert worst < 2.0 ** -40
