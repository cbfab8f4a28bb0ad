"""Host-side pin of FP64 mode's error bound (CPU only).

FP64 mode reaches FP64 results on B300's FP32 pipes: the forward transform
a = (A x A x A) u of arXiv 2407.20731 Sec. IV-B's spectral truncation runs in
FP32, and every keep or rounding decision that FP32 value cannot settle is
recomputed exactly.  Which decisions are "settled" rests on one claim: the
FP32 coefficient is within

    M = (3 (H + 2) + 2) 2^-24 2 sqrt(2) 2 max|u'|,   H = ceil(lx / 2),

of the exact one, for the block u' = u 2^-ke that the kernels transform
(ke the binary exponent of the element's largest |u|).  The terms: H + 2
roundings per folded contraction (its H products and sums, the fold, the
FP32 table), three contractions, two more for the round-toward-zero input
conversion; every row of A has sum |A_pi| <= sqrt(2), so |A|^3 |u| <=
2^1.5 max|u|; a factor 2 of safety.  The kernels use max|u'| rounded toward
zero to 20 bits, times 1.000002, in place of max|u'|.

This test replays the kernels' FP32 arithmetic here in numpy, in their
operation order: the integer round-toward-zero conversion of each double
(with the prescale folded into the exponent rebias), then per pencil the
folded sums and differences and the product chain A[p][0] e_0, then
fma(A[p][i], e_i, .) for i = 1 .. H-1 (FMA emulated as the exact float64
product plus the addend, rounded once to float32 -- within a float64 rounding
of a true FMA, far below M), along i, then j, then k.  On adversarial blocks
-- signs aligned with the coefficient being bounded, magnitudes just below
2 (largest round-toward-zero loss), alternating extremes, values deep in
the flush range, raw magnitudes of 2^+-120 -- it asserts |a32 - a| <= M with
a the oracle's FP64 forward transform of u', and that every decision the
kernel takes as settled (|a32| beyond g +- Mg, the rounding screen) is the
exact one.
"""
import math

import numpy as np
import pytest

import oracle


def _rz_prescaled(u):
    """The kernels' integer conversion: float32 of u 2^-ke rounded toward zero
    (bias = 0x38000000 + (ke << 20)), for a whole element block u."""
    bits = np.ascontiguousarray(u, dtype=np.float64).view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.int64)
    lo = (bits & np.uint64(0xFFFFFFFF)).astype(np.int64)
    hmax = int((hi & 0x7FFFFFFF).max())
    ke = 0 if hmax < 0x00100000 else min((hmax >> 20) - 1023, 1023)
    bias = 0x38000000 + (ke << 20)
    t = np.maximum((hi & 0x7FFFFFFF) - bias, 0)
    f = ((t << 3) | (lo >> 29)) & 0xFFFFFFFF
    f = f | (hi & 0x80000000)
    umax = np.array([0x3F800000 | ((hmax & 0xFFFFF) << 3)], dtype=np.uint32).view(np.float32)[0]
    return f.astype(np.uint32).view(np.float32), ke, np.float32(umax)


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _fold_fwd(A32, x):
    """Folded 1-D forward transform along the last axis, in the kernels' order."""
    lx = x.shape[-1]
    H = lx // 2
    ev = [x[..., i] + x[..., lx - 1 - i] for i in range(H)]
    od = [x[..., i] - x[..., lx - 1 - i] for i in range(H)]
    y = np.empty_like(x)
    for p in range(lx):
        if p % 2 == 0:
            if lx % 2:
                s = A32[p, H] * x[..., H]
                for i in range(H):
                    s = _fma(np.full_like(s, A32[p, i]), ev[i], s)
            else:
                s = A32[p, 0] * ev[0]
                for i in range(1, H):
                    s = _fma(np.full_like(s, A32[p, i]), ev[i], s)
        else:
            s = A32[p, 0] * od[0]
            for i in range(1, H):
                s = _fma(np.full_like(s, A32[p, i]), od[i], s)
        y[..., p] = s
    return y


def _fwd32(A32, uh):
    """uh[k, j, i] -> a32[r, q, p]: contract i, then j, then k."""
    y1 = _fold_fwd(A32, uh)                                    # [k, j, p]
    y2 = _fold_fwd(A32, y1.transpose(0, 2, 1)).transpose(0, 2, 1)  # [k, q, p]
    y3 = _fold_fwd(A32, y2.transpose(1, 2, 0)).transpose(2, 0, 1)  # [r, q, p]
    return y3


def _blocks(lx, amat, rng):
    """Adversarial element blocks u[k, j, i] (raw doubles)."""
    n = lx
    out = []
    near2 = 2.0 - 2.0 ** -23 + 0.9 * 2.0 ** -24  # RZ drops ~0.9 of a float ulp
    for (p, q, r) in [(0, 0, 0), (n - 1, n - 1, n - 1), (1, 2, 3), (n - 2, 1, n - 3), (n // 2, n // 2 - 1, 0)]:
        sgn = np.sign(amat[r][:, None, None] * amat[q][None, :, None] * amat[p][None, None, :])
        sgn[sgn == 0] = 1.0
        out.append(near2 * sgn)                                   # all aligned with mode (p, q, r)
        alt = np.where((np.arange(n ** 3).reshape(n, n, n) % 2) == 0, near2, 2.0 ** -20)
        out.append(alt * sgn)                                     # alternating extremes, aligned
        mant = 1.0 + rng.integers(1, 2 ** 52, size=(n, n, n)) * 2.0 ** -52  # full mantissas in [1, 2)
        out.append(mant * sgn)
    out.append(rng.normal(size=(n, n, n)))
    out.append(rng.uniform(-2, 2, size=(n, n, n)))
    spike = rng.choice([-1.0, 1.0], size=(n, n, n)) * 2.0 ** rng.uniform(-130, -118, size=(n, n, n))
    spike[0, 0, 0] = 1.5
    out.append(spike)                                             # values deep in the flush range
    base = [b.copy() for b in out]
    for sc in (2.0 ** 120, 2.0 ** -120):                          # raw magnitudes far from 1
        out += [b * sc for b in base[:4]]
    return out


@pytest.mark.parametrize("lx", [6, 7, 8, 10])
def test_fp32_forward_within_bound_and_settled_decisions_exact(lx):
    rng = np.random.default_rng(lx)
    _, amat = oracle.tables(lx)
    A32 = amat.astype(np.float32)
    H = (lx + 1) // 2
    kmarg = np.float32((3.0 * (H + 2) + 2.0) * 5.9604645e-8 * 2.8285 * 2.0)
    worst = 0.0
    for u in _blocks(lx, amat, rng):
        uh, ke, umax_e = _rz_prescaled(u)
        # the conversion is u 2^-ke rounded toward zero (flushed below 2^-126)
        up = u * 2.0 ** -ke
        ref = np.where(np.abs(up) < 2.0 ** -126, 0.0, up)
        assert np.all(np.abs(uh.astype(np.float64) - ref) <= np.maximum(np.abs(ref) * 2.0 ** -23, 2.0 ** -126))
        assert np.all(np.abs(uh.astype(np.float64)) <= np.abs(up) + 2.0 ** -126)
        a32 = _fwd32(A32, uh).astype(np.float64)
        a = oracle.forward(lx, up)  # exact to ~1e-16 max|u'|
        M = float(kmarg * umax_e * np.float32(1.000002))
        err = np.abs(a32 - a).max()
        assert err <= M, (lx, err, M)
        worst = max(worst, err / M)
        # decisions taken as settled are the exact ones
        S = float(np.sum(a * a))
        for tau in (1e-1, 1e-3, 1e-5):
            t = tau * S
            g = np.float32(math.sqrt(t))
            while float(g) * float(g) < t:
                g = np.nextafter(g, np.float32(np.inf))
            while float(np.nextafter(g, np.float32(0))) ** 2 >= t:
                g = np.nextafter(g, np.float32(0))
            Mg = M + float(g) * 2.4e-7
            aa = np.abs(a32)
            sure_keep = aa >= float(g) + Mg
            sure_drop = aa < float(g) - Mg
            assert np.all(a[sure_keep] ** 2 >= t) and np.all(a[sure_drop] ** 2 < t)
            s = (math.frexp(t)[1] - 1) // 2
            y = aa[sure_keep] * 2.0 ** -s
            Mq = Mg * 2.0 ** -s
            settled = np.abs((y - np.floor(y)) - 0.5) > Mq + y * 1.2e-7
            exact = np.abs(a[sure_keep]) * 2.0 ** -s
            assert np.array_equal(np.rint(y[settled]), np.rint(exact[settled]))
    # the bound is not vacuous: the worst block uses a visible share of it
    assert 0.01 < worst < 1.0, worst
