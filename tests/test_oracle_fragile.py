"""Pins of the oracle's fragile list, kinds 1-3 (CPU only).

The fragile list names the decisions of the method that an FP64 rounding
difference could flip: the keep test a_m^2 >= tau S_e (kind 1), the
round-half-to-even of a kept code a_m / q_e (kind 2) and the binary exponent
of t = tau S_e that fixes the step q_e (kind 3).  The GPU path may differ from
the oracle only there, so the list must hold every such decision and nothing
else: too few entries would fail correct kernels, too many would hide wrong
ones.  The method is the spectral truncation and quantisation of arXiv
2407.20731, Sec. IV-B, with the decisions as the oracle states them.

Each block is built here in modal space with one decision planted at a chosen
distance from its tie, turned into nodal values by the oracle's inverse
transform, and reduced by the oracle, whose forward transform brings back the
planted coefficients up to about 1e-16 relative.  The planted distance 1e-12
(kind 1), 1e-13 (kind 2) or an exact tie (kind 3) lies inside the list's 1e-9
band, so the entry must be there, at that element and mode; the same block
moved 1e-6 away must have no entry at all.  The other coefficients of every
block are chosen far from every tie (dropped modes at about a tenth of the
threshold energy, the kept dominant mode at an integer code, mu away from 1/2
and 1), which the test also checks from the oracle's own coefficients.
"""
import math

import numpy as np
import pytest

import oracle

TAU = 2.0 ** -7  # a power of two: t = tau S_e is S_e with its exponent moved, no rounding


def _step(t):
    m, ex = math.frexp(t)  # t = m 2^ex, m in [1/2, 1)
    return (ex - 1) // 2, m


def _base(n3):
    a = np.zeros(n3)
    a[0] = 1.0
    for m, v in ((5, 0.021), (9, -0.017), (22, 0.013), (41, -0.019)):  # dropped: a^2 ~ t / 10
        a[m] = v
    return a


def _kind1(n3, delta, m1=17):
    """Mode m1 with a^2 = tau S (1 + delta), S including a^2 itself."""
    a = _base(n3)
    rest = float(np.sum(a * a))
    c = TAU * (1.0 + delta)
    a[m1] = math.sqrt(c * rest / (1.0 - c))
    return a


def _kind2(n3, eps, m2=33, k=2):
    """Kept mode m2 with |a| / q = k + 1/2 + eps."""
    a = _base(n3)
    s, _ = _step(TAU * float(np.sum(a * a)))
    a[m2] = (k + 0.5 + eps) * 2.0 ** s
    assert _step(TAU * float(np.sum(a * a)))[0] == s  # the added mode leaves the step alone
    return a


def _kind3(n3, mu):
    """t = tau S = mu 2^-6: S = 2 mu, set through the dominant mode."""
    a = _base(n3)
    rest = float(np.sum(a * a)) - 1.0
    a[0] = math.sqrt(2.0 * mu - rest)
    return a


CASES = [  # (name, builder, planted decision (mode or -1 for the step, kind), flagged?)
    ("threshold +1e-12", lambda n: _kind1(n, 1e-12), (17, 1), True),
    ("threshold -1e-12", lambda n: _kind1(n, -1e-12), (17, 1), True),
    ("threshold +1e-6", lambda n: _kind1(n, 1e-6), (17, 1), False),
    ("threshold -1e-6", lambda n: _kind1(n, -1e-6), (17, 1), False),
    ("rounding +1e-13", lambda n: _kind2(n, 1e-13), (33, 2), True),
    ("rounding -1e-13", lambda n: _kind2(n, -1e-13), (33, 2), True),
    ("rounding +1e-6", lambda n: _kind2(n, 1e-6), (33, 2), False),
    ("rounding -1e-6", lambda n: _kind2(n, -1e-6), (33, 2), False),
    ("mu = 1/2", lambda n: _kind3(n, 0.5), (-1, 3), True),
    ("mu = 1 - 2^-52", lambda n: _kind3(n, 1.0 - 2.0 ** -52), (-1, 3), True),
    ("mu = 1/2 (1 + 1e-6)", lambda n: _kind3(n, 0.5 * (1.0 + 1e-6)), (-1, 3), False),
    ("mu = 1 - 1e-6", lambda n: _kind3(n, 1.0 - 1e-6), (-1, 3), False),
]


@pytest.mark.parametrize("lx", [4, 6, 8])
def test_planted_ties_are_listed_and_clear_gaps_are_not(lx):
    n3 = lx ** 3
    blocks = [oracle.inverse(lx, b(n3).reshape(lx, lx, lx)).reshape(-1) for _, b, _, _ in CASES]
    u = np.stack(blocks)[None]
    r = oracle.reduce(u, np.ones(len(CASES)), TAU, fragile_cap=1000)
    listed = {}
    for f, e, m, k in r.fragile.tolist():
        assert f == 0
        listed.setdefault(e, set()).add((m, k))
    for e, (name, _, planted, flagged) in enumerate(CASES):
        got = listed.get(e, set())
        assert got == ({planted} if flagged else set()), (lx, name, got)
    assert r.n_fragile == sum(fl for _, _, _, fl in CASES)

    # the rest of each block is far from every tie (checked on the oracle's own coefficients)
    for e, (name, _, planted, _) in enumerate(CASES):
        a = r.coeffs[0, e]
        t = TAU * float(np.sum(a * a))
        s, mu = _step(t)
        if planted[1] != 3:
            assert 1e-3 < abs(mu - 0.5) and 1e-3 < abs(mu - 1.0), (name, mu)
        q = 2.0 ** s
        for m in range(n3):
            if m == planted[0]:
                continue
            e2 = a[m] * a[m]
            assert abs(e2 - t) > 1e-3 * t, (name, m)
            if e2 >= t:
                y = abs(a[m]) / q
                assert abs((y - math.floor(y)) - 0.5) > 1e-3, (name, m, y)


def test_planted_decisions_go_the_planted_way():
    """Outside the 1e-9 band the planted decisions come out as planted: the
    threshold mode kept 1e-6 above t and dropped 1e-6 below, and the code
    planted 1e-6 above or below a half-integer rounded to the nearer integer."""
    lx, n3 = 4, 64
    names = ["threshold +1e-6", "threshold -1e-6", "rounding +1e-6", "rounding -1e-6"]
    builders = {n: b for n, b, _, _ in CASES}
    u = np.stack([oracle.inverse(lx, builders[n](n3).reshape(lx, lx, lx)).reshape(-1) for n in names])[None]
    r = oracle.reduce(u, np.ones(len(names)), TAU)
    s = oracle.sections(r.payload)
    assert s["masks"][0, 0, 17] and not s["masks"][0, 1, 17]
    codes = s["codes"].astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(s["counts"][0].astype(np.int64))])
    # elements 2 and 3: modes 0 and 33 kept; |code 33| = 3 above the half, 2 below
    assert list(np.nonzero(s["masks"][0, 2])[0]) == [0, 33]
    assert abs(codes[offs[2] + 1]) == 3 and abs(codes[offs[3] + 1]) == 2
