"""Pins of the CPU oracle against mathematics it does not compute itself.

Each test checks the oracle against something fixed outside it: closed forms
of the Legendre polynomials and of the small Lobatto rules, high-precision
roots from mpmath, quadrature exactness, brute-force Kronecker products built
here from numpy's Legendre evaluation, Parseval's identity, exact rational
arithmetic for the step exponent, and the special cases of the method (tau = 0
lossless, tau >= 1, zero blocks, single modes, constants).  The method is the
lossy SEM compression of arXiv 2407.20731, Sec. IV-B.
"""
import math
import os
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
import synth

LX_ALL = list(range(2, 17))


# --------------------------------------------------------------- Legendre

@pytest.mark.parametrize("x", [-1.0, -0.73, -0.2, 0.0, 0.31, 0.5, 0.999, 1.0])
def test_legendre_closed_forms(x):
    closed = {
        0: 1.0,
        1: x,
        2: (3 * x**2 - 1) / 2,
        3: (5 * x**3 - 3 * x) / 2,
        4: (35 * x**4 - 30 * x**2 + 3) / 8,
        5: (63 * x**5 - 70 * x**3 + 15 * x) / 8,
    }
    for k, v in closed.items():
        assert oracle.legendre(k, x) == pytest.approx(v, abs=1e-15)


def test_legendre_end_value_and_parity():
    for k in range(0, 17):
        assert oracle.legendre(k, 1.0) == pytest.approx(1.0, abs=1e-14)
        for x in (0.13, 0.57, 0.91):
            assert oracle.legendre(k, -x) == pytest.approx((-1) ** k * oracle.legendre(k, x), abs=1e-14)


# ------------------------------------------------------------- GLL rule

def _closed_form(expr):
    """Value of an expression of numbers, + - * / ( ) and sqrt (the golden
    table's notation), evaluated by walking its syntax tree."""
    import ast
    import operator as op
    ops = {ast.Add: op.add, ast.Sub: op.sub, ast.Mult: op.mul, ast.Div: op.truediv, ast.USub: op.neg}

    def ev(n):
        if isinstance(n, ast.Expression):
            return ev(n.body)
        if isinstance(n, ast.Constant) and isinstance(n.value, (int, float)):
            return float(n.value)
        if isinstance(n, ast.BinOp) and type(n.op) in ops:
            return ops[type(n.op)](ev(n.left), ev(n.right))
        if isinstance(n, ast.UnaryOp) and type(n.op) in ops:
            return ops[type(n.op)](ev(n.operand))
        if isinstance(n, ast.Call) and isinstance(n.func, ast.Name) and n.func.id == "sqrt" and len(n.args) == 1:
            return math.sqrt(ev(n.args[0]))
        raise ValueError(f"unsupported expression {expr!r}")
    return ev(ast.parse(expr.strip(), mode="eval"))


def _golden_gll():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gll_lobatto_closed_forms.txt")
    table = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            lx, xs, ws = (part.strip() for part in line.split("|"))
            table[int(lx)] = ([_closed_form(v) for v in xs.split(";")], [_closed_form(v) for v in ws.split(";")])
    return table


def test_gll_closed_forms():
    """The oracle's GLL rule against the textbook Lobatto tables
    (tests/golden/gll_lobatto_closed_forms.txt), lx = 2..6."""
    table = _golden_gll()
    assert sorted(table) == [2, 3, 4, 5, 6]
    for lx, (xs, ws) in table.items():
        x, w = oracle.gll(lx)
        np.testing.assert_allclose(x, xs, rtol=0, atol=2e-15)
        np.testing.assert_allclose(w, ws, rtol=0, atol=2e-15)


@pytest.mark.parametrize("lx", LX_ALL)
def test_gll_nodes_match_high_precision_roots(lx):
    """Interior nodes are the roots of P_N' (mpmath at 40 digits)."""
    N = lx - 1
    x, w = oracle.gll(lx)
    mpmath.mp.dps = 40
    if N >= 2:
        # coefficients of P_N' from the Legendre power-series coefficients
        coeffs = np.polynomial.legendre.leg2poly([0] * N + [1])
        dcoef = [mpmath.mpf(int(round(c * 2**N))) / 2**N for c in coeffs]
        deriv = [k * dcoef[k] for k in range(1, N + 1)]
        roots = sorted(float(mpmath.re(r)) for r in mpmath.polyroots(deriv[::-1], maxsteps=200, extraprec=200))
        np.testing.assert_allclose(x[1:-1], roots, rtol=0, atol=1e-14)
    assert x[0] == -1.0 and x[-1] == 1.0
    # weights: w_j = 2 / (N (N+1) P_N(x_j)^2), P_N evaluated by mpmath
    for j in range(lx):
        pn = mpmath.legendre(N, mpmath.mpf(x[j]))
        assert w[j] == pytest.approx(float(2 / (N * (N + 1) * pn**2)), rel=1e-14)


@pytest.mark.parametrize("lx", LX_ALL)
def test_gll_quadrature_exactness(lx):
    """Exact for x^d, d <= 2N-1; not exact at d = 2N (that is what makes it the
    Lobatto rule and not a Gauss rule)."""
    N = lx - 1
    x, w = oracle.gll(lx)
    assert w.sum() == pytest.approx(2.0, abs=1e-14)
    for d in range(0, 2 * N):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert np.dot(w, x**d) == pytest.approx(exact, abs=2e-14)
    d = 2 * N
    assert abs(np.dot(w, x**d) - 2.0 / (d + 1)) > 1e-10


# ----------------------------------------------------------- basis tables

def _indep_basis(lx):
    """Phi and A built here: nodes from mpmath roots, orthonormal Legendre
    from numpy's legval, gamma_N = 2/N for the top mode."""
    N = lx - 1
    x, w = oracle.gll(lx)  # nodes/weights already pinned above
    phi = np.zeros((lx, lx))
    for k in range(lx):
        c = np.zeros(k + 1)
        c[k] = 1.0
        gamma = 2.0 / (2 * k + 1) if k < N else 2.0 / N
        phi[:, k] = np.polynomial.legendre.legval(x, c) / math.sqrt(gamma)
    return phi, phi.T * w[None, :], w


@pytest.mark.parametrize("lx", LX_ALL)
def test_basis_tables_against_numpy_legval(lx):
    phi, amat = oracle.tables(lx)
    phi_i, amat_i, _ = _indep_basis(lx)
    np.testing.assert_allclose(phi, phi_i, rtol=0, atol=1e-13)
    np.testing.assert_allclose(amat, amat_i, rtol=0, atol=1e-13)


@pytest.mark.parametrize("lx", LX_ALL)
def test_basis_discrete_orthonormality(lx):
    phi, amat = oracle.tables(lx)
    _, w = oracle.gll(lx)
    g = phi.T @ np.diag(w) @ phi
    assert np.abs(g - np.eye(lx)).max() <= 1e-13
    assert np.abs(amat @ phi - np.eye(lx)).max() <= 1e-13


# -------------------------------------------------------------- transform

@pytest.mark.parametrize("lx", [2, 3, 4, 5])
def test_forward_matches_bruteforce_kronecker(lx):
    rng = np.random.default_rng(lx)
    _, amat_i, _ = _indep_basis(lx)
    K = np.kron(np.kron(amat_i, amat_i), amat_i)  # K[(r,q,p),(k,j,i)]
    for _ in range(4):
        u = rng.normal(size=(lx, lx, lx))
        a = oracle.forward(lx, u)
        np.testing.assert_allclose(a.reshape(-1), K @ u.reshape(-1), rtol=0, atol=1e-13)
        phi_i, _, _ = _indep_basis(lx)
        Kinv = np.kron(np.kron(phi_i, phi_i), phi_i)
        np.testing.assert_allclose(oracle.inverse(lx, a).reshape(-1), Kinv @ a.reshape(-1),
                                   rtol=0, atol=1e-13)


@pytest.mark.parametrize("lx", [3, 6, 8, 10])
def test_single_mode_input(lx):
    phi_i, _, _ = _indep_basis(lx)
    rng = np.random.default_rng(100 + lx)
    for _ in range(6):
        p, q, r = rng.integers(0, lx, size=3)
        u = np.einsum("k,j,i->kji", phi_i[:, r], phi_i[:, q], phi_i[:, p])
        a = oracle.forward(lx, u).reshape(-1)
        m = p + lx * (q + lx * r)
        e = np.zeros(lx**3)
        e[m] = 1.0
        np.testing.assert_allclose(a, e, rtol=0, atol=1e-13)


@pytest.mark.parametrize("lx", [2, 5, 8, 10])
def test_constant_input(lx):
    c = 1.7
    a = oracle.forward(lx, np.full((lx, lx, lx), c)).reshape(-1)
    assert a[0] == pytest.approx(c * 2**1.5, rel=1e-14)
    assert np.abs(a[1:]).max() <= 1e-14


@pytest.mark.parametrize("lx", LX_ALL)
def test_forward_inverse_identity_and_parseval(lx):
    rng = np.random.default_rng(7 * lx)
    _, w = oracle.gll(lx)
    W3 = np.einsum("k,j,i->kji", w, w, w)
    for _ in range(3):
        u = rng.normal(size=(lx, lx, lx)) * rng.uniform(0.1, 10)
        a = oracle.forward(lx, u)
        back = oracle.inverse(lx, a)
        assert np.abs(back - u).max() <= 1e-13 * np.abs(u).max()
        assert abs((W3 * u * u).sum() - (a * a).sum()) <= 1e-13 * (a * a).sum()


# --------------------------------------------------- truncation / quantisation

def _case(ne=64, lx=8, seed=3, nf=1):
    f, j = synth.snapshot(ne, lx, [seed + i for i in range(nf)])
    return f.numpy().reshape(nf, ne, -1), j.numpy()


def test_lossless_at_tau_zero():
    f, j = _case(ne=27, lx=6)
    r = oracle.reduce(f, j, 0.0)
    s = oracle.sections(r.payload)
    assert s["header"]["flags"] & oracle.FLAG_LOSSLESS
    assert s["masks"].all()
    assert (s["counts"] == 6**3).all()
    np.testing.assert_array_equal(s["codes"], r.coeffs.reshape(-1))
    assert np.abs(r.recon - f).max() <= 1e-13 * np.abs(f).max()
    assert r.n_fragile == 0


def test_bruteforce_mask_codes_tiny():
    """lx = 2 and 3: mask, steps and codes recomputed here from Kronecker
    coefficients and exact rational step exponents."""
    for lx in (2, 3):
        rng = np.random.default_rng(lx)
        ne = 40
        f = rng.normal(size=(1, ne, lx**3)) * rng.uniform(0.01, 100, size=(1, ne, 1))
        j = rng.uniform(0.5, 2.0, size=ne)
        tau = 0.05
        r = oracle.reduce(f, j, tau)
        s = oracle.sections(r.payload)
        _, amat_i, _ = _indep_basis(lx)
        K = np.kron(np.kron(amat_i, amat_i), amat_i)
        pos = 0
        for e in range(ne):
            a = K @ f[0, e]
            S = float(np.sum(a * a))
            t = tau * S
            keep = a * a >= t
            fr = set(map(tuple, r.fragile[:, 1:3].tolist()))
            if any((e, m) in fr for m in range(lx**3)) or (e, -1) in fr:
                pos += int(s["counts"][0, e])
                continue
            np.testing.assert_array_equal(s["masks"][0, e], keep)
            # s = floor(log2 sqrt(t)) exactly: 4^s <= t < 4^(s+1)
            sv = int(s["steps"][0, e])
            T = Fraction(t)
            assert Fraction(4) ** sv <= T < Fraction(4) ** (sv + 1)
            q = 2.0**sv
            codes = np.rint(a[keep] / q)
            np.testing.assert_array_equal(s["codes"][pos:pos + keep.sum()], codes)
            pos += int(keep.sum())


def test_step_exponent_exact_rational():
    f, j = _case(ne=125, lx=8, seed=5)
    for tau in (1e-2, 1e-3, 3.7e-5):
        r = oracle.reduce(f, j, tau)
        s = oracle.sections(r.payload)
        flagged = {int(e) for e, m, k in r.fragile[:, 1:4] if m == -1}
        for e in range(125):
            if e in flagged:
                continue
            S = 0.0
            for v in r.coeffs[0, e]:
                S += v * v
            T = Fraction(tau * S)
            sv = int(s["steps"][0, e])
            assert Fraction(4) ** sv <= T < Fraction(4) ** (sv + 1)


def test_code_magnitude_bounds():
    f, j = _case(ne=125, lx=8, seed=9)
    for tau in (1e-1, 1e-3, 1e-6):
        r = oracle.reduce(f, j, tau)
        s = oracle.sections(r.payload)
        c = np.abs(s["codes"].astype(np.int64))
        assert c.min() >= 1
        assert c.max() <= 2.0 / math.sqrt(tau)


def test_mask_monotone_in_tau():
    f, j = _case(ne=64, lx=8, seed=11)
    prev = None
    for tau in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1):
        m = oracle.sections(oracle.reduce(f, j, tau).payload)["masks"]
        if prev is not None:
            assert not np.any(m & ~prev)
        prev = m


def test_tau_at_or_above_one():
    lx = 6
    f, j = _case(ne=27, lx=lx, seed=13)
    r = oracle.reduce(f, j, 1.5)
    assert oracle.sections(r.payload)["counts"].sum() == 0
    phi_i, _, _ = _indep_basis(lx)
    u = 3.0 * np.einsum("k,j,i->kji", phi_i[:, 2], phi_i[:, 1], phi_i[:, 4]).reshape(1, 1, -1)
    r = oracle.reduce(u, np.array([1.3]), 0.999)
    s = oracle.sections(r.payload)
    assert s["counts"][0, 0] == 1 and s["masks"][0, 0, 4 + lx * (1 + lx * 2)]


def test_zero_block():
    lx = 8
    f = np.zeros((1, 3, lx**3))
    f[0, 1] = 1e-3 * np.arange(lx**3)
    r = oracle.reduce(f, np.ones(3), 1e-3)
    s = oracle.sections(r.payload)
    assert s["counts"][0, 0] == 0 and s["steps"][0, 0] == -32768
    assert s["counts"][0, 2] == 0 and s["steps"][0, 2] == -32768
    assert np.all(r.recon[0, 0] == 0.0) and np.all(r.elem_report[0, 0] == 0.0)


def test_code_width_switch():
    f, j = _case(ne=8, lx=6, seed=17)
    assert oracle.parse_header(oracle.reduce(f, j, 1e-8).payload)["flags"] == 0
    h = oracle.parse_header(oracle.reduce(f, j, 1e-9).payload)
    assert h["flags"] & oracle.FLAG_CODE32


# -------------------------------------------------------------- error norms

def test_nodal_error_equals_modal_parseval():
    f, j = _case(ne=64, lx=8, seed=19, nf=2)
    tau = 1e-3
    r = oracle.reduce(f, j, tau)
    s = oracle.sections(r.payload)
    a = r.coeffs
    # a~ from the payload: codes times 2^s at the kept modes
    at = np.zeros_like(a)
    pos = 0
    for fi in range(2):
        for e in range(64):
            m = s["masks"][fi, e]
            n = int(m.sum())
            at[fi, e, m] = np.ldexp(s["codes"][pos:pos + n].astype(np.float64), int(s["steps"][fi, e]))
            pos += n
    modal = j[None, :] * ((a - at) ** 2).sum(axis=2)
    np.testing.assert_allclose(r.elem_report[:, :, 0], modal, rtol=1e-12, atol=0)
    energy = j[None, :] * (a * a).sum(axis=2)
    np.testing.assert_allclose(r.elem_report[:, :, 1], energy, rtol=1e-12)
    # and the truncation/quantisation bound
    S = (a * a).sum(axis=2)
    q = np.ldexp(1.0, s["steps"].astype(np.int64))
    kept = s["counts"].astype(np.float64)
    bound = j[None, :] * ((512 - kept) * tau * S + kept * q * q / 4)
    assert np.all(r.elem_report[:, :, 0] <= bound * (1 + 1e-12))
    # Linf is the unweighted nodal max
    np.testing.assert_array_equal(r.elem_report[:, :, 2], np.abs(f - r.recon).max(axis=2))


def test_field_norms_from_element_rows():
    f, j = _case(ne=64, lx=6, seed=23, nf=3)
    r = oracle.reduce(f, j, 1e-4)
    er, fr = r.elem_report, r.field_report
    se2, sen = er[:, :, 0].sum(axis=1), er[:, :, 1].sum(axis=1)
    np.testing.assert_allclose(fr[:, 0], np.sqrt(se2), rtol=1e-13)
    np.testing.assert_allclose(fr[:, 1], np.sqrt(se2 / sen), rtol=1e-13)
    np.testing.assert_array_equal(fr[:, 2], er[:, :, 2].max(axis=1))
    np.testing.assert_array_equal(fr[:, 6], np.abs(f).max(axis=(1, 2)))
    np.testing.assert_allclose(fr[:, 3], fr[:, 2] / fr[:, 6], rtol=1e-15)


# ------------------------------------------------------------------ payload

@pytest.mark.parametrize("lx,nf,ne,tau", [(8, 1, 64, 1e-3), (6, 3, 50, 1e-2), (10, 2, 9, 1e-5), (8, 2, 5, 0.0)])
def test_payload_roundtrip_and_size(lx, nf, ne, tau):
    f, j = _case(ne=ne, lx=lx, seed=29, nf=nf)
    r = oracle.reduce(f, j, tau)
    h = oracle.parse_header(r.payload)
    assert (h["lx"], h["n_fields"], h["n_elem"], h["tau"]) == (lx, nf, ne, tau)
    s = oracle.sections(r.payload)
    assert h["code_total"] == int(s["counts"].astype(np.int64).sum())
    np.testing.assert_array_equal(h["code_count"], s["counts"].astype(np.int64).sum(axis=1))
    width = s["width"]
    mb = (lx**3 + 7) // 8
    pad = lambda v: (v + 15) // 16 * 16  # noqa: E731
    expect = pad(48 + 8 * nf) + nf * (pad(ne * mb) + 2 * pad(2 * ne)) + width * h["code_total"]
    assert r.payload.size == expect
    assert np.array_equal(oracle.decode(r.payload), r.recon)
    np.testing.assert_array_equal(s["masks"].sum(axis=2), s["counts"])


def _paper_claims():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_claims.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = (part.strip() for part in line.split("|"))
            out[k] = float(v)
    return out


def test_compression_ratio_eq1():
    """Eq. 1, CR = 1 - compressed / original bytes, with the payload's size
    from its sections (header, 64 mask bytes + step + count per element,
    2 bytes per kept code); and, as context only, the paper's one
    quantitative compression claim (tests/golden/paper_claims.txt: about
    98 % compressed at a maximal allowed error of 1e-2, Sec. IV-B, lossy and
    lossless stages on the paper's own data): the lossy stage alone, on the
    synthetic stand-in at the same threshold, lands within a few percent."""
    claims = _paper_claims()
    tau = claims["max_allowed_error"]
    f, j = _case(ne=125, lx=8, seed=31)
    r = oracle.reduce(f, j, tau)
    sec = oracle.sections(r.payload)
    E = f.shape[1]
    n_codes = int(sec["counts"].sum())
    assert sec["width"] == 2 and sec["codes"].size == n_codes
    assert r.payload.size == oracle.header_bytes(1) + oracle.field_fixed_bytes(8, E) + 2 * n_codes
    orig = f.size * 8
    cr = (orig - r.payload.size) / orig
    assert abs(cr - claims["compressed_fraction_about"]) < 0.02, cr


# --------------------------------------------------- cumulative-energy variant

def _cum_bruteforce(e, t):
    """Largest energy value v with sum of strictly smaller energies <= t
    (exact rational sums); keep e >= v.  None when every mode fits."""
    vals = sorted(set(e.tolist()))
    best = None
    for v in vals:
        d = sum(Fraction(x) for x in e.tolist() if x < v)
        if d <= Fraction(t):
            best = v
    if sum(Fraction(x) for x in e.tolist()) <= Fraction(t):
        return None
    return best


@pytest.mark.parametrize("lx", [2, 3, 4])
def test_cumulative_bruteforce_tiny(lx):
    rng = np.random.default_rng(200 + lx)
    ne = 30
    f = rng.normal(size=(1, ne, lx ** 3)) * np.exp(rng.normal(size=(1, ne, lx ** 3)))
    j = rng.uniform(0.5, 2.0, size=ne)
    for tau in (0.02, 0.2):
        r = oracle.reduce(f, j, tau, cumulative=True)
        s = oracle.sections(r.payload)
        assert s["header"]["flags"] & oracle.FLAG_CUMULATIVE
        flagged = {int(e) for _, e, m, k in r.fragile if k == 4}
        for e in range(ne):
            if e in flagged:
                continue
            a = r.coeffs[0, e]
            en = a * a
            S = 0.0
            for v in a:
                S += v * v
            v = _cum_bruteforce(en, tau * S)
            expect = np.zeros(lx ** 3, bool) if v is None else en >= v
            np.testing.assert_array_equal(s["masks"][0, e], expect)


def test_cumulative_budget_invariants():
    f, j = _case(ne=125, lx=8, seed=37)
    for tau in (1e-5, 1e-3, 1e-1):
        r = oracle.reduce(f, j, tau, cumulative=True)
        s = oracle.sections(r.payload)
        flagged = {int(e) for _, e, m, k in r.fragile if k == 4}
        for e in range(125):
            if e in flagged:
                continue
            en = r.coeffs[0, e] ** 2
            S = float(np.sum(en))
            kept = s["masks"][0, e]
            dropped = float(np.sum(en[~kept]))
            assert dropped <= tau * S * (1 + 1e-12)
            if kept.any():  # dropping the smallest kept energy as well would break the budget
                assert dropped + en[kept].min() > tau * S * (1 - 1e-12)


def test_cumulative_monotone_and_limits():
    f, j = _case(ne=64, lx=6, seed=39)
    prev = None
    for tau in (1e-6, 1e-4, 1e-2, 0.5):
        m = oracle.sections(oracle.reduce(f, j, tau, cumulative=True).payload)["masks"]
        if prev is not None:
            assert not np.any(m & ~prev)
        prev = m
    assert oracle.sections(oracle.reduce(f, j, 1.5, cumulative=True).payload)["counts"].sum() == 0
    r = oracle.reduce(f, j, 0.0, cumulative=True)  # tau = 0 stays lossless
    assert oracle.sections(r.payload)["masks"].all()


def test_cumulative_near_tie_flagged():
    """Two modes of (nearly) equal energy straddle the cumulative boundary (the
    budget fits one of them, not both): which one is kept depends on rounding,
    so the element is fragile (kind 4).  An exact tie keeps both (equal
    energies are kept together); moving one energy well away clears the flag."""
    lx, tau = 4, 1e-2
    n = lx ** 3
    blocks = []
    for x2 in (0.6, 0.6 * (1 + 1e-12), 0.6 * 1.5):  # exact tie, near tie, clear gap
        a = np.zeros(n)
        a[0] = 1.0
        a[5] = math.sqrt(0.6 * tau)  # energy 0.6 t (with S ~ 1)
        a[9] = math.sqrt(x2 * tau)
        blocks.append(oracle.inverse(lx, a).reshape(-1))
    f = np.stack(blocks)[None]
    r = oracle.reduce(f, np.ones(3), tau, cumulative=True)
    kinds = {(int(e), int(k)) for _, e, m, k in r.fragile}
    assert (0, 4) in kinds and (1, 4) in kinds
    assert (2, 4) not in kinds
    c = r.coeffs[0]
    m = oracle.sections(r.payload)["masks"][0]
    for e in range(3):
        assert m[e, 0]
        # the larger of the pair always survives; the smaller only on an exact tie
        big, small = (9, 5) if c[e, 9] ** 2 >= c[e, 5] ** 2 else (5, 9)
        assert m[e, big]
        assert m[e, small] == (c[e, 5] ** 2 == c[e, 9] ** 2)
    assert m[2, 9] and not m[2, 5]


# --------------------------------------------------- slice image (Sec. IV-A)

import oracle.slice as oslice  # noqa: E402


@pytest.mark.parametrize("lx", [2, 5, 8, 12])
def test_slice_basis_partition_kronecker_polynomials(lx):
    nodes, _ = oracle.gll(lx)
    x = np.linspace(-1.0, 1.0, 37)
    L = oslice.lagrange(nodes, x)
    np.testing.assert_allclose(L.sum(axis=1), 1.0, atol=1e-13)         # partition of unity
    np.testing.assert_allclose(oslice.lagrange(nodes, nodes), np.eye(lx), atol=1e-14)  # Kronecker
    for d in range(lx):                                                 # degree <= N reproduced
        np.testing.assert_allclose(L @ nodes ** d, x ** d, atol=1e-12)


def _poly_mesh(lx, n, mo, h, seed):
    """Nodal values of a polynomial of per-axis degree lx - 1 on a lattice,
    and the closed form."""
    rng = np.random.default_rng(seed)
    cx, cy, cz = (rng.normal(size=lx) for _ in range(3))
    f = lambda X, Y, Z: (np.polyval(cx, X / 3.0) * np.polyval(cy, Y / 3.0) + np.polyval(cz, Z / 3.0))  # noqa: E731
    nodes, _ = oracle.gll(lx)
    ex, ey, ez = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    # element e = ex + nx (ey + ny ez); block [k][j][i]
    E = n[0] * n[1] * n[2]
    u = np.zeros((E, lx, lx, lx))
    for e in range(E):
        ix, iy, iz = e % n[0], (e // n[0]) % n[1], e // (n[0] * n[1])
        X = mo[0] + h[0] * (ix + 0.5 * (nodes + 1.0))
        Y = mo[1] + h[1] * (iy + 0.5 * (nodes + 1.0))
        Z = mo[2] + h[2] * (iz + 0.5 * (nodes + 1.0))
        u[e] = f(X[None, None, :], Y[None, :, None], Z[:, None, None])
    return u, f


@pytest.mark.parametrize("lx", [3, 6, 8])
def test_slice_reproduces_polynomials(lx):
    n, mo, h = (3, 4, 2), (-1.0, 0.5, 2.0), (0.7, 0.45, 1.3)
    u, f = _poly_mesh(lx, n, mo, h, seed=lx)
    # an oblique plane through the box, image rectangle inside the box
    origin = np.array([-0.9, 0.6, 2.1])
    U = np.array([1.9, 0.3, 0.4])
    V = np.array([0.1, 1.3, 2.0])
    rgba, s, y = oslice.slice_rgba(u[None], lx, n, mo, h, origin, U, V, 23, 17, -3.0, 3.0,
                                   [[0, 0, 0, 1], [1, 1, 0, 0]])
    p = oslice.pixel_points(origin, U, V, 23, 17)
    assert np.all(np.isfinite(s))
    np.testing.assert_allclose(s, f(p[..., 0], p[..., 1], p[..., 2]), rtol=1e-11, atol=1e-11)


def test_slice_location_faces_and_outside():
    n, mo, h = (2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    pts = np.array([[1.0, 0.25, 0.25],    # shared face x = 1 belongs to the upper element, xi = -1
                    [2.0, 2.0, 2.0],      # top corner belongs to the last element, xi = +1
                    [0.0, 0.0, 0.0],      # lower corner, xi = -1
                    [-1e-12, 0.5, 0.5],   # just outside
                    [0.5, 2.0 + 1e-12, 0.5]])
    e, xi, inside = oslice.locate(pts, n, mo, h)
    assert list(inside) == [True, True, True, False, False]
    assert e[0] == 1 and xi[0, 0] == -1.0 and xi[0, 1] == -0.5
    assert e[1] == 7 and np.all(xi[1] == 1.0)
    assert e[2] == 0 and np.all(xi[2] == -1.0)


def test_slice_colour_table_and_background():
    ctrl = [[0.0, 0.2, 0.3, 0.8], [0.5, 0.902, 0.902, 0.902], [1.0, 0.7, 0.0, 0.1]]  # 255 c off the .5 ties
    s = np.array([-5.0, 0.0, 0.25, 0.5, 0.75, 1.0, 7.0])
    y = oslice.colour_channels(s, 0.0, 1.0, ctrl)
    c = np.asarray(ctrl)[:, 1:]
    np.testing.assert_allclose(y[0] / 255, c[0])            # clamped below
    np.testing.assert_allclose(y[1] / 255, c[0])
    np.testing.assert_allclose(y[2] / 255, (c[0] + c[1]) / 2)  # midpoint of segment 0
    np.testing.assert_allclose(y[3] / 255, c[1])            # at a control point
    np.testing.assert_allclose(y[4] / 255, (c[1] + c[2]) / 2)
    np.testing.assert_allclose(y[5] / 255, c[2])
    np.testing.assert_allclose(y[6] / 255, c[2])            # clamped above
    # a plane partly outside the mesh: background there, opaque inside
    u = np.ones((1, 8, 4, 4, 4))
    rgba, s2, _ = oslice.slice_rgba(u, 4, (2, 2, 2), (0, 0, 0), (1, 1, 1), (-1, 0.5, 0.5), (4, 0, 0),
                                    (0, 1, 0), 8, 2, 0.0, 2.0, ctrl, background=(1, 2, 3, 4))
    assert np.all(rgba[:, :2] == [1, 2, 3, 4]) and np.all(rgba[:, 6:] == [1, 2, 3, 4])
    assert np.all(rgba[:, 2:6, 3] == 255) and np.allclose(s2[:, 2:6], 1.0)
    assert np.all(rgba[:, 2:6, :3] == np.floor(255 * np.asarray(ctrl[1][1:]) + 0.5))


def test_slice_magnitude():
    lx, n, mo, h = 4, (2, 1, 1), (0, 0, 0), (1, 1, 1)
    rng = np.random.default_rng(3)
    u = rng.normal(size=(3, 2, lx, lx, lx))
    pts = np.array([[0.3, 0.2, 0.9], [1.7, 0.5, 0.1]])
    e, xi, inside = oslice.locate(pts, n, mo, h)
    v = oslice.interpolate(u, lx, e, xi)
    np.testing.assert_allclose(oslice.scalar(v), np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    # each component separately equals the one-component interpolation
    for c in range(3):
        np.testing.assert_array_equal(oslice.interpolate(u[c:c + 1], lx, e, xi)[0], v[c])
