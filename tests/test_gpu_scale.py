"""Magnitude independence of the reduction (CUDA path through the C ABI).

The method's threshold is relative -- keep a mode iff a_m^2 >= tau S_e,
arXiv 2407.20731 Sec. IV-B's maximal allowed error read per element -- so
the result cannot depend on the units of a field.  Scaling every value by an
exact power of two 2^k scales each coefficient by 2^k and each energy by
2^2k with no rounding at all, so in exact arithmetic (and in the FP64 oracle,
barring under- or overflow) masks, counts and codes are unchanged and every
step moves by exactly k.  The library reads each element as u 2^-ke (ke the
binary exponent of its largest |u|), so its payloads must show the same
invariance bit for bit, in both precisions, for the warp kernel (lx = 8) and
the warp-group kernel (lx = 6, 10), and with either truncation (the
cumulative budget t = tau S_e scales by 2^2k like every energy).  Norms scale
by exactly 2^2k (e2_e, E_e) and 2^k (Linf_e).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, compare_reports, make_case, run_gpu

pytestmark = pytest.mark.gpu

SCALES = [-120, -80, -40, 40, 80]
NOSTEP = -32768


@pytest.mark.parametrize("cumulative", [False, True])
@pytest.mark.parametrize("precision", [semr.SEMR_FP64, semr.SEMR_FP32])
@pytest.mark.parametrize("lx", [6, 8, 10])
def test_power_of_two_scaling_invariance(lx, precision, cumulative):
    tau = 1e-3
    fields, jac = make_case(301, lx, 2, seed=20 + lx)
    base, _ = run_gpu(fields, jac, lx, tau, precision=precision, recon=False, cumulative=cumulative)
    assert base.summary.status == 0
    b = oracle.sections(base.payload)
    kept = b["steps"] != NOSTEP
    assert kept.all()
    j_np = jac.cpu().numpy()
    for k in SCALES:
        scaled = fields * (2.0 ** k)  # exact: no value under- or overflows
        res, _ = run_gpu(scaled, jac, lx, tau, precision=precision, recon=False, cumulative=cumulative)
        assert res.summary.status == 0, (k, res.summary.status)
        g = oracle.sections(res.payload)
        assert np.array_equal(g["masks"], b["masks"]), k
        assert np.array_equal(g["counts"], b["counts"]), k
        assert np.array_equal(g["codes"], b["codes"]), k
        assert np.array_equal(g["steps"].astype(np.int32), b["steps"].astype(np.int32) + k), k
        assert res.payload.size == base.payload.size
        er, eb = res.elem_report, base.elem_report
        assert np.array_equal(er[:, :, 0], eb[:, :, 0] * 2.0 ** (2 * k)), k
        assert np.array_equal(er[:, :, 1], eb[:, :, 1] * 2.0 ** (2 * k)), k
        assert np.array_equal(er[:, :, 2], eb[:, :, 2] * 2.0 ** k), k
        for f in range(2):
            assert res.summary.field[f].umax == base.summary.field[f].umax * 2.0 ** k
        if precision == semr.SEMR_FP64:
            # FP64 mode against the oracle on the scaled snapshot itself
            f_np = scaled.cpu().numpy()
            o = oracle.reduce(f_np, j_np, tau, fragile_cap=100000, cumulative=cumulative)
            compare_payloads(res.payload, o.payload, o.fragile)


@pytest.mark.parametrize("lx", [6, 8, 10])
def test_small_and_large_magnitude_blocks_match_oracle(lx):
    """A unit-scale field in which some elements hold values around 1e-16 (a
    quiescent region: their energies are ~1e-32, below float range once
    squared) and others around 1e100: FP64 mode equals the oracle outside its
    fragile list, element by element, with the usual reconstruction and norm
    tolerances (relative to each element's own magnitude class)."""
    tau = 1e-3
    fields, jac = make_case(260, lx, 1, seed=40 + lx)
    fields[0, 30:90] *= 1e-16
    fields[0, 150:170] *= 1e100
    res, rec = run_gpu(fields, jac, lx, tau)
    assert res.summary.status == 0
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, tau, fragile_cap=100000)
    differ = compare_payloads(res.payload, o.payload, o.fragile)
    assert differ == 0
    # the tiny elements keep codes (they were dropped when the energy underflowed)
    s = oracle.sections(res.payload)
    assert (s["counts"][0, 30:90] > 0).all()
    # reports: each magnitude class against its own scale
    for sl in (slice(0, 30), slice(30, 90), slice(150, 170)):
        um = np.abs(f_np[0, sl]).max()
        assert np.abs(rec[0, sl] - o.recon[0, sl]).max() <= 1e-12 * um
        np.testing.assert_allclose(res.elem_report[0, sl, 1], o.elem_report[0, sl, 1], rtol=1e-12, atol=0)
        assert np.abs(res.elem_report[0, sl, 2] - o.elem_report[0, sl, 2]).max() <= 1e-12 * um


@pytest.mark.parametrize("lx", [6, 8])
@pytest.mark.parametrize("precision", [semr.SEMR_FP64, semr.SEMR_FP32])
def test_subnormal_elements_are_zero_blocks(lx, precision):
    """Elements whose values are all subnormal doubles (|u| < 2^-1022) keep
    nothing, as in FP64 (t = tau S_e underflows), report zero norms and set the
    informational SEMR_STATUS_TINY bit; the rest of the payload is unchanged."""
    fields, jac = make_case(200, lx, 1, seed=60 + lx)
    zeroed = fields.clone()
    zeroed[0, 10:14] = 0.0
    fields[0, 10:14] *= 2.0 ** -1030
    res, _ = run_gpu(fields, jac, lx, 1e-3, precision=precision, recon=False)
    ref, _ = run_gpu(zeroed, jac, lx, 1e-3, precision=precision, recon=False)
    assert res.summary.status == semr.SEMR_STATUS_TINY
    assert ref.summary.status == 0
    assert np.array_equal(res.payload, ref.payload)
    assert np.all(res.elem_report[0, 10:14, :2] == 0.0)
