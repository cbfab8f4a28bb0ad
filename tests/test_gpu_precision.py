"""The precision form (FP32 transforms) and the native-FP64 reference path,
checked against the FP64 oracle.

FP32 form: its decisions and reconstruction are not required to equal the
FP64 oracle's; the test checks what FP32 arithmetic guarantees.  Each 1-D
folded contraction rounds at most 5 times, the tables and the input carry
one more rounding each, and the discrete orthonormality gives row sums
sum_i |A_pi| <= sqrt(2) and |Phi| rows bounded by 1/sqrt(w_min), so for
element-fields whose decisions match the oracle's, |u~_fp32 - u~_oracle| is
well below 2e-5 max|u_f| (that bound is what the test asserts).  Decisions
may flip only for coefficients whose FP64 value lies within the FP32 error of
a threshold or rounding boundary: a small fraction of element-fields.  The
field error norms then agree with the oracle's to a relative 1e-3.
"""
import numpy as np
import pytest

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, compare_reports, make_case, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lx,n_elem,nf,tau", [(8, 4000, 4, 1e-3), (8, 2000, 2, 1e-5), (6, 1500, 2, 1e-3),
                                              (10, 700, 1, 1e-4), (5, 900, 1, 1e-2)])
def test_fp32_form_against_fp64_oracle(lx, n_elem, nf, tau):
    fields, jac = make_case(n_elem, lx, nf, seed=41)
    res, rec = run_gpu(fields, jac, lx, tau, precision=semr.SEMR_FP32)
    assert res.summary.status == 0
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, tau, fragile_cap=0)
    g, s = oracle.sections(res.payload), oracle.sections(o.payload)
    assert g["header"]["flags"] & semr.SEMR_PAYLOAD_FP32
    same = (np.all(g["masks"] == s["masks"], axis=2) & (g["steps"] == s["steps"]) & (g["counts"] == s["counts"]))
    # codes of matching elements
    go = np.concatenate([[0], np.cumsum(g["counts"].astype(np.int64).reshape(-1))])
    oo = np.concatenate([[0], np.cumsum(s["counts"].astype(np.int64).reshape(-1))])
    flat = same.reshape(-1)
    for i in np.nonzero(flat)[0]:
        if not np.array_equal(g["codes"][go[i]:go[i + 1]], s["codes"][oo[i]:oo[i + 1]]):
            flat[i] = False
    same = flat.reshape(same.shape)
    frac_diff = 1.0 - same.mean()
    assert frac_diff <= 0.01, frac_diff
    umax = np.abs(f_np).reshape(nf, -1).max(axis=1)
    for fi in range(nf):
        d = np.abs(rec[fi] - o.recon[fi])[same[fi]]
        assert d.size == 0 or d.max() <= 2e-5 * umax[fi], (d.max(), umax[fi])
        fr, orr = res.summary.field[fi], o.field_report[fi]
        assert abs(fr.l2_rel - orr[1]) <= 1e-3 * orr[1] + 1e-7
        assert abs(fr.linf_abs - orr[2]) <= 1e-3 * orr[2] + 2e-5 * umax[fi]


@pytest.mark.parametrize("lx", [3, 6, 8, 10])
def test_native_fp64_reference_path(lx):
    fields, jac = make_case(257, lx, 2, seed=43)
    tau = 1e-3
    res, rec = run_gpu(fields, jac, lx, tau, precision=semr.SEMR_FP64_NATIVE)
    assert res.summary.status == 0
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, tau, fragile_cap=100000)
    compare_payloads(res.payload, o.payload, o.fragile)
    compare_reports(f_np, j_np, rec, o, res.elem_report, res.summary, lx)


def test_fp64_pair_and_native_agree_bitwise_on_payload():
    fields, jac = make_case(3000, 8, 2, seed=47)
    a, ra = run_gpu(fields, jac, 8, 1e-4, precision=semr.SEMR_FP64)
    b, rb = run_gpu(fields, jac, 8, 1e-4, precision=semr.SEMR_FP64_NATIVE)
    o = oracle.reduce(fields.cpu().numpy(), jac.cpu().numpy(), 1e-4, want_recon=False, want_coeffs=False)
    if o.n_fragile == 0:
        assert np.array_equal(a.payload, b.payload)
    assert np.abs(ra - rb).max() <= 1e-12 * np.abs(fields.cpu().numpy()).max()
