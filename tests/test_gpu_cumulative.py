"""Cumulative-energy truncation (SEMR_CUMULATIVE) on the GPU against the
FP64 oracle's cumulative variant.

The variant reads Sec. IV-B's maximal allowed error as a budget on the
discarded energy: sort an element's mode energies, drop the longest prefix
whose sum stays <= tau S_e, keep every mode at least as energetic as the
first one not dropped.  FP64 mode must reproduce the oracle's payload bit for
bit outside its fragile list (kind 4 covers the boundary sums and near-ties
within 1e-9 t); the FP32 precision form must keep a set that satisfies the
budget for the FP64 coefficients up to the FP32 coefficient error.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, compare_reports, make_case, run_gpu

pytestmark = pytest.mark.gpu


def _compare(fields, jac, lx, tau):
    res, rec = run_gpu(fields, jac, lx, tau, cumulative=True)
    assert res.summary.status == 0
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, tau, fragile_cap=100000, cumulative=True)
    compare_payloads(res.payload, o.payload, o.fragile, lossless=(tau == 0.0))
    compare_reports(f_np, j_np, rec, o, res.elem_report, res.summary, lx)
    if tau > 0:
        assert oracle.parse_header(res.payload)["flags"] & semr.SEMR_PAYLOAD_CUMULATIVE
        dec = semr.semr_decode(res.payload)
        umax = np.abs(f_np).reshape(fields.shape[0], -1).max(axis=1)
        assert np.all(np.abs(dec - rec).reshape(fields.shape[0], -1).max(axis=1) <= 1e-12 * umax)
    return res, o


def _white(n_elem, lx, n_fields, seed):
    """Seeded white noise: flat spectra, so an element's energies crowd a few
    octaves and the boundary octave holds many keys (the bisection path)."""
    g = torch.Generator().manual_seed(seed)
    f = torch.randn(n_fields, n_elem, lx ** 3, dtype=torch.float64, generator=g)
    j = 0.5 + 1.5 * torch.rand(n_elem, dtype=torch.float64, generator=g)
    return f.cuda().contiguous(), j.cuda().contiguous()


def test_small_case_bit_exact():
    fields, jac = make_case(512, 8, 1, seed=1)
    res, o = _compare(fields, jac, 8, 1e-3)
    assert o.n_fragile == 0
    assert res.summary.code_total > 0


@pytest.mark.parametrize("lx", [2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_every_lx_ragged(lx):
    fields, jac = make_case(203, lx, 2, seed=60 + lx)
    _compare(fields, jac, lx, 1e-3)


@pytest.mark.parametrize("tau", [1e-1, 1e-2, 1e-4, 1e-6])
def test_thresholds_three_fields(tau):
    fields, jac = make_case(1001, 8, 3, seed=71)
    _compare(fields, jac, 8, tau)


@pytest.mark.parametrize("lx,tau", [(8, 0.3), (8, 1e-2), (12, 0.1), (5, 0.2), (6, 0.3), (10, 1e-2)])
def test_flat_spectra_bisection(lx, tau):
    fields, jac = _white(150, lx, 1, seed=80 + lx)
    res, _ = _compare(fields, jac, lx, tau)
    if lx in (6, 8, 10):
        # the warp-level kernels: white noise keeps many modes, so most elements take the general
        # path, which recomputes an element's lx^3 coefficients once (a few single roundings come on
        # top from the elements the fast path settles)
        n = res.summary.recomputed
        assert 0 < n <= 150 * lx ** 3 + 150 and n // lx ** 3 >= 50, n


def test_many_tiles():
    """40,000 element-fields at lx = 8: the warp kernel settles most boundaries
    from its FP32 coefficients and sends the rest (boundary sums within the
    coefficients' error bound of t, about one element in a hundred) to the
    general path, which recomputes the element in FP64 (512 coefficients,
    counted in the summary's recomputed)."""
    fields, jac = make_case(20000, 8, 2, seed=5)
    res, _ = _compare(fields, jac, 8, 1e-3)
    assert res.summary.recomputed >= 512


@pytest.mark.parametrize("lx,n_elem,tau", [(6, 6000, 1e-3), (10, 2500, 1e-4)])
def test_many_tiles_warp_group(lx, n_elem, tau):
    """The warp-group kernel (lx = 6: one warp per element, lx = 10: two) over
    many look-back tiles: boundaries settled from the FP32 coefficients, the
    rest through the general path, bit-exact with the oracle outside kind 4."""
    fields, jac = make_case(n_elem, lx, 2, seed=40 + lx)
    _compare(fields, jac, lx, tau)


def test_keeps_more_than_threshold_form():
    """The budget form drops a subset of what the per-coefficient threshold
    drops: every mode with a^2 >= t is kept by both, and the budget keeps
    more in total."""
    fields, jac = make_case(3000, 8, 1, seed=9)
    thr, _ = run_gpu(fields, jac, 8, 1e-3, recon=False)
    cum, _ = run_gpu(fields, jac, 8, 1e-3, recon=False, cumulative=True)
    mt, mc = oracle.sections(thr.payload)["masks"], oracle.sections(cum.payload)["masks"]
    assert not np.any(mt & ~mc)
    assert cum.summary.code_total > thr.summary.code_total
    assert cum.summary.field[0].l2_rel <= thr.summary.field[0].l2_rel


@pytest.mark.parametrize("lx", [6, 8, 10, 7])
def test_edge_cases(lx):
    """Zero and constant blocks, tau >= 1, lossless tau = 0 and a single element,
    on each kernel that runs the variant (warp-group, warp, CTA)."""
    fields, jac = make_case(40, lx, 1)
    fields[0, :10] = 0.0
    fields[0, 10:20] = 3.25
    _compare(fields, jac, lx, 1e-3)
    # tau >= 1: the whole energy fits the budget, nothing is kept
    res, _ = _compare(fields, jac, lx, 1.5)
    assert res.summary.code_total == 0
    # tau = 0 stays lossless: no cumulative flag, every mode kept
    res, _ = run_gpu(fields, jac, lx, 0.0, cumulative=True)
    h = oracle.parse_header(res.payload)
    assert h["flags"] & semr.SEMR_PAYLOAD_LOSSLESS and not h["flags"] & semr.SEMR_PAYLOAD_CUMULATIVE
    # a single element
    f1, j1 = make_case(1, lx, 1, seed=3)
    _compare(f1, j1, lx, 1e-2)


@pytest.mark.parametrize("lx", [6, 8, 10])
def test_deterministic_repeat(lx):
    fields, jac = _white(500, lx, 2, seed=90)
    a, ra = run_gpu(fields, jac, lx, 0.05, cumulative=True)
    b, rb = run_gpu(fields, jac, lx, 0.05, cumulative=True)
    assert np.array_equal(a.payload, b.payload) and np.array_equal(ra, rb)


def test_native_path_rejects_cumulative():
    fields, jac = make_case(10, 6, 1)
    with pytest.raises(RuntimeError, match="unsupported"):
        semr.reduce([fields[0]], jac, 6, 1e-3, precision=semr.SEMR_FP64_NATIVE, cumulative=True)


@pytest.mark.parametrize("lx,tau,white", [(8, 1e-3, False), (8, 1e-5, False), (6, 1e-2, False), (8, 0.05, True),
                                          (10, 1e-3, False), (6, 0.05, True)])
def test_fp32_form_budget(lx, tau, white):
    """FP32 precision form: with the oracle's FP64 coefficients a, the modes the
    GPU dropped fit the budget and the smallest kept one does not, up to the
    FP32 coefficient error delta <= 1e-5 max|u_e| (the forward transform's
    rounding bound with a wide margin)."""
    # white noise keeps hundreds of modes per element: the general (bisection) path
    fields, jac = _white(300, lx, 2, seed=34) if white else make_case(2000, lx, 2, seed=33)
    res, rec = run_gpu(fields, jac, lx, tau, precision=semr.SEMR_FP32, cumulative=True)
    assert res.summary.status == 0
    f_np = fields.cpu().numpy()
    o = oracle.reduce(f_np, jac.cpu().numpy(), tau, fragile_cap=0, cumulative=True)
    g, s = oracle.sections(res.payload), oracle.sections(o.payload)
    assert g["header"]["flags"] & semr.SEMR_PAYLOAD_CUMULATIVE and g["header"]["flags"] & semr.SEMR_PAYLOAD_FP32
    a = o.coeffs
    en = a * a
    t = tau * en.sum(axis=2)
    delta = 1e-5 * np.abs(f_np).max(axis=2)
    n = lx ** 3
    mask = g["masks"]
    dropped = np.where(mask, 0.0, en).sum(axis=2)
    err = 2 * delta * np.where(mask, 0.0, np.abs(a)).sum(axis=2) + n * delta ** 2
    assert np.all(dropped <= t + err)
    kept_min = np.where(mask, en, np.inf).min(axis=2)
    has = mask.any(axis=2)
    err_k = err + 2 * delta * np.sqrt(np.where(has, kept_min, 0.0)) + delta ** 2
    assert np.all(~has | (dropped + kept_min > t - err_k))
    same = np.all(mask == s["masks"], axis=2).mean()
    assert same >= (0.5 if white else 0.9), same
    for fi in range(f_np.shape[0]):
        fr, orr = res.summary.field[fi], o.field_report[fi]
        assert abs(fr.l2_rel - orr[1]) <= 2e-2 * orr[1] + 1e-7
