"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every case generates one seeded snapshot on the GPU, runs libsemr on it and
the oracle on a host copy of the same buffer, and compares payloads, masks,
codes, reconstructions and error reports element by element (see
tests/parity.py for the tolerances and their derivation).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, compare_reports, make_case, run_gpu

pytestmark = pytest.mark.gpu


def _full_compare(n_elem, lx, n_fields, tau, seed=1, slope=-5.0 / 3.0):
    fields, jac = make_case(n_elem, lx, n_fields, seed, slope)
    res, rec = run_gpu(fields, jac, lx, tau)
    assert res.summary.status == 0
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, tau, fragile_cap=100000)
    compare_payloads(res.payload, o.payload, o.fragile, lossless=(tau == 0.0))
    compare_reports(f_np, j_np, rec, o, res.elem_report, res.summary, lx)
    if tau > 0:
        # the library's host decoder rebuilds the GPU reconstruction
        dec = semr.semr_decode(res.payload)
        umax = np.abs(f_np).reshape(n_fields, -1).max(axis=1)
        assert np.all(np.abs(dec - rec).reshape(n_fields, -1).max(axis=1) <= 1e-12 * umax)
    return res, o


def test_small_case_bit_exact():
    """512 elements (8^3), lx = 8, one field, tau = 1e-3: identical payload bytes."""
    res, o = _full_compare(512, 8, 1, 1e-3)
    assert o.n_fragile == 0
    assert res.summary.payload_bytes == o.payload.size


@pytest.mark.parametrize("lx", [2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_every_lx_ragged(lx):
    """All supported orders, an element count that leaves a ragged last tile,
    two fields (the look-back crosses the field boundary)."""
    _full_compare(203, lx, 2, 1e-3, seed=lx)


@pytest.mark.parametrize("tau", [1e-1, 1e-2, 1e-4, 1e-6])
def test_thresholds_three_fields(tau):
    _full_compare(1001, 8, 3, tau, seed=7)


@pytest.mark.parametrize("lx", [6, 10])
def test_steep_spectrum(lx):
    _full_compare(777, lx, 2, 1e-3, seed=3, slope=-3.0)


def test_lossless_tau_zero():
    _full_compare(130, 8, 2, 0.0)


def test_int32_codes():
    res, o = _full_compare(64, 6, 1, 1e-9)
    assert oracle.parse_header(res.payload)["flags"] & semr.SEMR_PAYLOAD_CODE32


@pytest.mark.parametrize("n_elem,lx,n_fields,tau,seed", [(4096, 8, 3, 1e-6, 80), (3000, 6, 2, 1e-6, 84),
                                                          (5000, 8, 2, 1e-7, 87), (2500, 10, 2, 1e-6, 82)])
def test_small_tau_decisions_in_fp64(n_elem, lx, n_fields, tau, seed):
    """Small tau keeps coefficients down to ~1e-5 max|u| of their element,
    and the quantisation then decides codes |a|/q near half-integers to
    ~1e-8 relative: the exact recomputation must be FP64-accurate there (at
    seed 80, element 2551 of field 0 has |a|/q = 4.500000017 for mode 81,
    outside the 1e-9 fragile band; float pairs rounded it to 4)."""
    _full_compare(n_elem, lx, n_fields, tau, seed=seed)


def test_tau_above_one_keeps_nothing():
    res, o = _full_compare(100, 8, 1, 2.0)
    assert res.summary.code_total == 0


def test_single_element():
    _full_compare(1, 8, 1, 1e-3)


def test_many_tiles_lookback():
    """~10k tiles: the decoupled look-back chains across many CTAs.  Also the
    exact-recomputation path of FP64 mode: at this size some coefficients
    always fall within the FP32 error bound of a decision."""
    res, o = _full_compare(20000, 8, 2, 1e-3, seed=5)
    assert res.summary.recomputed > 0


def test_zero_and_constant_blocks():
    lx, E = 8, 40
    fields, jac = make_case(E, lx, 1)
    fields[0, :10] = 0.0
    fields[0, 10:20] = 3.25
    res, rec = run_gpu(fields, jac, lx, 1e-3)
    o = oracle.reduce(fields.cpu().numpy(), jac.cpu().numpy(), 1e-3)
    compare_payloads(res.payload, o.payload, o.fragile)
    compare_reports(fields.cpu().numpy(), jac.cpu().numpy(), rec, o, res.elem_report, res.summary, lx)
    s = oracle.sections(res.payload)
    assert np.all(s["counts"][0, :10] == 0) and np.all(s["steps"][0, :10] == -32768)


def test_deterministic_repeat():
    fields, jac = make_case(3000, 8, 2, seed=11)
    a, ra = run_gpu(fields, jac, 8, 1e-3)
    b, rb = run_gpu(fields, jac, 8, 1e-3)
    assert np.array_equal(a.payload, b.payload)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.elem_report, b.elem_report)


def test_payload_overflow_reported():
    lx, E = 8, 64
    fields, jac = make_case(E, lx, 1)
    sz = semr.semr_sizes_for(lx, E, 1, 1e-3)
    bufs = semr.alloc_buffers(lx, E, 1, 1e-3, payload_cap=int(sz.code_base))
    semr.reduce_async([fields[0]], jac, lx, 1e-3, bufs)
    torch.cuda.synchronize()
    sm = semr.summary_from(bufs)
    assert sm.status & semr.SEMR_STATUS_OVERFLOW


def test_nonfinite_input_flagged():
    lx, E = 6, 30
    fields, jac = make_case(E, lx, 1)
    fields[0, 4, 17] = float("nan")
    res, _ = run_gpu(fields, jac, lx, 1e-3)
    assert res.summary.status & semr.SEMR_STATUS_NONFINITE
    assert oracle.sections(res.payload)["counts"][0, 4] == 0


def _mixed(n_elem, n_fields, seed):
    """lx = 8 snapshot where every 7th element is white noise (hundreds of codes:
    more than a staging slot holds, and the dense inverse) among smooth ones."""
    fields, jac = make_case(n_elem, 8, n_fields, seed)
    g = torch.Generator().manual_seed(seed + 99)
    noisy = torch.arange(n_elem) % 7 == 3
    noise = torch.randn(n_fields, int(noisy.sum()), 512, dtype=torch.float64, generator=g)
    fields[:, noisy.cuda()] = noise.cuda()
    return fields.contiguous(), jac


def test_elements_with_many_codes_among_few():
    """Codes of elements that keep more than a staging slot go straight to
    their final place; the others are staged and copied per tile.  Both kinds
    interleave across ragged tiles and two fields: payload bytes identical."""
    fields, jac = _mixed(300, 2, seed=21)
    res, rec = run_gpu(fields, jac, 8, 1e-3)
    assert res.summary.status == 0
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, 1e-3, fragile_cap=100000)
    counts = oracle.sections(res.payload)["counts"]
    assert counts.max() > 100 and counts.min() < 10
    compare_payloads(res.payload, o.payload, o.fragile)
    compare_reports(f_np, j_np, rec, o, res.elem_report, res.summary, 8)


def test_fp32_form_many_codes_decode():
    """The FP32 form places every code: the payload decodes to its own
    reconstruction (up to FP32 rounding)."""
    fields, jac = _mixed(300, 2, seed=22)
    res, rec = run_gpu(fields, jac, 8, 1e-3, precision=semr.SEMR_FP32)
    assert res.summary.status == 0
    assert oracle.sections(res.payload)["counts"].max() > 100
    dec = semr.semr_decode(res.payload)
    umax = np.abs(fields.cpu().numpy()).reshape(2, -1).max(axis=1)
    assert np.all(np.abs(dec - rec).reshape(2, -1).max(axis=1) <= 1e-5 * umax)


def _kept_exactly(counts, n_fields, seed):
    """lx = 8 blocks with a chosen number of kept modes: k coefficients of size
    1..1.5 at random modes, the rest below 1e-7 (built through the oracle's
    inverse transform).  At tau = 1e-2 exactly the k large ones are kept while
    k <= 44 (the smallest share, 1 / (2.25 k), stays above tau)."""
    rng = np.random.default_rng(seed)
    E = len(counts)
    f = np.empty((n_fields, E, 512))
    for fi in range(n_fields):
        for e, k in enumerate(counts):
            a = rng.uniform(-1e-7, 1e-7, 512)
            m = rng.choice(512, k, replace=False)
            a[m] = rng.choice([-1.0, 1.0], k) * rng.uniform(1.0, 1.5, k)
            f[fi, e] = oracle.inverse(8, a).reshape(-1)
    j = rng.uniform(0.5, 2.0, E)
    return torch.from_numpy(f).cuda().contiguous(), torch.from_numpy(j).cuda().contiguous()


def test_sparse_and_dense_reconstruction_limits():
    """Elements that keep just below and just above each sparse-path limit of the
    lx = 8 kernel (10, 16 and 24 kept modes; past the limit the dense inverse
    runs): FP64 mode bit-exact with the oracle and its reconstruction within
    1e-12 max|u|; the FP32 form's counts as the oracle's and its codes within
    one unit of the FP64 ones."""
    counts = [1, 2, 9, 10, 11, 15, 16, 17, 23, 24, 25, 26, 40] * 19
    fields, jac = _kept_exactly(counts, 2, seed=77)
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, 1e-2, fragile_cap=100000)
    assert np.array_equal(oracle.sections(o.payload)["counts"][0], np.array(counts))
    res, rec = run_gpu(fields, jac, 8, 1e-2)
    assert res.summary.status == 0
    compare_payloads(res.payload, o.payload, o.fragile)
    compare_reports(f_np, j_np, rec, o, res.elem_report, res.summary, 8)
    r32, rec32 = run_gpu(fields, jac, 8, 1e-2, precision=semr.SEMR_FP32)
    g, s = oracle.sections(r32.payload), oracle.sections(o.payload)
    assert np.array_equal(g["counts"], s["counts"]) and np.array_equal(g["masks"], s["masks"])
    assert np.array_equal(g["steps"], s["steps"])
    assert np.abs(g["codes"].astype(np.int32) - s["codes"].astype(np.int32)).max() <= 1
    umax = np.abs(f_np).reshape(2, -1).max(axis=1)
    assert np.abs(rec32 - o.recon).reshape(2, -1).max(axis=1).max() <= 2e-5 * umax.max()


@pytest.mark.parametrize("precision", [semr.SEMR_FP64, semr.SEMR_FP32])
def test_lx8_nonfinite_and_out_of_range_flagged(precision):
    """lx = 8 (the warp-per-element kernel): a NaN, an infinity and a value of
    2^500 or more (whose element energy leaves the FP64 range) each flag
    SEMR_STATUS_NONFINITE, and their elements keep nothing.  Every other byte of the payload equals the
    payload of the same snapshot with those three blocks set to zero (a zero
    block also keeps nothing and stores the sentinel step)."""
    fields, jac = make_case(300, 8, 2, seed=13)
    zeroed = fields.clone()
    bad = [(0, 5, 17, float("nan")), (0, 130, 0, float("inf")), (1, 200, 511, 1e160)]
    for f, e, i, v in bad:
        fields[f, e, i] = v
        zeroed[f, e] = 0.0
    res, _ = run_gpu(fields, jac, 8, 1e-3, precision=precision)
    ref, _ = run_gpu(zeroed, jac, 8, 1e-3, precision=precision)
    assert res.summary.status & semr.SEMR_STATUS_NONFINITE
    assert ref.summary.status == 0
    counts = oracle.sections(res.payload)["counts"]
    assert all(counts[f, e] == 0 for f, e, _, _ in bad)
    assert res.payload.size == ref.payload.size and np.array_equal(res.payload, ref.payload)
