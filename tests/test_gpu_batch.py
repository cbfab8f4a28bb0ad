"""The batched form: many uneven snapshots and orders in one launch sequence
(one persistent kernel per order over a shared work queue), captured in a
CUDA graph, with elements per CTA chosen by the autotuner.  Every snapshot's
result must be byte-identical to the single-snapshot entry point's (same
arithmetic, deterministic order), before and after graph capture, and agree
with the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, make_case

pytestmark = pytest.mark.gpu

SHAPES = [(257, 6, 2, 1e-3), (1200, 8, 3, 1e-2), (64, 10, 1, 1e-4), (3001, 8, 1, 1e-3), (500, 6, 4, 1e-5),
          (333, 10, 2, 1e-3), (1, 8, 1, 1e-3), (90, 5, 2, 1e-3)]


def _snapshots(precision):
    snaps = []
    for i, (ne, lx, nf, tau) in enumerate(SHAPES):
        f, j = make_case(ne, lx, nf, seed=60 + i, slope=-5.0 / 3.0 - 0.2 * i)
        snaps.append(([f[k] for k in range(nf)], j, lx, tau, precision, f))
    return snaps


def _single(fields, jac, lx, tau, prec):
    res = semr.reduce(fields, jac, lx, tau, precision=prec)
    return res.payload, res.summary


def _warp_level(sched, lx):
    """Whether every group of this order runs its warp-level kernel (tiles of 64 or 128 elements;
    the CTA kernels' tiles hold at most 32), as a single launch at lx = 6, 8 and 10 does."""
    return lx in (6, 8, 10) and all(g[2] >= 64 for g in sched if g[0] == lx)


def _same_reports(sm, ref, exact, precision):
    """Field reports of a batched snapshot against its single launch: bit for bit when both run the
    same kernel (the same per-element arithmetic, and both finalize the same tile partials in the
    same order); where the autotuner chose a CTA-kernel tile instead, the threads map to other
    points and the partial sums regroup, so the norms agree to rounding (FP64 mode) or to the FP32
    form's own arithmetic."""
    assert (sm.n_fields, sm.code_total, sm.recomputed, sm.cr) == (ref.n_fields, ref.code_total, ref.recomputed, ref.cr)
    for f in range(sm.n_fields):
        a, r = sm.field[f], ref.field[f]
        assert (a.kept, a.bytes, a.cr, a.umax) == (r.kept, r.bytes, r.cr, r.umax)
        for k in ("l2_abs", "l2_rel", "linf_abs", "linf_rel", "sum_err2", "sum_energy"):
            if exact:
                assert getattr(a, k) == getattr(r, k), (f, k)
            else:
                np.testing.assert_allclose(getattr(a, k), getattr(r, k),
                                           rtol=1e-12 if precision == semr.SEMR_FP64 else 1e-5)


@pytest.mark.parametrize("precision", [semr.SEMR_FP64, semr.SEMR_FP32])
def test_batch_matches_single_launches_and_graph_replay(precision):
    snaps = _snapshots(precision)
    b = semr.Batch([s[:5] for s in snaps], autotune=True)
    sched = b.schedule()
    assert sum(g[3] for g in sched) == len(snaps)
    for lx, pr, tile, n, tuned in sched:
        assert tile in tuned
        if len(tuned) > 1:  # timed variants: the chosen one is the fastest that ran
            ran = {t: ms for t, ms in tuned.items() if ms > 0}
            assert tile == min(ran, key=ran.get)
    b.launch()
    first = b.results()
    b.capture()
    for _ in range(2):
        b.replay()
        again = b.results()
        for (p1, _), (p2, _) in zip(first, again):
            assert np.array_equal(p1, p2)
    for (payload, sm), (fields, jac, lx, tau, prec, f) in zip(first, snaps):
        assert sm.status == 0
        ref_p, ref_s = _single(fields, jac, lx, tau, prec)
        assert np.array_equal(payload, ref_p)
        _same_reports(sm, ref_s, _warp_level(sched, lx), prec)
        if precision == semr.SEMR_FP64:
            o = oracle.reduce(f.cpu().numpy(), jac.cpu().numpy(), tau, want_recon=False, want_coeffs=False,
                              fragile_cap=100000)
            compare_payloads(payload, o.payload, o.fragile)
    b.close()


@pytest.mark.parametrize("precision", [semr.SEMR_FP64, semr.SEMR_FP32])
def test_batch_cumulative_truncation(precision):
    """Cumulative-energy truncation in a batch, next to threshold snapshots of the
    same orders (their own groups): each result byte-identical to its single
    launch, and in FP64 mode to the oracle's cumulative variant outside its
    fragile list; a cumulative snapshot of an order without a warp-level kernel
    is refused (single launches only)."""
    shapes = [(700, 6, 2, 1e-3, True), (1500, 8, 1, 1e-3, True), (300, 10, 2, 1e-4, True), (900, 8, 2, 1e-3, False),
              (400, 6, 1, 1e-2, False), (2500, 8, 1, 1e-5, True)]
    snaps = []
    for i, (ne, lx, nf, tau, cum) in enumerate(shapes):
        f, j = make_case(ne, lx, nf, seed=130 + i)
        snaps.append(([f[k] for k in range(nf)], j, lx, tau, precision, cum, f))
    b = semr.Batch([s[:6] for s in snaps], autotune=True)
    sched = b.schedule()
    assert len(sched) == 5  # (lx, truncation) groups: 6 cum, 8 cum, 10 cum, 8 thr, 6 thr
    b.capture()
    b.replay()
    for (payload, sm), (fields, jac, lx, tau, prec, cum, f) in zip(b.results(), snaps):
        assert sm.status == 0
        assert bool(oracle.parse_header(payload)["flags"] & semr.SEMR_PAYLOAD_CUMULATIVE) == cum
        ref = semr.reduce(fields, jac, lx, tau, precision=prec, cumulative=cum)
        assert np.array_equal(payload, ref.payload)
        _same_reports(sm, ref.summary, cum or _warp_level(sched, lx), prec)  # cumulative groups: warp-level only
        if precision == semr.SEMR_FP64:
            o = oracle.reduce(f.cpu().numpy(), jac.cpu().numpy(), tau, want_recon=False, want_coeffs=False,
                              fragile_cap=100000, cumulative=cum)
            compare_payloads(payload, o.payload, o.fragile)
    b.close()
    f, j = make_case(50, 7, 1, seed=140)
    with pytest.raises(semr.SemrError) as e:
        semr.Batch([([f[0]], j, 7, 1e-3, precision, True)])
    assert e.value.code == semr.SEMR_EUNSUPPORTED
