"""Helpers shared by the parity tests: run the CUDA path and the oracle on
the same seeded snapshot and compare them element by element.

Acceptance (arXiv 2407.20731 gives no numbers for this; these follow from the
method's definition and FP64 rounding):
  * masks, step exponents, counts and codes: identical, except at the
    oracle's fragile entries (decisions within 1e-9 relative of a tie); with
    no fragile entry the payload bytes are identical;
  * reconstruction: |u~_gpu - u~_oracle| <= 1e-12 max|u_f| per field (FP64);
  * element energies E_e: relative 1e-12; Linf_e: absolute 1e-12 max|u_f|;
    e2_e: within the bound that the reconstruction tolerance delta implies,
    2 delta sqrt(8 J_e e2_e) + 8 J_e delta^2 (sum of the GLL weight products
    is 8), plus relative 1e-12.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2407_20731_b300 as semr
import synth

RECON_TOL = 1e-12


def make_case(n_elem, lx, n_fields, seed=1, slope=-5.0 / 3.0, device="cuda"):
    f, j = synth.snapshot(n_elem, lx, [seed + 10 * i for i in range(n_fields)], slope=slope, device=device)
    return f.reshape(n_fields, n_elem, lx ** 3).contiguous(), j.contiguous()


def run_gpu(fields, jac, lx, tau, precision=semr.SEMR_FP64, recon=True, cumulative=False):
    F, E = fields.shape[0], fields.shape[1]
    rec = [torch.empty_like(fields[i]) for i in range(F)] if recon else None
    res = semr.reduce([fields[i] for i in range(F)], jac, lx, tau, precision=precision, recon=rec,
                      cumulative=cumulative)
    torch.cuda.synchronize()
    rec_np = torch.stack(rec).cpu().numpy() if recon else None
    return res, rec_np


def per_element_codes(sec):
    """Split the code stream into per-(field, element) arrays."""
    counts = sec["counts"].astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(counts.reshape(-1))])
    return counts, offs


def compare_payloads(gp: np.ndarray, op: np.ndarray, fragile: np.ndarray, lossless=False, rtol_lossless=1e-13,
                     max_fragile_share=1e-3):
    """Element-by-element payload comparison with the fragile exemptions.
    Returns the number of element-fields that differ (all at fragile spots).

    The exemptions themselves are bounded: decisions within 1e-9 relative of
    a tie are rare on smooth or noisy data (a few per million element-fields),
    so more than max_fragile_share of the element-fields listed (at least 2)
    means an over-eager fragile list, which would hide kernel errors."""
    gs, os_ = oracle.sections(gp), oracle.sections(op)
    hg, ho = gs["header"], os_["header"]
    for k in ("version", "lx", "n_fields", "flags", "header_bytes", "n_elem", "tau", "code_base"):
        assert hg[k] == ho[k], (k, hg[k], ho[k])
    fr_elem = {(int(f), int(e)) for f, e, m, k in fragile}
    gc, go = per_element_codes(gs)
    oc, oo = per_element_codes(os_)
    F, E = gs["counts"].shape
    assert len(fr_elem) <= max(2, max_fragile_share * F * E), (
        f"{len(fr_elem)} of {F * E} element-fields on the fragile list")
    differ = 0
    for f in range(F):
        for e in range(E):
            i = f * E + e
            same = (np.array_equal(gs["masks"][f, e], os_["masks"][f, e]) and gs["steps"][f, e] == os_["steps"][f, e]
                    and gs["counts"][f, e] == os_["counts"][f, e])
            if same:
                a = gs["codes"][go[i]:go[i + 1]]
                b = os_["codes"][oo[i]:oo[i + 1]]
                if lossless:
                    scale = max(np.abs(b).max(initial=0.0), 1e-300)
                    same = np.all(np.abs(a - b) <= rtol_lossless * scale)
                else:
                    same = np.array_equal(a, b)
            if not same:
                assert (f, e) in fr_elem, (
                    f"element-field ({f},{e}) differs outside the fragile list: "
                    f"steps {gs['steps'][f, e]}/{os_['steps'][f, e]} counts {gs['counts'][f, e]}/{os_['counts'][f, e]} "
                    f"mask diff at {np.nonzero(gs['masks'][f, e] != os_['masks'][f, e])[0][:8]} "
                    f"codes {gs['codes'][go[i]:go[i + 1]][:8]} / {os_['codes'][oo[i]:oo[i + 1]][:8]}")
                differ += 1
    assert differ <= len(fr_elem)
    if len(fragile) == 0 and not lossless:
        assert gp.size == op.size
        bad = np.nonzero(gp != op)[0]
        assert bad.size == 0, f"payload bytes differ with no fragile entry at {bad[:16]} (sizes {gp.size})"
    return differ


def compare_reports(fields_np, jac_np, g_recon, o: "oracle.Result", g_elem, g_summary, lx):
    F = fields_np.shape[0]
    umax = np.abs(fields_np).reshape(F, -1).max(axis=1)
    delta = RECON_TOL * umax
    if g_recon is not None:
        err = np.abs(g_recon - o.recon).reshape(F, -1).max(axis=1)
        assert np.all(err <= delta), (err, delta)
    ge, oe = g_elem, o.elem_report
    J = jac_np[None, :]
    d = delta[:, None]
    bound = 2 * d * np.sqrt(8 * J * oe[:, :, 0]) + 8 * J * d * d + 1e-12 * oe[:, :, 0]
    assert np.all(np.abs(ge[:, :, 0] - oe[:, :, 0]) <= bound)
    np.testing.assert_allclose(ge[:, :, 1], oe[:, :, 1], rtol=1e-12, atol=0)
    assert np.all(np.abs(ge[:, :, 2] - oe[:, :, 2]) <= d)
    for f in range(F):
        fr = g_summary.field[f]
        orr = o.field_report[f]
        assert fr.umax == orr[6]
        assert abs(fr.linf_abs - orr[2]) <= delta[f]
        np.testing.assert_allclose(fr.sum_energy, orr[5], rtol=1e-12)
        se2 = orr[4]
        tol = 2 * delta[f] * np.sqrt(8 * jac_np.sum() * se2) + 8 * jac_np.sum() * delta[f] ** 2 + 1e-12 * se2
        assert abs(fr.sum_err2 - se2) <= tol
