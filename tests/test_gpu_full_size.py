"""Parity at the benchmark's full size: 64^3 = 262,144 elements, lx = 8, the
four fields u, v, w, p (seeds 10..13), tau = 1e-3, in the launch
configuration bench.py times (alloc_buffers with the recommended scratch,
reduce_async, no reconstruction written).

The oracle cannot reduce a million element-fields in seconds, but each
element-field's mask, step, codes and element report depend only on its own
block, J_e and tau (Sec. IV-B: the compression works element by element).  So
sampled element-fields are compared one by one with an oracle run on just
those blocks, and properties that hold at any size cover every element-field:
the counts are the masks' popcounts, the codes sit where the counts' prefix
places them (the payload's code order), every kept code is a nonzero integer
with |c| <= 2/sqrt(tau) (the quantisation's range), and the field report is
the sum and maximum of the element reports.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2407_20731_b300 as semr
import synth

pytestmark = pytest.mark.gpu

LX, N_SIDE, TAU = 8, 64, 1e-3
E = N_SIDE ** 3
F = 4
N3 = LX ** 3


@pytest.fixture(scope="module")
def snapshot():
    f, j = synth.full_case(device="cuda")
    fields = f.reshape(F, E, N3).contiguous()
    yield fields, j.contiguous()
    del fields
    torch.cuda.empty_cache()


def _run(fields, jac, precision, cumulative=False):
    bufs = semr.alloc_buffers(LX, E, F, TAU, fields.device)
    semr.reduce_async([fields[i] for i in range(F)], jac, LX, TAU, bufs, precision, cumulative=cumulative)
    torch.cuda.synchronize()
    sm = semr.summary_from(bufs)
    n = int(sm.payload_bytes)
    payload = bufs.payload[:n].cpu().numpy()
    er = bufs.elem_report.view(F, E, 3).cpu().numpy()
    return sm, payload, er


def _sections(payload):
    """Masks as bytes [F, E, 64], steps, counts and the code array."""
    h = oracle.parse_header(payload)
    assert (h["lx"], h["n_fields"], h["n_elem"]) == (LX, F, E)
    fixed = oracle.field_fixed_bytes(LX, E)
    pad = lambda v: (v + 15) & ~15  # noqa: E731
    masks = np.empty((F, E, 64), np.uint8)
    steps = np.empty((F, E), np.int16)
    counts = np.empty((F, E), np.uint16)
    for f in range(F):
        base = h["header_bytes"] + f * fixed
        masks[f] = payload[base:base + 64 * E].reshape(E, 64)
        sb = base + pad(64 * E)
        steps[f] = payload[sb:sb + 2 * E].view("<i2")
        cb = sb + pad(2 * E)
        counts[f] = payload[cb:cb + 2 * E].view("<u2")
    codes = payload[h["code_base"]:h["code_base"] + 2 * h["code_total"]].view("<i2")
    return h, masks, steps, counts, codes


def _sample(seed=7, n=1500):
    """Element indices: seeded random ones plus tile and array boundaries."""
    rng = np.random.default_rng(seed)
    edges = [0, 1, 31, 32, 127, 128, 129, 255, 256, E // 2, E - 129, E - 128, E - 2, E - 1]
    return np.unique(np.concatenate([rng.choice(E, n, replace=False), edges]))


def _check_any_size(sm, payload, er, fields, cumulative=False):
    h, masks, steps, counts, codes = _sections(payload)
    assert sm.status == 0
    # counts are the masks' popcounts; the code section holds exactly their sum
    pc = np.bitwise_count(masks).sum(axis=2, dtype=np.int64)
    assert np.array_equal(pc, counts.astype(np.int64))
    total = int(counts.astype(np.int64).sum())
    assert h["code_total"] == total == sm.code_total
    assert sm.payload_bytes == h["code_base"] + 2 * total == payload.size
    # every kept code is an integer within the quantisation's range, and nonzero under threshold
    # truncation (a kept a^2 >= t >= q^2); the cumulative budget can keep modes below half a step
    assert codes.size == total
    if not cumulative:
        assert np.all(codes != 0)
    assert np.abs(codes.astype(np.int32)).max() <= 2.0 / math.sqrt(TAU)
    # per field: kept codes, sums and maxima of the element reports
    umax = fields.reshape(F, -1).abs().amax(dim=1).cpu().numpy()
    for f in range(F):
        fr = sm.field[f]
        assert fr.kept == int(counts[f].astype(np.int64).sum())
        assert fr.umax == umax[f]
        assert fr.linf_abs == er[f, :, 2].max()
        np.testing.assert_allclose(fr.sum_energy, er[f, :, 1].sum(), rtol=1e-12)
        np.testing.assert_allclose(fr.sum_err2, er[f, :, 0].sum(), rtol=1e-12)
        np.testing.assert_allclose(fr.l2_rel, math.sqrt(fr.sum_err2 / fr.sum_energy), rtol=1e-14)
        assert fr.cr == 1.0 - (oracle.field_fixed_bytes(LX, E) + 2 * fr.kept) / (8.0 * N3 * E)
    return masks, steps, counts, codes


def _oracle_sample(fields, jac, idx, cumulative=False):
    f_np = fields[:, torch.as_tensor(idx, device=fields.device)].cpu().numpy()
    j_np = jac[torch.as_tensor(idx, device=jac.device)].cpu().numpy()
    o = oracle.reduce(f_np, j_np, TAU, want_recon=False, want_coeffs=False, fragile_cap=100000,
                      cumulative=cumulative)
    return f_np, j_np, o


def _per_element(idx, masks, steps, counts, codes, osec):
    """Yield (f, k, same_mask_step_count, gpu_codes, oracle_codes) for sampled (f, idx[k])."""
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64).reshape(-1))])
    o_offs = np.concatenate([[0], np.cumsum(osec["counts"].astype(np.int64).reshape(-1))])
    om = np.packbits(osec["masks"], axis=2, bitorder="little")
    S = idx.size
    for f in range(F):
        for k, e in enumerate(idx):
            same = (np.array_equal(masks[f, e], om[f, k]) and steps[f, e] == osec["steps"][f, k]
                    and counts[f, e] == osec["counts"][f, k])
            i, j = f * E + e, f * S + k
            yield f, k, same, codes[offs[i]:offs[i + 1]], osec["codes"][o_offs[j]:o_offs[j + 1]]


@pytest.mark.parametrize("cumulative", [False, True])
def test_full_size_fp64_mode(snapshot, cumulative):
    """FP64 mode (the benchmark's), with threshold truncation and with the
    cumulative-energy variant (the bench's cumulative leg): sampled
    element-fields bit-exact outside the oracle's fragile entries; their
    reports within the parity tolerances."""
    fields, jac = snapshot
    sm, payload, er = _run(fields, jac, semr.SEMR_FP64, cumulative)
    assert bool(oracle.parse_header(payload)["flags"] & semr.SEMR_PAYLOAD_CUMULATIVE) == cumulative
    masks, steps, counts, codes = _check_any_size(sm, payload, er, fields, cumulative)
    idx = _sample()
    f_np, j_np, o = _oracle_sample(fields, jac, idx, cumulative)
    osec = oracle.sections(o.payload)
    fragile = {(int(f), int(k)) for f, k, _, _ in o.fragile}
    for f, k, same, gc, oc in _per_element(idx, masks, steps, counts, codes, osec):
        if not (same and np.array_equal(gc, oc)):
            assert (f, k) in fragile, f"element-field ({f}, {idx[k]}) differs outside the fragile list"
    # element reports of the sample (as in the small-size parity tests)
    umax = fields.reshape(F, -1).abs().amax(dim=1).cpu().numpy()
    d = (1e-12 * umax)[:, None]
    ge, oe = er[:, idx], o.elem_report
    J = j_np[None, :]
    bound = 2 * d * np.sqrt(8 * J * oe[:, :, 0]) + 8 * J * d * d + 1e-12 * oe[:, :, 0]
    assert np.all(np.abs(ge[:, :, 0] - oe[:, :, 0]) <= bound)
    np.testing.assert_allclose(ge[:, :, 1], oe[:, :, 1], rtol=1e-12, atol=0)
    assert np.all(np.abs(ge[:, :, 2] - oe[:, :, 2]) <= d)


def test_full_size_fp32_form(snapshot):
    """FP32 precision form: the any-size properties hold exactly; sampled
    decisions agree with the FP64 oracle for at least 99% of element-fields
    (the precision-form bar), and matching ones carry identical codes."""
    fields, jac = snapshot
    sm, payload, er = _run(fields, jac, semr.SEMR_FP32)
    assert oracle.parse_header(payload)["flags"] & semr.SEMR_PAYLOAD_FP32
    masks, steps, counts, codes = _check_any_size(sm, payload, er, fields)
    idx = _sample(seed=8)
    _, _, o = _oracle_sample(fields, jac, idx)
    osec = oracle.sections(o.payload)
    agree = [same and np.array_equal(gc, oc) for _, _, same, gc, oc in
             _per_element(idx, masks, steps, counts, codes, osec)]
    assert np.mean(agree) >= 0.99, np.mean(agree)
