"""The checking build (libsemr_bounds.so, compiled with -DSEMR_BOUNDS) on small
cases of every kernel, with canary words after every output buffer.

compute-sanitizer stands in for nothing here; instead every kernel of the
checking build tests the index or byte range of each global access against
its buffer before making it, skips any that falls outside and raises
SEMR_STATUS_BOUNDS (the slice kernels, which have no status word, record it
for semr_bounds_status).  Each output buffer -- payload, element report,
summary, scratch, reconstruction, slice image and values -- is allocated
with 4 KiB of canary bytes after its end.

A child process loads the checking build (SEMR_BOUNDS=1) and runs the cases:
the warp kernel (lx = 8, FP64 mode and FP32 form, threshold and cumulative
truncation, the cumulative cases large enough to reach its general path), the
warp-group kernel (lx = 6 and 10, both truncations), the CTA kernel (lx = 5
and 7, cumulative truncation, lossless), the hardware-FP64 kernel, a payload
too small for the codes, a batched launch over lx 6, 8 and 10, the
no-allocation entry point, and both slice kernels.  For each it asserts SEMR_STATUS_BOUNDS clear and the canaries
intact; the parent runs the same cases on the default build and requires the
same bytes from both.  A self-test of the checking build (a launch told a
payload capacity short of its fixed sections, inside buffers of the full size)
must report SEMR_STATUS_BOUNDS: the tests do fire.
"""
import ctypes
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for _p in (ROOT, HERE):
    if _p not in sys.path:
        sys.path.insert(0, _p)

CANARY = 4096
PATTERN = 0xA5


def _buf(nbytes):
    """Device bytes with CANARY pattern bytes after the first nbytes (the whole
    buffer starts filled with the pattern)."""
    t = torch.empty(int(nbytes) + CANARY, dtype=torch.uint8, device="cuda")
    t.fill_(PATTERN)
    return t


def _intact(t, nbytes):
    return bool((t[int(nbytes):] == PATTERN).all().item())


def _digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:20]


def _outputs(semr, lx, E, F, tau, payload_cap=None):
    sz = semr.semr_sizes_for(lx, E, F, tau)
    cap = int(sz.payload_worst if payload_cap is None else payload_cap)
    bufs = {"payload": (_buf(cap), cap),
            "elem": (_buf(24 * F * E), 24 * F * E),
            "summary": (_buf(ctypes.sizeof(semr.semr_summary)), ctypes.sizeof(semr.semr_summary)),
            "scratch": (_buf(int(sz.scratch_bytes)), int(sz.scratch_bytes))}
    o = semr.semr_outputs()
    o.payload = bufs["payload"][0].data_ptr()
    o.payload_cap = cap
    o.elem_report = bufs["elem"][0].data_ptr()
    o.summary = bufs["summary"][0].data_ptr()
    o.scratch = bufs["scratch"][0].data_ptr()  # torch blocks are 512-byte aligned
    o.scratch_bytes = int(sz.scratch_bytes)
    return bufs, o


def _summary(semr, bufs):
    raw = bufs["summary"][0][: ctypes.sizeof(semr.semr_summary)].cpu().numpy().tobytes()
    return semr.semr_summary.from_buffer_copy(raw)


def _finish(semr, bufs, recon=None, F=1, E=1):
    torch.cuda.synchronize()
    sm = _summary(semr, bufs)
    canaries = all(_intact(t, n) for t, n in bufs.values())
    if recon is not None:
        canaries = canaries and all(_intact(r, 8 * E * r_n) for r, r_n in recon)
    payload = bufs["payload"][0][: min(int(sm.payload_bytes), bufs["payload"][1])].cpu().numpy()
    elem = bufs["elem"][0][: 24 * F * E].cpu().numpy()
    parts = [payload, elem]
    if recon is not None:
        parts += [r[: 8 * E * n].cpu().numpy() for r, n in recon]
    return {"status": int(sm.status), "canaries": canaries, "digest": _digest(*parts),
            "codes": int(sm.code_total)}


def _reduce_case(semr, lx, E, F, tau, precision, recon=False, cumulative=False, payload_cap=None, seed=1):
    from parity import make_case
    f, j = make_case(E, lx, F, seed=seed)
    bufs, o = _outputs(semr, lx, E, F, tau, payload_cap)
    rec = [(_buf(8 * E * lx ** 3), lx ** 3) for _ in range(F)] if recon else None
    fs = semr.make_fieldset([f[i] for i in range(F)], tau, precision, cumulative=cumulative)
    if recon:
        fs.flags |= semr.SEMR_WRITE_RECON
        for i in range(F):
            fs.recon[i] = rec[i][0].data_ptr()
    rc = semr.semr_reduce_async(fs, semr.make_mesh(lx, j), o, torch.cuda.current_stream().cuda_stream)
    assert rc == semr.SEMR_OK, rc
    return _finish(semr, bufs, rec, F, E)


def _batch_case(semr):
    from parity import make_case
    specs = [(6, 700, 2, 1e-3, semr.SEMR_FP64, 11, False), (8, 900, 1, 1e-3, semr.SEMR_FP64, 12, False),
             (10, 300, 2, 1e-4, semr.SEMR_FP64, 13, False), (8, 500, 2, 1e-3, semr.SEMR_FP32, 14, False),
             (8, 600, 1, 1e-4, semr.SEMR_FP64, 15, True), (10, 200, 1, 1e-3, semr.SEMR_FP32, 16, True)]
    items = (semr.semr_batch_item * len(specs))()
    keep = []
    for i, (lx, E, F, tau, prec, seed, cum) in enumerate(specs):
        f, j = make_case(E, lx, F, seed=seed)
        bufs, o = _outputs(semr, lx, E, F, tau)
        items[i].fs = semr.make_fieldset([f[k] for k in range(F)], tau, prec, cumulative=cum)
        items[i].mesh = semr.make_mesh(lx, j)
        items[i].out = o
        keep.append((f, j, bufs, F, E))
    h = ctypes.c_void_p()
    st = torch.cuda.current_stream().cuda_stream
    assert semr._lib.semr_batch_create(ctypes.byref(h), items, len(specs), 0, st) == semr.SEMR_OK
    try:
        assert semr._lib.semr_batch_launch(h.value, st) == semr.SEMR_OK
        out = [_finish(semr, bufs, None, F, E) for (_, _, bufs, F, E) in keep]
    finally:
        semr._lib.semr_batch_destroy(h.value)
    return {"status": max(r["status"] for r in out), "canaries": all(r["canaries"] for r in out),
            "digest": _digest(np.array([r["digest"] for r in out])), "codes": sum(r["codes"] for r in out)}


def _noalloc_case(semr):
    from parity import make_case
    lx, E, F, tau = 8, 600, 2, 1e-3
    f, j = make_case(E, lx, F, seed=21)
    bufs, o = _outputs(semr, lx, E, F, tau)
    del bufs["scratch"]  # the entry point's scratch is the library's own array
    fs = semr.make_fieldset([f[i] for i in range(F)], tau, semr.SEMR_FP64)
    rc = semr.semr_reduce_async_noalloc(fs, semr.make_mesh(lx, j), o.payload, o.payload_cap, o.elem_report,
                                        o.summary, torch.cuda.current_stream().cuda_stream)
    assert rc == semr.SEMR_OK, rc
    return _finish(semr, bufs, None, F, E)


def _slice_case(semr, generic):
    import synth
    lx, n = 7, (6, 5, 4)
    E = n[0] * n[1] * n[2]
    f, _ = synth.snapshot(E, lx, [31, 32], device="cuda")
    f = f.reshape(2, -1).contiguous()
    W, H = 97, 61
    two_pi = 2.0 * np.pi
    if generic:  # a tilted plane that leaves the lattice: the generic kernel and the fill
        sl = semr.make_slice((-0.5, -0.3, 1.1), (7.0, 0.0, 1.3), (0.4, 7.2, 0.9), W, H, 0.0, 2.0, 2)
    else:        # an axis-aligned plane through the middle of an element layer
        sl = semr.make_slice((0.0, 0.0, 2.9), (two_pi, 0.0, 0.0), (0.0, two_pi, 0.0), W, H, 0.0, 2.0, 2)
    mesh = semr.make_lattice(lx, n)
    rgba, vals = _buf(4 * W * H), _buf(4 * W * H)
    semr.semr_bounds_status(True)
    rc = semr.semr_slice_rgba(mesh, [f[0].data_ptr(), f[1].data_ptr()], sl, rgba.data_ptr(), vals.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == semr.SEMR_OK, rc
    torch.cuda.synchronize()
    return {"status": int(semr.semr_bounds_status(True)), "canaries": _intact(rgba, 4 * W * H) and
            _intact(vals, 4 * W * H), "digest": _digest(rgba[: 4 * W * H].cpu().numpy(),
                                                        vals[: 4 * W * H].cpu().numpy()), "codes": 0}


def run_cases(semr):
    torch.cuda.set_device(0)
    P64, P32 = semr.SEMR_FP64, semr.SEMR_FP32
    cases = {
        "warp_lx8_fp64": lambda: _reduce_case(semr, 8, 700, 2, 1e-3, P64, recon=True, seed=1),
        "warp_lx8_fp32": lambda: _reduce_case(semr, 8, 700, 1, 1e-3, P32, recon=True, seed=2),
        "group_lx6_fp64": lambda: _reduce_case(semr, 6, 333, 2, 1e-3, P64, recon=True, seed=3),
        "group_lx10_fp32": lambda: _reduce_case(semr, 10, 129, 1, 1e-3, P32, recon=True, seed=4),
        "group_lx10_fp64": lambda: _reduce_case(semr, 10, 200, 2, 1e-4, P64, recon=True, seed=5),
        "cta_lx7_fp64": lambda: _reduce_case(semr, 7, 100, 1, 1e-3, P64, recon=True, seed=6),
        "cta_lx5_fp32": lambda: _reduce_case(semr, 5, 90, 2, 1e-4, P32, seed=7),
        "warp_lx8_cumulative_fp64": lambda: _reduce_case(semr, 8, 3000, 1, 1e-4, P64, cumulative=True, recon=True, seed=8),
        "warp_lx8_cumulative_fp32": lambda: _reduce_case(semr, 8, 300, 2, 1e-3, P32, cumulative=True, seed=18),
        "group_lx6_cumulative": lambda: _reduce_case(semr, 6, 2000, 1, 1e-4, P64, cumulative=True, recon=True, seed=19),
        "group_lx10_cumulative": lambda: _reduce_case(semr, 10, 600, 2, 1e-4, P64, cumulative=True, seed=20),
        "cta_lx7_cumulative": lambda: _reduce_case(semr, 7, 200, 1, 1e-3, P64, cumulative=True, seed=22),
        "cta_lx8_lossless": lambda: _reduce_case(semr, 8, 50, 1, 0.0, P64, recon=True, seed=9),
        "native_lx8_fp64": lambda: _reduce_case(semr, 8, 200, 1, 1e-3, semr.SEMR_FP64_NATIVE, seed=10),
        "warp_lx8_overflow": lambda: _reduce_case(
            semr, 8, 400, 1, 1e-3, P64, seed=11,
            payload_cap=int(semr.semr_sizes_for(8, 400, 1, 1e-3).code_base) + 64),
        "batched_lx6_8_10": lambda: _batch_case(semr),
        "noalloc_lx8": lambda: _noalloc_case(semr),
        "slice_axis": lambda: _slice_case(semr, False),
        "slice_generic": lambda: _slice_case(semr, True),
    }
    return {name: fn() for name, fn in cases.items()}


def _child():
    import paper_2407_20731_b300 as semr
    assert semr.BOUNDS_BUILD and semr.semr_build_flags() == semr.SEMR_BUILD_BOUNDS
    res = run_cases(semr)
    # the range tests fire: a launch told a payload capacity short of its fixed sections
    res["selftest"] = semr.semr_selftest_bounds()
    print("RESULT " + json.dumps(res))


@pytest.mark.gpu
def test_bounds_build_every_kernel_clean_and_identical():
    import paper_2407_20731_b300 as semr
    assert semr.semr_build_flags() == 0  # the default build
    env = dict(os.environ, SEMR_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--child"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    checked = json.loads(line[len("RESULT "):])
    rc, st = checked.pop("selftest")
    assert rc == semr.SEMR_OK and st & semr.SEMR_STATUS_BOUNDS, (rc, st)
    assert semr.semr_selftest_bounds()[0] == semr.SEMR_EUNSUPPORTED  # the default build has no tests
    plain = run_cases(semr)
    assert set(checked) == set(plain)
    for name, res in checked.items():
        assert not (res["status"] & semr.SEMR_STATUS_BOUNDS), (name, res)
        assert res["canaries"], (name, "a canary after an output buffer was overwritten")
        assert plain[name]["canaries"], (name, "default build")
        assert res["digest"] == plain[name]["digest"], (name, "the two builds' outputs differ")
        assert res["status"] == plain[name]["status"], name
    # the case with a too-small payload reports the overflow and writes nothing past it
    assert checked["warp_lx8_overflow"]["status"] & semr.SEMR_STATUS_OVERFLOW
    for name in checked:
        if name != "warp_lx8_overflow" and not name.startswith("slice"):
            assert checked[name]["status"] & ~semr.SEMR_STATUS_TINY == 0, (name, checked[name])


if __name__ == "__main__" and "--child" in sys.argv:
    _child()
