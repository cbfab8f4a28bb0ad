"""Host-side checks of the C ABI: the library loads, exports every entry
point that include/semr.h declares, validates its arguments without touching
a GPU, sizes buffers like the payload format says, and its host decoder
rebuilds oracle payloads."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2407_20731_b300 as semr
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_declared_symbol_is_exported():
    text = open(os.path.join(ROOT, "include", "semr.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|uint32_t|const char\*)\s+(semr_\w+)\s*\(", text, re.M))
    assert declared, "no declarations parsed"
    for path in (semr.LIB_PATH, os.path.join(os.path.dirname(semr.LIB_PATH), "libsemr_bounds.so")):
        lib = ctypes.CDLL(path)
        for name in sorted(declared):
            assert hasattr(lib, name), (path, name)
    assert declared == {n for n, _, _ in semr.EXPORTS}


def test_build_flags_name_the_checking_build():
    """libsemr.so is the default build; libsemr_bounds.so (the same ABI) was
    compiled with -DSEMR_BOUNDS and says so."""
    here = os.path.dirname(semr.LIB_PATH)
    for name, flags in (("libsemr.so", 0), ("libsemr_bounds.so", semr.SEMR_BUILD_BOUNDS)):
        lib = ctypes.CDLL(os.path.join(here, name))
        lib.semr_build_flags.restype = ctypes.c_int
        assert lib.semr_build_flags() == flags, name


@pytest.mark.parametrize("lx,ne,nf,tau", [(8, 262144, 4, 1e-3), (6, 1001, 3, 0.0), (10, 7, 1, 1e-9), (2, 5, 16, 0.5)])
def test_sizes_match_payload_format(lx, ne, nf, tau):
    s = semr.semr_sizes_for(lx, ne, nf, tau)
    assert s.header_bytes == oracle.header_bytes(nf)
    assert s.code_base == oracle.header_bytes(nf) + nf * oracle.field_fixed_bytes(lx, ne)
    width = 8 if tau == 0 else (2 if tau * 32767.0 ** 2 > 4 else 4)
    assert s.code_width == width
    assert s.payload_worst == s.code_base + width * lx ** 3 * ne * nf


@pytest.mark.parametrize("lx,ne,nf", [(8, 262144, 4), (8, 1, 1), (8, 1000000, 16), (6, 1001, 3), (10, 7, 1)])
def test_scratch_sizes(lx, ne, nf):
    s = semr.semr_sizes_for(lx, ne, nf, 1e-3)
    assert 0 < s.scratch_min_bytes <= s.scratch_bytes
    if lx == 8:
        # the lx = 8 kernel keeps one float per element-field (its rounded max |u|)
        assert s.scratch_min_bytes > 4 * ne * nf
    # the no-allocation entry point's array: the 64^3 x 4 snapshot fits its minimum,
    # 16 million element-fields do not
    if (lx, ne, nf) == (8, 262144, 4):
        assert s.scratch_min_bytes <= semr.SEMR_NOALLOC_SCRATCH_BYTES
    if (lx, ne, nf) == (8, 1000000, 16):
        assert s.scratch_min_bytes > semr.SEMR_NOALLOC_SCRATCH_BYTES


def test_argument_validation_needs_no_gpu():
    fs, mesh, out = semr.semr_fieldset(), semr.semr_mesh(), semr.semr_outputs()
    assert semr.semr_reduce_async(fs, mesh, out, 0) == semr.SEMR_EINVAL  # zero sizes, null pointers
    mesh.lx, mesh.n_elem = 8, 10
    fs.n_fields, fs.tau = 1, 1e-3
    assert semr.semr_reduce_async(fs, mesh, out, 0) == semr.SEMR_EINVAL  # null device pointers
    fs.tau = -1.0
    assert semr.semr_reduce_async(fs, mesh, out, 0) == semr.SEMR_EINVAL
    fs.tau, fs.precision = 1e-3, 7
    mesh.jac = 16
    assert semr.semr_reduce_async(fs, mesh, out, 0) in (semr.SEMR_EINVAL, semr.SEMR_EUNSUPPORTED)
    mesh.lx = 13
    assert semr.semr_reduce_async(fs, mesh, out, 0) == semr.SEMR_EUNSUPPORTED
    # flags: unknown bits are rejected; the cumulative variant has no native-FP64 form
    mesh.lx, fs.precision = 8, semr.SEMR_FP64
    fs.flags = 4
    assert semr.semr_reduce_async(fs, mesh, out, 0) == semr.SEMR_EINVAL
    fs.flags, fs.precision = semr.SEMR_CUMULATIVE, semr.SEMR_FP64_NATIVE
    assert semr.semr_reduce_async(fs, mesh, out, 0) == semr.SEMR_EUNSUPPORTED
    fs.flags = 0
    with pytest.raises(semr.SemrError):
        semr.semr_sizes_for(1, 10, 1, 1e-3)
    with pytest.raises(semr.SemrError):
        semr.semr_sizes_for(8, 10, 17, 1e-3)
    with pytest.raises(semr.SemrError):
        semr.semr_sizes_for(8, 10, 1, float("inf"))
    assert "budget" in semr.semr_strerror(semr.SEMR_EBUDGET)


@pytest.mark.parametrize("lx", range(2, 13))
def test_library_gll_matches_oracle(lx):
    x, w = semr.semr_gll(lx)
    xo, wo = oracle.gll(lx)
    np.testing.assert_allclose(x, xo, rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, wo, rtol=2e-15, atol=0)


@pytest.mark.parametrize("lx,tau", [(8, 1e-3), (5, 1e-2), (6, 0.0), (10, 1e-9)])
def test_host_decoder_rebuilds_oracle_payload(lx, tau):
    f, j = synth.snapshot(45, lx, [3, 4])
    f = f.numpy().reshape(2, 45, -1)
    r = oracle.reduce(f, j.numpy(), tau)
    dec = semr.semr_decode(r.payload)
    assert np.abs(dec - r.recon).max() <= 1e-13 * np.abs(f).max()


def test_host_decoder_rejects_malformed():
    f, j = synth.snapshot(8, 6, [1])
    r = oracle.reduce(f.numpy().reshape(1, 8, -1), j.numpy(), 1e-3)
    bad = r.payload.copy()
    bad[0] = ord("X")
    with pytest.raises(semr.SemrError):
        semr.semr_decode(bad)
    with pytest.raises(semr.SemrError):
        semr.semr_decode(r.payload[:-2])  # truncated code section


def test_host_decoder_survives_corruption():
    """Seeded corruptions of a valid payload -- header fields set to extreme
    values (a code count whose size in bytes wraps around 2^64 among them),
    random bytes flipped anywhere, truncations -- make the decoder return an
    error or a finite-sized result; it never reads outside the buffer."""
    import struct
    f, j = synth.snapshot(20, 6, [5, 6])
    r = oracle.reduce(f.numpy().reshape(2, 20, -1), j.numpy(), 1e-3)
    good = r.payload
    cases = []
    for off, fmt, val in [(40, "<Q", 2 ** 63), (40, "<Q", 2 ** 62 + 1), (40, "<Q", 2 ** 64 - 1), (32, "<Q", 2 ** 63),
                          (32, "<Q", 0), (16, "<Q", 2 ** 39), (16, "<Q", 0), (12, "<I", 0), (6, "<H", 13),
                          (8, "<H", 17), (8, "<H", 0), (4, "<H", 7), (10, "<H", 0xffff)]:
        bad = bytearray(good)
        struct.pack_into(fmt, bad, off, val)
        cases.append(np.frombuffer(bytes(bad), dtype=np.uint8))
    rng = np.random.default_rng(11)
    for _ in range(300):
        bad = good.copy()
        for pos in rng.integers(0, bad.size, size=rng.integers(1, 6)):
            bad[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        cases.append(bad)
    for cut in (1, 2, 17, good.size // 2, good.size - 1):
        cases.append(good[:cut].copy())
    ok = 0
    for bad in cases:
        try:
            out = semr.semr_decode(bad)
            assert out.ndim == 3
            ok += 1
        except semr.SemrError:
            pass
    assert ok < len(cases)  # most corruptions are caught


def test_slice_argument_validation_needs_no_gpu():
    """Every case below is invalid, so the call returns before any CUDA work."""
    good_mesh = semr.make_lattice(8, (4, 4, 4))
    ok = dict(origin=(0, 0, 1), axis_u=(6, 0, 0), axis_v=(0, 6, 0), width=16, height=16, vmin=0.0, vmax=1.0,
              n_comp=1)
    fake = [256, 256, 256]

    def call(mesh=good_mesh, rgba=4096, fields=fake, **kw):
        a = dict(ok)
        a.update(kw)
        sl = semr.make_slice(a["origin"], a["axis_u"], a["axis_v"], a["width"], a["height"], a["vmin"], a["vmax"],
                             a["n_comp"], a.get("ctrl", semr.COOL_WARM))
        return semr.semr_slice_rgba(mesh, fields, sl, rgba, None, 0)

    assert call(rgba=0) == semr.SEMR_EINVAL
    assert call(mesh=semr.make_lattice(13, (4, 4, 4))) == semr.SEMR_EUNSUPPORTED
    assert call(mesh=semr.make_lattice(8, (0, 4, 4), h=(1.0, 1.0, 1.0))) == semr.SEMR_EINVAL
    assert call(mesh=semr.make_lattice(8, (4, 4, 4), h=(1.0, -1.0, 1.0))) == semr.SEMR_EINVAL
    assert call(width=0) == semr.SEMR_EINVAL
    assert call(height=semr.SEMR_SLICE_MAX_SIDE + 1) == semr.SEMR_EINVAL
    assert call(n_comp=4) == semr.SEMR_EINVAL
    assert call(vmax=0.0) == semr.SEMR_EINVAL
    assert call(vmin=float("nan")) == semr.SEMR_EINVAL
    assert call(origin=(0, float("inf"), 0)) == semr.SEMR_EINVAL
    assert call(ctrl=[(0.0, 0, 0, 0)]) == semr.SEMR_EINVAL                          # one control point
    assert call(ctrl=[(0.0, 0, 0, 0), (0.9, 1, 1, 1)]) == semr.SEMR_EINVAL          # does not end at 1
    assert call(ctrl=[(0.0, 0, 0, 0), (0.6, 1, 1, 1), (0.5, 1, 1, 1), (1, 0, 0, 0)]) == semr.SEMR_EINVAL
    assert call(ctrl=[(0.0, 0, 0, 0), (1.0, 1.5, 1, 1)]) == semr.SEMR_EINVAL         # channel above 1
    assert call(rgba=4098) == semr.SEMR_EINVAL                                       # unaligned output
    assert call(fields=[264, 256, 256]) == semr.SEMR_EINVAL                          # unaligned field (even lx)
    assert call(fields=[0, 0, 0]) == semr.SEMR_EINVAL
