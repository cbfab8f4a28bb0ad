"""Python binding of the plain FP64 CPU oracle (``semr_oracle.c``).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package's
``smoke()`` check and the CPU-baseline leg of ``bench.py`` import this module.
It shares no code with the CUDA path (``paper_2407_20731_b300``) and never
imports it.

The oracle follows the lossy compression of SEM fields that arXiv 2407.20731
runs in situ (Sec. IV-B): a per-element transform to a Legendre basis, energy-
relative truncation and quantisation, reconstruction and error norms.  The C
source states every step and every reading of the paper it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "semr_oracle.c")
_LIB = os.path.join(_HERE, "libsemr_oracle.so")

OK, EINVAL, ENOSPACE = 0, 1, 2
FLAG_LOSSLESS, FLAG_CODE32, FLAG_CUMULATIVE = 1, 2, 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-Wextra", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        P = ctypes.c_void_p
        _lib.oracle_legendre.restype = d
        _lib.oracle_legendre.argtypes = [i, d]
        _lib.oracle_gll.restype = i
        _lib.oracle_gll.argtypes = [i, P, P]
        _lib.oracle_tables.restype = i
        _lib.oracle_tables.argtypes = [i, P, P]
        _lib.oracle_forward.restype = None
        _lib.oracle_forward.argtypes = [i, P, P, P]
        _lib.oracle_inverse.restype = None
        _lib.oracle_inverse.argtypes = [i, P, P, P]
        _lib.oracle_header_bytes.restype = i64
        _lib.oracle_header_bytes.argtypes = [i]
        _lib.oracle_field_fixed_bytes.restype = i64
        _lib.oracle_field_fixed_bytes.argtypes = [i, i64]
        _lib.oracle_reduce.restype = i
        _lib.oracle_reduce.argtypes = [i, i64, i, P, P, d, P, i64, P, P, P, P, P, P, i64, P, i, i]
        _lib.oracle_decode.restype = i
        _lib.oracle_decode.argtypes = [P, i64, P, i64]
        _lib.oracle_max_threads.restype = i
        _lib.oracle_max_threads.argtypes = []
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def legendre(k: int, x: float) -> float:
    """P_k(x) by the Bonnet recurrence."""
    return lib().oracle_legendre(k, float(x))


def gll(lx: int) -> tuple[np.ndarray, np.ndarray]:
    """GLL nodes (ascending) and weights of the lx-point rule."""
    x = np.zeros(lx)
    w = np.zeros(lx)
    rc = lib().oracle_gll(lx, _ptr(x), _ptr(w))
    if rc != OK:
        raise ValueError(f"oracle_gll({lx}) -> {rc}")
    return x, w


def tables(lx: int) -> tuple[np.ndarray, np.ndarray]:
    """(Phi, A): Phi[i, k] = phi_k(x_i) and A[k, i] = phi_k(x_i) w_i."""
    phi = np.zeros((lx, lx))
    amat = np.zeros((lx, lx))
    rc = lib().oracle_tables(lx, _ptr(phi), _ptr(amat))
    if rc != OK:
        raise ValueError(f"oracle_tables({lx}) -> {rc}")
    return phi, amat


def forward(lx: int, u: np.ndarray) -> np.ndarray:
    """Modal coefficients a[r, q, p] of one element block u[k, j, i]."""
    _, amat = tables(lx)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(lx, lx, lx)
    a = np.zeros_like(u)
    lib().oracle_forward(lx, _ptr(amat), _ptr(u), _ptr(a))
    return a


def inverse(lx: int, a: np.ndarray) -> np.ndarray:
    """Nodal values u[k, j, i] of one element's modal coefficients a[r, q, p]."""
    phi, _ = tables(lx)
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(lx, lx, lx)
    u = np.zeros_like(a)
    lib().oracle_inverse(lx, _ptr(phi), _ptr(a), _ptr(u))
    return u


def header_bytes(n_fields: int) -> int:
    return int(lib().oracle_header_bytes(n_fields))


def field_fixed_bytes(lx: int, n_elem: int) -> int:
    return int(lib().oracle_field_fixed_bytes(lx, n_elem))


@dataclass
class Result:
    """Everything oracle_reduce returns for one snapshot."""
    payload: np.ndarray        # uint8 [bytes]
    elem_report: np.ndarray    # [F, E, 3] = (e2_e, E_e, Linf_e)
    field_report: np.ndarray   # [F, 8] = (L2_abs, L2_rel, Linf_abs, Linf_rel, sum e2, sum E, max|u|, kept)
    recon: np.ndarray | None   # [F, E, lx^3]
    coeffs: np.ndarray | None  # [F, E, lx^3]
    fragile: np.ndarray        # [n, 4] = (field, element, mode or -1, kind)
    n_fragile: int


def reduce(fields: np.ndarray, jac: np.ndarray, tau: float, *, want_recon: bool = True,
           want_coeffs: bool = True, fragile_cap: int = 4096, n_threads: int = 0, cumulative: bool = False) -> Result:
    """Run the whole reduction of one snapshot.

    ``fields`` is [F, E, lx^3] (or [F, E, lx, lx, lx]) FP64, ``jac`` is [E].
    ``cumulative`` selects the cumulative-energy truncation variant.
    """
    fields = np.ascontiguousarray(fields, dtype=np.float64)
    F, E = fields.shape[0], fields.shape[1]
    n = int(np.prod(fields.shape[2:]))
    lx = int(round(n ** (1.0 / 3.0)))
    if lx ** 3 != n:
        raise ValueError("element blocks must hold lx^3 values")
    jac = np.ascontiguousarray(jac, dtype=np.float64)
    if jac.shape != (E,):
        raise ValueError("jac must have one entry per element")
    L = lib()
    elem = np.zeros((F, E, 3))
    frep = np.zeros((F, 8))
    recon = np.zeros((F, E, n)) if want_recon else None
    coeffs = np.zeros((F, E, n)) if want_coeffs else None
    fragile = np.zeros((max(fragile_cap, 1), 4), dtype=np.int64)
    nbytes = ctypes.c_int64(0)
    nfr = ctypes.c_int64(0)
    # First call sizes the payload (ENOSPACE with cap 0), second call fills it.
    args = [lx, E, F, _ptr(fields), _ptr(jac), float(tau)]
    trunc = 1 if cumulative else 0
    rc = L.oracle_reduce(*args, None, 0, ctypes.byref(nbytes), None, None, None, None,
                         None, 0, ctypes.byref(nfr), n_threads, trunc)
    if rc not in (OK, ENOSPACE):
        raise ValueError(f"oracle_reduce -> {rc}")
    payload = np.zeros(nbytes.value, dtype=np.uint8)
    rc = L.oracle_reduce(*args, _ptr(payload), payload.size, ctypes.byref(nbytes), _ptr(elem),
                         _ptr(frep), _ptr(recon), _ptr(coeffs), _ptr(fragile), fragile_cap,
                         ctypes.byref(nfr), n_threads, trunc)
    if rc != OK:
        raise ValueError(f"oracle_reduce -> {rc}")
    k = min(nfr.value, fragile_cap)
    return Result(payload, elem, frep, recon, coeffs, fragile[:k].copy(), nfr.value)


def decode(payload: np.ndarray) -> np.ndarray:
    """Rebuild [F, E, lx^3] fields from a payload with the oracle's own loops."""
    payload = np.ascontiguousarray(payload, dtype=np.uint8)
    hdr = parse_header(payload)
    n = hdr["lx"] ** 3
    out = np.zeros((hdr["n_fields"], hdr["n_elem"], n))
    rc = lib().oracle_decode(_ptr(payload), payload.size, _ptr(out), out.size)
    if rc != OK:
        raise ValueError(f"oracle_decode -> {rc}")
    return out


def parse_header(payload: np.ndarray) -> dict:
    """Header fields and section views of a payload (oracle's own parser)."""
    b = payload.tobytes() if isinstance(payload, np.ndarray) else bytes(payload)
    if b[:4] != b"SEMR":
        raise ValueError("bad magic")
    version, lx, nf, flags = np.frombuffer(b, dtype="<u2", count=4, offset=4)
    hdr_bytes = int(np.frombuffer(b, dtype="<u4", count=1, offset=12)[0])
    n_elem = int(np.frombuffer(b, dtype="<u8", count=1, offset=16)[0])
    tau = float(np.frombuffer(b, dtype="<f8", count=1, offset=24)[0])
    code_base, code_total = (int(v) for v in np.frombuffer(b, dtype="<u8", count=2, offset=32))
    counts = np.frombuffer(b, dtype="<u8", count=int(nf), offset=48).astype(np.int64)
    return dict(version=int(version), lx=int(lx), n_fields=int(nf), flags=int(flags),
                header_bytes=hdr_bytes, n_elem=n_elem, tau=tau, code_base=code_base,
                code_total=code_total, code_count=counts)


def sections(payload: np.ndarray) -> dict:
    """Split a payload into per-field masks [F, E, lx^3] (bool), steps [F, E],
    counts [F, E] and the per-element code lists (oracle's own parser)."""
    payload = np.ascontiguousarray(payload, dtype=np.uint8)
    h = parse_header(payload)
    lx, F, E = h["lx"], h["n_fields"], h["n_elem"]
    n = lx ** 3
    mb = (n + 7) // 8
    pad = lambda v: (v + 15) & ~15  # noqa: E731
    fixed = field_fixed_bytes(lx, E)
    masks = np.zeros((F, E, n), dtype=bool)
    steps = np.zeros((F, E), dtype=np.int16)
    counts = np.zeros((F, E), dtype=np.uint16)
    for f in range(F):
        base = h["header_bytes"] + f * fixed
        mbytes = payload[base:base + E * mb].reshape(E, mb)
        bits = np.unpackbits(mbytes, axis=1, bitorder="little")[:, :n]
        masks[f] = bits.astype(bool)
        sb = base + pad(E * mb)
        steps[f] = payload[sb:sb + 2 * E].view("<i2")
        cb = sb + pad(2 * E)
        counts[f] = payload[cb:cb + 2 * E].view("<u2")
    lossless = bool(h["flags"] & FLAG_LOSSLESS)
    width = 8 if lossless else (4 if h["flags"] & FLAG_CODE32 else 2)
    dt = "<f8" if lossless else ("<i4" if width == 4 else "<i2")
    codes = payload[h["code_base"]:h["code_base"] + width * h["code_total"]].view(dt)
    return dict(header=h, masks=masks, steps=steps, counts=counts, codes=codes, width=width)


def max_threads() -> int:
    return int(lib().oracle_max_threads())
