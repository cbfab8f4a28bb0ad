"""Plain FP64 CPU oracle of the in-situ slice image.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package's
``smoke()`` check and the CPU-baseline leg of ``bench.py`` use this module.
It shares no code with the CUDA path and never imports it.

arXiv 2407.20731 (Sec. IV-A) renders, in situ, images of a slice through the
Taylor-Green-vortex fields: its ParaView/Catalyst pipeline fixes the camera,
the image size and the slice position.  What such a slice image computes is
written out here from its definition:

1. Pixel centres.  The image spans the rectangle origin + a U + b V, a, b in
   [0, 1]; pixel (column c, row r) of a W x H image sits at
       p = (origin + ((c + 0.5) / W) U) + ((r + 0.5) / H) V
   (evaluated in that order, each operation rounded once, no fused
   multiply-add).  Row 0 is the row nearest ``origin`` along V.
2. Element and reference coordinates.  The mesh is an (nx, ny, nz) lattice of
   axis-aligned affine hexahedra with lower corner mo and edge lengths h,
   element e = ex + nx (ey + ny ez).  Per axis: q = (p - mo) / h,
   e_a = floor(q) (q == n exactly belongs to the last element), reference
   coordinate xi = 2 (q - e_a) - 1.  A point with some e_a outside [0, n_a)
   lies outside the mesh and gets the background colour.
3. Value.  The spectral-element field is the tensor-product Lagrange
   interpolant through the element's lx^3 GLL nodal values:
       s = sum_{k,j,i} l_k(zeta) l_j(eta) l_i(xi) u[e][k][j][i],
       l_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m).
   With several components the colour shows the magnitude sqrt(sum s_c^2).
4. Colour.  t = clamp((s - vmin) / (vmax - vmin), 0, 1); the control points
   (t_k, r_k, g_k, b_k) with t_0 = 0 < t_1 < ... = 1 define each channel by
   linear interpolation on the segment [t_k, t_{k+1}] that holds t (the last
   one when t = 1); byte = floor(255 c + 0.5); alpha 255.

Pinned in tests/test_oracle_pins.py against closed forms: partition of
unity and the Kronecker property of the basis, exact reproduction of
polynomials of degree <= lx - 1 per axis, face and corner ownership, the
colour table at and between control points, and the vector magnitude.
"""
from __future__ import annotations

import numpy as np

from . import gll


def lagrange(nodes: np.ndarray, x) -> np.ndarray:
    """l_i(x) for every node i: the product definition, shape x.shape + (lx,)."""
    x = np.asarray(x, dtype=np.float64)
    lx = len(nodes)
    out = np.ones(x.shape + (lx,))
    for i in range(lx):
        for m in range(lx):
            if m != i:
                out[..., i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return out


def pixel_points(origin, U, V, width: int, height: int) -> np.ndarray:
    """[H, W, 3] pixel centres, step 1 above."""
    o, U, V = (np.asarray(v, dtype=np.float64) for v in (origin, U, V))
    fc = (np.arange(width) + 0.5) / width
    fr = (np.arange(height) + 0.5) / height
    a = o[None, :] + fc[:, None] * U[None, :]                 # [W, 3]
    return a[None, :, :] + fr[:, None, None] * V[None, None, :]  # [H, W, 3]


def locate(p: np.ndarray, lattice, mesh_origin, h):
    """(element index [...], reference coordinates [..., 3], inside [...]), step 2."""
    n = np.asarray(lattice, dtype=np.int64)
    q = (p - np.asarray(mesh_origin, dtype=np.float64)) / np.asarray(h, dtype=np.float64)
    ea = np.floor(q)
    ea = np.where((ea == n) & (q == n), n - 1, ea)
    inside = np.all((ea >= 0) & (ea < n), axis=-1)
    xi = 2.0 * (q - ea) - 1.0
    eai = np.where(inside[..., None], ea, 0).astype(np.int64)
    e = eai[..., 0] + n[0] * (eai[..., 1] + n[1] * eai[..., 2])
    return e, xi, inside


def interpolate(fields: np.ndarray, lx: int, e: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Step 3 for every point: [n_comp, ...] values (any value where not inside)."""
    nodes, _ = gll(lx)
    fields = np.asarray(fields, dtype=np.float64)
    C = fields.shape[0]
    blocks = fields.reshape(C, -1, lx, lx, lx)
    shp = e.shape
    ef = e.reshape(-1)
    L = [lagrange(nodes, xi.reshape(-1, 3)[:, a]) for a in range(3)]  # x, y, z
    out = np.empty((C, ef.size))
    for c in range(C):
        # u[e][k][j][i] l_k(zeta) l_j(eta) l_i(xi)
        out[c] = np.einsum("pkji,pk,pj,pi->p", blocks[c][ef], L[2], L[1], L[0])
    return out.reshape((C,) + shp)


def scalar(values: np.ndarray) -> np.ndarray:
    """The scalar that is coloured: the value, or the magnitude of several."""
    return values[0] if values.shape[0] == 1 else np.sqrt(np.sum(values * values, axis=0))


def colour_channels(s: np.ndarray, vmin: float, vmax: float, ctrl) -> np.ndarray:
    """Step 4 before rounding: [..., 3] channel values 255 c in [0, 255]."""
    ctrl = np.asarray(ctrl, dtype=np.float64)
    t = np.clip((s - vmin) / (vmax - vmin), 0.0, 1.0)
    k = np.clip(np.searchsorted(ctrl[:, 0], t, side="right") - 1, 0, len(ctrl) - 2)
    t0, t1 = ctrl[k, 0], ctrl[k + 1, 0]
    f = (t - t0) / (t1 - t0)
    c = ctrl[k, 1:4] + f[..., None] * (ctrl[k + 1, 1:4] - ctrl[k, 1:4])
    return 255.0 * c


def slice_rgba(fields, lx: int, lattice, mesh_origin, h, origin, U, V, width: int, height: int,
               vmin: float, vmax: float, ctrl, background=(0, 0, 0, 0)):
    """(rgba [H, W, 4] uint8, scalar [H, W] (NaN outside), channels [H, W, 3]
    before rounding (NaN outside)) of the whole image."""
    p = pixel_points(origin, U, V, width, height)
    e, xi, inside = locate(p, lattice, mesh_origin, h)
    s = np.full((height, width), np.nan)
    if inside.any():
        vals = interpolate(fields, lx, e[inside], xi[inside])
        s[inside] = scalar(vals)
    y = np.full((height, width, 3), np.nan)
    y[inside] = colour_channels(s[inside], vmin, vmax, ctrl)
    rgba = np.empty((height, width, 4), dtype=np.uint8)
    rgba[...] = np.asarray(background, dtype=np.uint8)
    rgba[inside, :3] = np.clip(np.floor(y[inside] + 0.5), 0, 255).astype(np.uint8)
    rgba[inside, 3] = 255
    return rgba, s, y


def slice_pixels(fields, lx: int, lattice, mesh_origin, h, origin, U, V, width: int, height: int,
                 cols: np.ndarray, rows: np.ndarray):
    """Scalar at selected pixels only (NaN outside): the oracle for sampled
    checks of full-size images."""
    o, U_, V_ = (np.asarray(v, dtype=np.float64) for v in (origin, U, V))
    fc = (np.asarray(cols) + 0.5) / width
    fr = (np.asarray(rows) + 0.5) / height
    p = (o[None, :] + fc[:, None] * U_[None, :]) + fr[:, None] * V_[None, :]  # step 1, same order
    e, xi, inside = locate(p, lattice, mesh_origin, h)
    s = np.full(cols.shape, np.nan)
    if inside.any():
        s[inside] = scalar(interpolate(fields, lx, e[inside], xi[inside]))
    return s
