"""In-situ slice image (Sec. IV-A) on the GPU against the FP64 oracle.

Which element owns a pixel is decided in FP64 on both sides with the same
operations, so the set of inside pixels, and the background elsewhere, must
match exactly.  The value and colour run in FP32 on the GPU: the value must
lie within the FP32 error bound of the oracle's FP64 value,
    eps_s = (8 lx + 16) 2^-24 Lambda^3 max|u|
(every basis value and every partial sum rounds O(lx) times; Lambda is the
Lebesgue constant of the GLL basis, max over x of sum_i |l_i(x)|, so
sum |l_i l_j l_k u| <= Lambda^3 max|u|), and each colour byte must equal the
oracle's except where the oracle's 255 c lies within the propagated bound of
a rounding tie k + 1/2, where it may differ by one.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.slice as oslice
import paper_2407_20731_b300 as semr
import synth

pytestmark = pytest.mark.gpu

TWO_PI = 2.0 * np.pi
CTRL = semr.COOL_WARM


def _lebesgue(lx):
    nodes, _ = oracle.gll(lx)
    x = np.linspace(-1.0, 1.0, 4001)
    return np.abs(oslice.lagrange(nodes, x)).sum(axis=1).max()


def _fields(n, lx, n_comp, seed=21):
    E = n[0] * n[1] * n[2]
    f, _ = synth.snapshot(E, lx, [seed + c for c in range(n_comp)], device="cuda")
    return f.reshape(n_comp, E, lx ** 3).contiguous()


def _render(fields, lx, n, origin, U, V, W, H, vmin, vmax, mo=(0.0, 0.0, 0.0), h=None, bg=0):
    nc = fields.shape[0]
    mesh = semr.make_lattice(lx, n, mo, h)
    sl = semr.make_slice(origin, U, V, W, H, vmin, vmax, nc, CTRL, bg)
    vals = torch.empty((H, W), dtype=torch.float32, device="cuda")
    rgba, _ = semr.slice_rgba([fields[c] for c in range(nc)], mesh, sl, values=vals)
    torch.cuda.synchronize()
    return rgba.cpu().numpy(), vals.cpu().numpy(), mesh


def _bounds(lx, umax, nc, vmin, vmax):
    eps_s = (8 * lx + 16) * 2.0 ** -24 * _lebesgue(lx) ** 3 * umax
    if nc > 1:
        eps_s = np.sqrt(nc) * eps_s
    c = np.asarray(CTRL)
    slope = np.max(np.abs(np.diff(c[:, 1:], axis=0)) / np.diff(c[:, 0])[:, None])
    eps_y = 255.0 * (slope * (2.0 * eps_s / (vmax - vmin) + 2.0 ** -20) + 2.0 ** -20)
    return 2.0 * eps_s, eps_y


def _check_against_oracle(rgba, vals, s_o, y_o, inside, bg, lx, umax, nc, vmin, vmax):
    # ownership: identical inside / outside sets, background outside
    assert np.array_equal(np.isfinite(vals), inside)
    bgb = np.frombuffer(np.uint32(bg).tobytes(), dtype=np.uint8)
    assert np.all(rgba[~inside] == bgb)
    assert np.all(rgba[inside, 3] == 255)
    eps_s, eps_y = _bounds(lx, umax, nc, vmin, vmax)
    err = np.abs(vals[inside].astype(np.float64) - s_o[inside])
    assert err.size == 0 or err.max() <= eps_s, (err.max(), eps_s)
    yo = y_o[inside]
    ob = np.clip(np.floor(yo + 0.5), 0, 255)
    gb = rgba[inside, :3].astype(np.float64)
    fr = (yo + 0.5) - np.floor(yo + 0.5)
    near = (fr <= eps_y) | (1.0 - fr <= eps_y)
    d = np.abs(gb - ob)
    assert np.all(d <= 1)
    assert np.all(d[~near] == 0), np.argwhere((d > 0) & ~near)[:5]
    return int(near.sum()), int((d > 0).sum())


def _full_check(fields, lx, n, origin, U, V, W, H, vmin, vmax, bg=0, h=None):
    rgba, vals, mesh = _render(fields, lx, n, origin, U, V, W, H, vmin, vmax, bg=bg, h=h)
    f_np = fields.cpu().numpy()
    hh = [mesh.h[d] for d in range(3)]
    ro, s_o, y_o = oslice.slice_rgba(f_np, lx, n, (0, 0, 0), hh, origin, U, V, W, H, vmin, vmax, CTRL,
                                     background=tuple(np.frombuffer(np.uint32(bg).tobytes(), dtype=np.uint8)))
    inside = np.isfinite(s_o)
    umax = float(np.abs(f_np).max())
    _check_against_oracle(rgba, vals, s_o, y_o, inside, bg, lx, umax, fields.shape[0], vmin, vmax)
    return rgba, vals, inside


@pytest.mark.parametrize("nc", [1, 3])
def test_z_slice_axis_path(nc):
    n, lx = (16, 16, 16), 8
    f = _fields(n, lx, nc)
    rgba, vals, inside = _full_check(f, lx, n, (0.0, 0.0, 2.0), (TWO_PI, 0, 0), (0, TWO_PI, 0), 192, 160,
                                     0.0 if nc > 1 else -2.0, 3.0)
    assert inside.all()


@pytest.mark.parametrize("lx", [2, 3, 4, 6, 10, 12])
def test_every_lx(lx):
    n = (6, 5, 4)
    f = _fields(n, lx, 2)
    _full_check(f, lx, n, (0.0, 0.0, 2.5), (TWO_PI, 0, 0), (0, TWO_PI, 0), 70, 53, 0.0, 3.0)


def test_x_normal_and_transposed_and_mirrored():
    n, lx = (8, 9, 10), 6
    f = _fields(n, lx, 1, seed=31)
    _full_check(f, lx, n, (1.3, 0.0, 0.0), (0, TWO_PI, 0), (0, 0, TWO_PI), 90, 100, -2.5, 2.5)   # x normal
    _full_check(f, lx, n, (0.0, 0.0, 4.0), (0, TWO_PI, 0), (TWO_PI, 0, 0), 64, 77, -2.5, 2.5)    # columns along y
    _full_check(f, lx, n, (TWO_PI, 0.0, 4.0), (-TWO_PI, 0, 0), (0, TWO_PI, 0), 81, 64, -2.5, 2.5)  # mirrored


def test_partly_outside_and_missing_plane():
    n, lx = (8, 8, 8), 8
    f = _fields(n, lx, 3, seed=41)
    bg = 0x44332211
    rgba, vals, inside = _full_check(f, lx, n, (-1.0, -0.5, 2.0), (TWO_PI + 2.0, 0, 0), (0, TWO_PI + 1.0, 0),
                                     97, 89, 0.0, 3.0, bg=bg)
    assert inside.any() and not inside.all()
    rgba, vals, inside = _full_check(f, lx, n, (0.0, 0.0, 10.0), (TWO_PI, 0, 0), (0, TWO_PI, 0), 40, 30, 0.0, 3.0,
                                     bg=bg)
    assert not inside.any()


def test_faces_of_the_lattice():
    """A slice exactly on an interior element face and on the top face: the
    upper element (zeta = -1) and the last element (zeta = +1) own them."""
    n, lx = (4, 4, 4), 5
    h = (1.0, 1.0, 1.0)  # exact face coordinates
    f = _fields(n, lx, 1, seed=51)
    _full_check(f, lx, n, (0.0, 0.0, 2.0), (4.0, 0, 0), (0, 4.0, 0), 32, 32, -2.0, 2.0, h=h)
    _full_check(f, lx, n, (0.0, 0.0, 4.0), (4.0, 0, 0), (0, 4.0, 0), 32, 32, -2.0, 2.0, h=h)


@pytest.mark.parametrize("lx", [5, 8])
def test_oblique_plane_generic_path(lx):
    n = (6, 6, 6)
    f = _fields(n, lx, 2, seed=61)
    rgba, vals, inside = _full_check(f, lx, n, (0.2, 0.3, 0.5), (5.0, 1.0, 0.5), (-0.5, 2.0, 4.0), 120, 96,
                                     0.0, 3.0, bg=0x01020304)
    assert inside.any() and not inside.all()


def test_deterministic_and_values_optional():
    n, lx = (8, 8, 8), 8
    f = _fields(n, lx, 3, seed=71)
    mesh = semr.make_lattice(lx, n)
    sl = semr.make_slice((0, 0, 1.0), (TWO_PI, 0, 0), (0, TWO_PI, 0), 128, 128, 0.0, 3.0, 3)
    a, _ = semr.slice_rgba([f[c] for c in range(3)], mesh, sl)
    b, _ = semr.slice_rgba([f[c] for c in range(3)], mesh, sl)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_full_size_sampled():
    """64^3 elements, lx = 8, velocity magnitude of three fields, 2048^2
    image of the plane z = 2: 4000 sampled pixels against the oracle (which
    gets the sliced layer of elements only)."""
    n, lx, W, H = (64, 64, 64), 8, 2048, 2048
    f = _fields(n, lx, 3, seed=10)
    z0, vmin, vmax = 2.0, 0.0, 3.0
    rgba, vals, mesh = _render(f, lx, n, (0.0, 0.0, z0), (TWO_PI, 0, 0), (0, TWO_PI, 0), W, H, vmin, vmax)
    hz = mesh.h[2]
    layer = int(np.floor(z0 / hz))
    ids = torch.arange(64 * 64, device="cuda") + 64 * 64 * layer
    sub = f[:, ids].cpu().numpy()
    rng = np.random.default_rng(5)
    cols, rows = rng.integers(0, W, 4000), rng.integers(0, H, 4000)
    s_o = oslice.slice_pixels(sub, lx, (64, 64, 1), (0.0, 0.0, layer * hz), [mesh.h[0], mesh.h[1], hz],
                              (0.0, 0.0, z0), (TWO_PI, 0, 0), (0, TWO_PI, 0), W, H, cols, rows)
    assert np.all(np.isfinite(s_o))
    y_o = oslice.colour_channels(s_o, vmin, vmax, CTRL)
    g = rgba[rows, cols]
    v = vals[rows, cols]
    _check_against_oracle(g[None], v[None], s_o[None], y_o[None], np.ones((1, s_o.size), bool), 0, lx,
                          float(np.abs(sub).max()), 3, vmin, vmax)
