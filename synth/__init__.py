"""Seeded synthetic SEM snapshots: the inputs that both the CUDA path and the
CPU oracle consume.

This module holds none of the reduction's arithmetic.  It only places sample
points and evaluates a made-up turbulent-looking field there.  The paper's
workload is a NEKO Taylor-Green-vortex snapshot on 64^3 hexahedral elements
(arXiv 2407.20731, Sec. IV-A/IV-B), which needs the NEKO solver to produce;
these generated snapshots stand in for it with the same shape:

* mesh: an (nx, ny, nz) lattice of affine hex elements on [0, 2 pi)^3, element
  index e = ex + nx (ey + ny ez); in each element the lx points per direction
  sit at the Gauss-Lobatto-Legendre positions (numpy's Legendre-series root
  finder places them), mapped affinely;
* Jacobians: J_e ~ U[0.5, 2], drawn independently per element (a synthetic
  mass scale, not the geometric volume), numpy PCG64 with seed ``jac_seed``;
* field: u(x) = sum_{m=1}^{16} A_m cos(k_m . x + phi_m) + N(0, sigma^2),
  sigma = 1e-6, with k_m integer vectors of uniformly random direction and
  magnitude log-uniform in [1, k_max] (rounded to integers, zero redrawn),
  k_max = the number of elements per side, A_m = |k_m|^slope and
  phi_m ~ U[0, 2 pi); mode parameters from numpy
  PCG64 with the field's seed; the noise from torch's generator on the device
  that holds the snapshot, seeded with the same seed.

Layout of a field: [n_elem, lx, lx, lx] FP64 = u[e][k][j][i], i fastest.
"""
from __future__ import annotations

import math

import numpy as np
import torch

N_MODES = 16
NOISE_SIGMA = 1e-6


def sample_points(lx: int) -> np.ndarray:
    """Reference-element sample positions in [-1, 1]: -1, the roots of P_N'
    (numpy's Legendre-series root finder), +1."""
    N = lx - 1
    if N < 1:
        raise ValueError("lx >= 2")
    inner = np.polynomial.legendre.Legendre.basis(N).deriv().roots() if N > 1 else np.zeros(0)
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


def lattice(n_elem: int) -> tuple[int, int, int]:
    """Element lattice (nx, ny, nz) that holds n_elem elements: a cube when
    n_elem is a perfect cube, else nx = ny = ceil(cbrt(n_elem)) and enough
    layers; the first n_elem lattice elements (x fastest) are used."""
    c = round(n_elem ** (1.0 / 3.0))
    if c ** 3 == n_elem:
        return c, c, c
    nx = int(math.ceil(n_elem ** (1.0 / 3.0)))
    nz = int(math.ceil(n_elem / (nx * nx)))
    return nx, nx, nz


def mode_parameters(seed: int, k_max: int, slope: float, n_modes: int = N_MODES):
    """(k [n_modes, 3] int, amplitude [n_modes], phase [n_modes]).

    Each wave vector has a uniformly random direction and a magnitude
    log-uniform in [1, k_max], rounded to the integer lattice (a zero vector is
    redrawn), so the 16 modes spread over the scales that the |k|^slope
    amplitude weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = []
    while len(ks) < n_modes:
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        mag = math.exp(rng.uniform(0.0, math.log(max(k_max, 1))))
        k = np.rint(d * mag).astype(np.int64)
        if np.any(k != 0):
            ks.append(k)
    k = np.array(ks, dtype=np.int64)
    amp = np.linalg.norm(k.astype(np.float64), axis=1) ** slope
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return k, amp, phase


def jacobians(n_elem: int, seed: int = 2, device="cpu") -> torch.Tensor:
    rng = np.random.Generator(np.random.PCG64(seed))
    return torch.from_numpy(rng.uniform(0.5, 2.0, size=n_elem)).to(device)


def field(n_elem: int, lx: int, seed: int, slope: float = -5.0 / 3.0, device="cpu",
          noise: float = NOISE_SIGMA) -> torch.Tensor:
    """One FP64 field [n_elem, lx, lx, lx] on ``device``."""
    nx, ny, nz = lattice(n_elem)
    k_max = max(nx, ny, nz)
    k, amp, phase = mode_parameters(seed, k_max, slope)
    xi = sample_points(lx)
    dev = torch.device(device)

    def axis(ne: int) -> torch.Tensor:  # global coordinate of every (element, point) along one axis
        h = 2.0 * np.pi / ne
        c = (np.arange(ne)[:, None] + 0.5 * (xi[None, :] + 1.0)) * h
        return torch.from_numpy(c.reshape(-1)).to(dev)

    X, Y, Z = axis(nx), axis(ny), axis(nz)
    # cos(kx X + ky Y + kz Z + phi) = Re(P[Z, Y] e^{i kx X}), P = A e^{i phi} e^{i kz Z} e^{i ky Y}:
    # one real GEMM [Z*Y, 2M] @ [2M, X] sums all modes.
    kt = torch.from_numpy(k).to(dev, torch.float64)
    ph = torch.from_numpy(phase).to(dev)
    am = torch.from_numpy(amp).to(dev)
    argzy = (kt[:, 2, None, None] * Z[None, :, None] + kt[:, 1, None, None] * Y[None, None, :]
             + ph[:, None, None])                                  # [M, Z, Y]
    pr = (am[:, None, None] * torch.cos(argzy)).reshape(len(amp), -1)
    pi = (am[:, None, None] * torch.sin(argzy)).reshape(len(amp), -1)
    argx = kt[:, 0, None] * X[None, :]                              # [M, X]
    lhs = torch.cat([pr, -pi], dim=0).T.contiguous()                 # [Z*Y, 2M]
    rhs = torch.cat([torch.cos(argx), torch.sin(argx)], dim=0)       # [2M, X]
    u = (lhs @ rhs).reshape(nz, lx, ny, lx, nx, lx)                  # [ez, k, ey, j, ex, i]
    u = u.permute(0, 2, 4, 1, 3, 5).reshape(nx * ny * nz, lx, lx, lx)[:n_elem].contiguous()
    if noise > 0:
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        u.add_(torch.randn(u.shape, generator=g, device=dev, dtype=torch.float64), alpha=noise)
    return u


def snapshot(n_elem: int, lx: int, seeds, slope: float = -5.0 / 3.0, device="cpu",
             jac_seed: int = 2, noise: float = NOISE_SIGMA):
    """(fields [F, n_elem, lx, lx, lx], jac [n_elem]) with one seed per field."""
    fs = torch.stack([field(n_elem, lx, s, slope, device, noise) for s in seeds])
    return fs, jacobians(n_elem, jac_seed, device)


# The workload shapes the benchmarks and parity tests use.
def small_case(device="cpu"):
    """512 elements (8^3), lx = 8, one field (seed 1), tau = 1e-3."""
    f, j = snapshot(512, 8, [1], device=device)
    return f, j, 1e-3


def full_case(device="cuda"):
    """64^3 = 262,144 elements, lx = 8, fields u, v, w, p (seeds 10..13)."""
    return snapshot(64 ** 3, 8, [10, 11, 12, 13], device=device)


def batched_cases(n_snap: int = 64, seed: int = 1000):
    """Shapes of the uneven batch: per snapshot (n_elem, lx, n_fields, slope,
    field seeds).  Element counts log-uniform in [4096, 200000], lx from
    {6, 8, 10}, 1-4 fields, spectral slope uniform in [-3, -5/3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_snap):
        ne = int(round(math.exp(rng.uniform(math.log(4096), math.log(200000)))))
        lx = int(rng.choice([6, 8, 10]))
        nf = int(rng.integers(1, 5))
        slope = float(rng.uniform(-3.0, -5.0 / 3.0))
        out.append(dict(n_elem=ne, lx=lx, n_fields=nf, slope=slope,
                        seeds=[seed + i * 8 + f for f in range(nf)]))
    return out
