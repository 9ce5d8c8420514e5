"""Seeded blob placements, rates and sources (no arithmetic of the method).

Random numbers come from numpy's PCG64 ``default_rng`` so that the x86 test host
and the aarch64 GPU host draw identical bytes for the same seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    return d - box * np.round(d / box)


def rsa_positions(n_blobs: int, dims, h: float, spacing: float, seed: int,
                  max_attempts: int = 200) -> np.ndarray:
    """Random sequential addition in a periodic box [0, n*h)^3.

    Draws uniform candidate centres and rejects any whose minimum-image distance
    to an accepted centre is below ``spacing``. Returns an (N, 3) FP64 array of
    (x, y, z) positions. A cell list with cells at least ``spacing`` wide keeps
    each test to the 27 neighbouring cells. Raises ``RuntimeError`` if the
    packing cannot be reached within ``max_attempts * n_blobs`` draws.
    """
    nx, ny, nz = (int(v) for v in dims)
    box = np.array([nx * h, ny * h, nz * h], dtype=np.float64)
    rng = np.random.default_rng(seed)
    ncell = np.maximum(1, np.floor(box / spacing).astype(int))
    csize = box / ncell
    cells: dict = {}
    out = np.empty((n_blobs, 3), dtype=np.float64)
    count = 0
    attempts = 0
    sp2 = spacing * spacing
    while count < n_blobs:
        attempts += 1
        if attempts > max_attempts * max(n_blobs, 1):
            raise RuntimeError(f"RSA could not place {n_blobs} blobs at spacing {spacing}")
        p = rng.random(3) * box
        ci = np.floor(p / csize).astype(int) % ncell
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((ci[0] + dx) % ncell[0], (ci[1] + dy) % ncell[1], (ci[2] + dz) % ncell[2])
                    for j in cells.get(key, ()):
                        d = _min_image(out[j] - p, box)
                        if float(d @ d) < sp2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        out[count] = p
        cells.setdefault((int(ci[0]), int(ci[1]), int(ci[2])), []).append(count)
        count += 1
    return out


def lattice_positions(dims, h: float, spacing_cells: int, offset=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Cubic array of blobs every ``spacing_cells`` cells along each axis.

    Blob (a, b, c) sits at ((a*spacing + offset_x) h, ...), so with a zero
    offset every blob is on a grid node (a cell corner).
    """
    nx, ny, nz = (int(v) for v in dims)
    s = int(spacing_cells)
    xs = (np.arange(0, nx, s) + offset[0]) * h
    ys = (np.arange(0, ny, s) + offset[1]) * h
    zs = (np.arange(0, nz, s) + offset[2]) * h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)


def single_blob_position(dims, h: float, seed: int) -> np.ndarray:
    """One blob at a seeded uniform sub-cell offset from the box centre node."""
    nx, ny, nz = (int(v) for v in dims)
    rng = np.random.default_rng(seed)
    u = rng.random(3)
    return (np.array([[nx // 2, ny // 2, nz // 2]], dtype=np.float64) + u[None, :]) * h


def loguniform_rates(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Per-blob rates drawn log-uniformly in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n)).astype(np.float64)


def uniform_source(dims, value: float = 1.0) -> np.ndarray:
    """Uniform source field, shaped (nz, ny, nx), x fastest."""
    nx, ny, nz = (int(v) for v in dims)
    return np.full((nz, ny, nx), float(value), dtype=np.float64)


@dataclasses.dataclass
class Workload:
    name: str
    dims: tuple
    h: float
    chi: float
    q: np.ndarray          # (N, 3) blob positions
    kappa: np.ndarray      # (N,) reaction rates (reaction-limited case)
    g: np.ndarray          # (nz, ny, nx) source
    alpha: float = 0.0


def workload(name: str) -> Workload:
    """Named synthetic workloads.

    * ``tiny``   : 32^3, one blob at (16 + u)h, u ~ U[0,1)^3 (seed 1), g = 1.
    * ``scale``  : 256^3, 4096 blobs, RSA spacing 4h (seed 2), rates
                   log-uniform in [0.1, 10] (seed 3), g = 1.
    * ``mixed``  : 512^3, 32768 blobs, RSA spacing 3h (seed 4), g = 1.
    * ``mixed64``: the ``mixed`` rule at 64^3 with 64 blobs (seed 4).
    * ``small``  : 32^3, 48 blobs, RSA spacing 4h (seed 5), rates as ``scale``
                   (seed 6): several tiles and a ragged blob count.
    """
    h, chi = 1.0, 1.0
    if name == "tiny":
        d = (32, 32, 32)
        q = single_blob_position(d, h, 1)
        kappa = np.ones(1)
    elif name == "scale":
        d = (256, 256, 256)
        q = rsa_positions(4096, d, h, 4.0, 2)
        kappa = loguniform_rates(4096, 0.1, 10.0, 3)
    elif name == "mixed":
        d = (512, 512, 512)
        q = rsa_positions(32768, d, h, 3.0, 4)
        kappa = loguniform_rates(32768, 0.1, 10.0, 7)
    elif name == "mixed64":
        d = (64, 64, 64)
        q = rsa_positions(64, d, h, 3.0, 4)
        kappa = loguniform_rates(64, 0.1, 10.0, 7)
    elif name == "small":
        d = (32, 32, 32)
        q = rsa_positions(48, d, h, 4.0, 5)
        kappa = loguniform_rates(48, 0.1, 10.0, 6)
    else:
        raise KeyError(name)
    return Workload(name, d, h, chi, q, kappa, uniform_source(d, 1.0))


def batch_workloads(count: int, sides=(64, 96, 128, 160), n_lo: int = 16, n_hi: int = 2000,
                    spacing: float = 3.0, seed: int = 11) -> list:
    """Independent disordered-suspension realisations of uneven size: realisation
    i has a cubic grid whose side is drawn uniformly from ``sides``, a blob count
    drawn log-uniformly in [n_lo, n_hi] (rounded), RSA placement with minimum
    centre spacing ``spacing`` h, rates log-uniform in [0.1, 10] and g = 1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(sides[int(rng.integers(len(sides)))])
        n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
        d = (side, side, side)
        q = rsa_positions(n, d, 1.0, spacing, seed * 1000 + 2 * i)
        kappa = loguniform_rates(n, 0.1, 10.0, seed * 1000 + 2 * i + 1)
        out.append(Workload(f"batch{i}", d, 1.0, 1.0, q, kappa, uniform_source(d, 1.0)))
    return out
