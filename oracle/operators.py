"""Grid and blob operators (oracle; test infrastructure only).

Conventions (readings of the paper where it is silent):
* Periodic domain [0, n_x h) x [0, n_y h) x [0, n_z h); cell (i, j, k) has its
  centre at ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h) (Sec. III.A: concentrations
  are cell-centred).
* Fields are NumPy arrays shaped (n_z, n_y, n_x), x fastest.
* Blob positions are an (N, 3) array of (x, y, z).
"""
from __future__ import annotations

import numpy as np

from .kernels import KERNELS, SUPPORT


def laplacian(c: np.ndarray, h: float) -> np.ndarray:
    """Standard 7-point periodic Laplacian L c (Sec. III.A: the (2d+1)-point L)."""
    s = np.zeros_like(c)
    for ax in range(3):
        s += np.roll(c, 1, axis=ax) + np.roll(c, -1, axis=ax)
    return (s - 6.0 * c) / (h * h)


def apply_A(c: np.ndarray, h: float, chi: float, alpha: float) -> np.ndarray:
    """A c = alpha c - chi L c  (Eq. Helmholtz with alpha = 1/dt; alpha = 0 is
    the steady case of Eq. steady_state / Appendix A)."""
    return alpha * c - chi * laplacian(c, h)


def axis_weights(x: float, n: int, h: float, w: int = 4) -> np.ndarray:
    """1-D periodic kernel weights phi_w(x/h - (i + 1/2)) for all n cells of an
    axis (Eq. tensor_product), summing over periodic images of the blob."""
    phi = KERNELS[w]
    centres = np.arange(n, dtype=np.float64) + 0.5
    u = x / h
    out = np.zeros(n, dtype=np.float64)
    m = int(np.ceil(SUPPORT[w] / n)) + 1
    for img in range(-m, m + 1):
        out += phi(u - centres + img * n)
    return out


def blob_weights(q: np.ndarray, dims, h: float, w: int = 4):
    """Per-blob (wx, wy, wz) full-axis weight vectors."""
    nx, ny, nz = dims
    return [(axis_weights(p[0], nx, h, w), axis_weights(p[1], ny, h, w),
             axis_weights(p[2], nz, h, w)) for p in np.asarray(q, dtype=np.float64)]


def interp(c: np.ndarray, q: np.ndarray, h: float, w: int = 4) -> np.ndarray:
    """Local averaging (J c)_i = sum_k phi_w(q_i - r_k) c_k (Sec. III.A, Eq.
    tensor_product; the composite operator of Sec. II.A)."""
    nz, ny, nx = c.shape
    out = np.zeros(len(q), dtype=np.float64)
    for b, (wx, wy, wz) in enumerate(blob_weights(q, (nx, ny, nz), h, w)):
        ix, iy, iz = np.nonzero(wx)[0], np.nonzero(wy)[0], np.nonzero(wz)[0]
        block = c[np.ix_(iz, iy, ix)]
        out[b] = np.einsum("kji,k,j,i->", block, wz[iz], wy[iy], wx[ix])
    return out


def spread(lam: np.ndarray, q: np.ndarray, dims, h: float, w: int = 4) -> np.ndarray:
    """Spreading (S lambda)_k = h^-3 sum_i phi_w(q_i - r_k) lambda_i, i.e.
    S = Delta V_f^-1 J^T with Delta V_f = h^3 (Sec. III.A)."""
    nx, ny, nz = dims
    out = np.zeros((nz, ny, nx), dtype=np.float64)
    for b, (wx, wy, wz) in enumerate(blob_weights(q, dims, h, w)):
        ix, iy, iz = np.nonzero(wx)[0], np.nonzero(wy)[0], np.nonzero(wz)[0]
        out[np.ix_(iz, iy, ix)] += lam[b] * np.einsum("k,j,i->kji", wz[iz], wy[iy], wx[ix])
    return out / h ** 3


def helmholtz_eigenvalues(dims, h: float, chi: float, alpha: float) -> np.ndarray:
    """Eigenvalues of A = alpha I - chi L on the periodic grid, shaped like the
    FFT of a field: alpha + (4 chi / h^2) sum_d sin^2(pi k_d / n_d)."""
    nx, ny, nz = dims
    sx = np.sin(np.pi * np.arange(nx) / nx) ** 2
    sy = np.sin(np.pi * np.arange(ny) / ny) ** 2
    sz = np.sin(np.pi * np.arange(nz) / nz) ** 2
    return alpha + (4.0 * chi / (h * h)) * (sz[:, None, None] + sy[None, :, None] + sx[None, None, :])


def green_apply(g: np.ndarray, h: float, chi: float, alpha: float) -> np.ndarray:
    """G g with G = A^-1 (alpha > 0), or, for alpha = 0, the restricted inverse
    of Appendix A: it acts on the mean-zero part of g and returns a mean-zero
    field (the k = 0 Fourier mode is dropped)."""
    nz, ny, nx = g.shape
    lam = helmholtz_eigenvalues((nx, ny, nz), h, chi, alpha)
    gh = np.fft.fftn(g)
    if alpha == 0.0:
        lam = lam.copy()
        lam[0, 0, 0] = 1.0
        gh[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(gh / lam))
