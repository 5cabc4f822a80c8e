"""Plain FP64 CPU oracle of the GLR step inside ADMM for Fourier-domain (MRI) imaging.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the library never imports it.

The MRI model of Section 3 is y = M F(x) (F the 2-D Fourier transform, M the
k-space sampling mask).  The paper forms GLR by replacing block matching with
global matching inside the NLR reconstruction (ADMM, ref. [26]).  Functions,
in the order one iteration uses them:

* ``fft2c`` / ``ifft2c``   -- the orthonormal, unshifted 2-D DFT and its inverse.
* ``mri_denoise``          -- one GLR pass on the complex image: key selection,
  global matching and aggregation treat the image as two channels (real,
  imaginary), which leaves every squared distance unchanged; the low-rank step
  works on the complex group matrix (``wnnm_complex``).
* ``admm_dc``              -- the data-consistency (x) update of ADMM.
* ``dc_residual``          -- ||M F(x) - y||_2, accumulated in FP64.
* ``mri_reconstruct``      -- the ADMM loop.

Readings (also listed in the design notes):

M1  Complex image = two channels (real plane, imaginary plane) for key
    selection (edge maps OR-ed over the two channels), matching (squared L2 of
    the 2 P^2 real values = sum of |p - q|^2 over the P^2 complex values) and
    aggregation (each plane averaged separately).
M2  Complex WNNM: the group is the complex P^2 x K matrix Y (column j =
    real half + i * imaginary half of patch j); its singular values s_i are
    shrunk with the formula of reading A9, sigma_w being the noise standard
    deviation per complex entry (E|n|^2 = sigma_w^2):
    sigma_hat_i = sqrt(max(s_i^2 - K sigma_w^2, 0)), tau_i = C sigma_w^2 /
    (sigma_hat_i + eps), s'_i = max(s_i - tau_i, 0), X^ = U diag(s') V^H.
M3  ADMM (scaled form): z = D(x + u); u = u + x - z;
    x = F^-1((M y + rho F(z - u)) / (M + rho)); start x = F^-1(y), u = 0.
    F is orthonormal and unshifted (k-space row k holds frequency k for k < H/2).
M4  The mask is Cartesian (whole k-space rows, variable density) as the
    workload description states; the paper's experiments use a radial mask.
M5  rho and the sigma_w schedule are workload parameters (the paper gives none).
"""
from __future__ import annotations

import numpy as np

from . import glr_oracle as G


def fft2c(x: np.ndarray) -> np.ndarray:
    """Orthonormal 2-D DFT of a complex image [H][W]: X[k,l] = sum x[r,c] e^{-2 pi i (kr/H + lc/W)} / sqrt(HW)."""
    return np.fft.fft2(np.asarray(x, dtype=np.complex128), norm="ortho")


def ifft2c(X: np.ndarray) -> np.ndarray:
    """Inverse of fft2c (the + sign in the exponent, same 1/sqrt(HW) scale)."""
    return np.fft.ifft2(np.asarray(X, dtype=np.complex128), norm="ortho")


def planes_to_complex(p: np.ndarray) -> np.ndarray:
    """[2][H][W] (real plane, imaginary plane) -> complex [H][W]."""
    p = np.asarray(p, dtype=np.float64)
    return p[0] + 1j * p[1]


def complex_to_planes(z: np.ndarray) -> np.ndarray:
    return np.stack([np.real(z), np.imag(z)])


def wnnm_complex(Y: np.ndarray, sigma_w: float, c: float, eps: float = 1e-16):
    """Reading M2 on one complex group Y (m rows x K columns).

    Returns (X_hat, rank, s, s')."""
    Yc = np.asarray(Y, dtype=np.complex128)
    K = Yc.shape[1]
    U, s, Vh = np.linalg.svd(Yc, full_matrices=False)
    sig_hat = np.sqrt(np.maximum(s * s - K * sigma_w * sigma_w, 0.0))
    tau = c * sigma_w * sigma_w / (sig_hat + eps)
    s_new = np.maximum(s - tau, 0.0)
    X = (U * s_new) @ Vh
    return X, int(np.count_nonzero(s_new > 0)), s, s_new


def group_to_complex(g: np.ndarray) -> np.ndarray:
    """A gathered group [K][2 m] (each row = real half, then imaginary half) -> complex m x K."""
    g = np.asarray(g, dtype=np.float64)
    m = g.shape[1] // 2
    return (g[:, :m] + 1j * g[:, m:]).T


def complex_to_group(Y: np.ndarray) -> np.ndarray:
    return np.concatenate([np.real(Y).T, np.imag(Y).T], axis=1)


def lowrank_groups_complex(groups: np.ndarray, sigma_w: float, c: float, eps: float = 1e-16):
    """wnnm_complex on every group [N][K][2 m]; returns (X_hat [N][K][2 m], rank[N])."""
    out = np.empty(groups.shape, dtype=np.float64)
    rank = np.empty(groups.shape[0], dtype=np.int32)
    for i in range(groups.shape[0]):
        X, r, _, _ = wnnm_complex(group_to_complex(groups[i]), sigma_w, c, eps)
        out[i] = complex_to_group(X)
        rank[i] = r
    return out, rank


def mri_denoise(x: np.ndarray, P: int, N: int, K: int, sigma_w: float, c: float, th: float, eps: float = 1e-16):
    """One GLR pass on a complex image given as planes x[2][H][W] (readings M1, M2)."""
    x = np.asarray(x, dtype=np.float64)
    Q = G.patch_matrix(x, P)
    keys, n_corner = G.select_keys(x, P, N, th)
    idx, dist = G.match_topk(x, P, keys, K, Q)
    groups = G.gather_groups(x, P, idx, Q)
    xh, rank = lowrank_groups_complex(groups, sigma_w, c, eps)
    v = G.aggregate(xh, idx, x, P)
    return v, {"keys": keys, "n_corner": n_corner, "idx": idx, "dist": dist, "rank": rank}


def admm_dc(y: np.ndarray, mask: np.ndarray, v: np.ndarray, rho: float) -> np.ndarray:
    """x = F^-1((M y + rho F(v)) / (M + rho)) with v = z - u (complex arrays; y in k-space)."""
    Mk = np.asarray(mask, dtype=np.float64)
    return ifft2c((Mk * np.asarray(y, dtype=np.complex128) + rho * fft2c(v)) / (Mk + rho))


def dc_residual(x: np.ndarray, y: np.ndarray, mask: np.ndarray) -> float:
    """||M F(x) - y||_2 (FP64)."""
    r = np.asarray(mask, dtype=np.float64) * fft2c(x) - np.asarray(y, dtype=np.complex128)
    return float(np.sqrt(np.sum(np.abs(r) ** 2)))


def mri_reconstruct(y, mask, P, N, K, sigmas, c, th, rho, eps=1e-16, callback=None):
    """ADMM with the GLR denoiser (reading M3).  y, the result: complex [H][W]."""
    y = np.asarray(y, dtype=np.complex128)
    x = ifft2c(y)
    u = np.zeros_like(x)
    for it, sw in enumerate(sigmas):
        zp, _ = mri_denoise(complex_to_planes(x + u), P, N, K, sw, c, th, eps)
        z = planes_to_complex(zp)
        u = u + x - z
        x = admm_dc(y, mask, z - u, rho)
        if callback is not None:
            callback(it, x, z, u)
    return x
