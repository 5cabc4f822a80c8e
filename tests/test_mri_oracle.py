"""Pins of the MRI (ADMM) oracle against closed forms and properties (CPU only)."""
import math

import numpy as np
import pytest

from oracle import glr_oracle as G
from oracle import mri_oracle as MO
from paper_2301_03047_gb300 import synth


def test_fft_convention_closed_forms():
    H, W = 8, 16
    d = np.zeros((H, W), complex)
    d[0, 0] = 1.0
    assert np.allclose(MO.fft2c(d), 1.0 / math.sqrt(H * W))
    r, c = np.mgrid[0:H, 0:W]
    k0, l0 = 3, 5
    tone = np.exp(2j * np.pi * (k0 * r / H + l0 * c / W))
    X = MO.fft2c(tone)
    want = np.zeros((H, W), complex)
    want[k0, l0] = math.sqrt(H * W)
    assert np.allclose(X, want, atol=1e-12)
    z = synth.rng_for("fft").standard_normal((H, W)) + 1j * synth.rng_for("fft", 1).standard_normal((H, W))
    assert np.isclose(np.linalg.norm(MO.fft2c(z)), np.linalg.norm(z))  # Parseval
    assert np.allclose(MO.ifft2c(MO.fft2c(z)), z)


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_dc_update_is_the_minimiser():
    """x = argmin ||M F x - y||^2 + rho ||x - v||^2: the gradient F^H M (M F x - y) + rho (x - v) vanishes."""
    rng = synth.rng_for("dc")
    H, W = 16, 12
    M = (rng.random((H, W)) < 0.3).astype(float)
    y = M * _cplx(rng, H, W)
    v = _cplx(rng, H, W)
    for rho in (0.1, 1.0, 7.0):
        x = MO.admm_dc(y, M, v, rho)
        g = MO.ifft2c(M * (M * MO.fft2c(x) - y)) + rho * (x - v)
        assert np.abs(g).max() < 1e-12
    # no samples: x = v; everything sampled and rho -> 0: x = F^-1 y
    assert np.allclose(MO.admm_dc(np.zeros((H, W)), np.zeros((H, W)), v, 0.5), v)
    yf = _cplx(rng, H, W)
    assert np.allclose(MO.admm_dc(yf, np.ones((H, W)), v, 1e-12), MO.ifft2c(yf), atol=1e-9)


def test_dc_residual_special_cases():
    rng = synth.rng_for("res")
    y = _cplx(rng, 8, 8)
    assert MO.dc_residual(MO.ifft2c(y), y, np.ones((8, 8))) < 1e-12
    assert np.isclose(MO.dc_residual(np.zeros((8, 8)), y, np.ones((8, 8))), np.linalg.norm(y))


def test_wnnm_complex_reduces_to_real_and_is_phase_invariant():
    rng = synth.rng_for("wc")
    Y = rng.standard_normal((36, 24))
    for sw in (0.0, 0.3, 1.0):
        Xc, rc, sc, _ = MO.wnnm_complex(Y.astype(complex), sw, 2 * math.sqrt(24))
        Xr, rr, sr, _ = G.wnnm(Y, sw, 2 * math.sqrt(24))
        assert np.allclose(Xc.imag, 0, atol=1e-12) and np.allclose(Xc.real, Xr) and rc == rr
        assert np.allclose(sc, sr)
    Yc = _cplx(rng, 36, 24)
    th = 0.7
    X1, _, _, _ = MO.wnnm_complex(Yc, 0.4, 9.8)
    X2, _, _, _ = MO.wnnm_complex(Yc * np.exp(1j * th), 0.4, 9.8)
    assert np.allclose(X2, X1 * np.exp(1j * th))
    Q, _ = np.linalg.qr(_cplx(rng, 36, 36))  # unitary
    X3, _, _, _ = MO.wnnm_complex(Q @ Yc, 0.4, 9.8)
    assert np.allclose(X3, Q @ X1)
    X0, r0, _, _ = MO.wnnm_complex(Yc, 0.0, 9.8)
    assert np.allclose(X0, Yc) and r0 == 24


def test_wnnm_complex_rank1_closed_form():
    rng = synth.rng_for("wc1")
    u = _cplx(rng, 18)
    u /= np.linalg.norm(u)
    v = _cplx(rng, 10)
    v /= np.linalg.norm(v)
    s, K, sw, c = 5.0, 10, 0.3, 2 * math.sqrt(10)
    Y = s * np.outer(u, v.conj())
    X, r, _, _ = MO.wnnm_complex(Y, sw, c)
    tau = c * sw * sw / math.sqrt(s * s - K * sw * sw)
    assert r == 1 and np.allclose(X, (s - tau) * np.outer(u, v.conj()))


def test_complex_group_layout_and_distance():
    """Reading M1: the two-channel distance is the sum of |p - q|^2 over complex entries."""
    rng = synth.rng_for("lay")
    P = 3
    x = rng.random((2, 9, 10))
    Q = G.patch_matrix(x, P)
    z = x[0] + 1j * x[1]
    q = 2 * 8 + 4  # r = 2, c = 4 (Wq = 8)
    g = MO.group_to_complex(Q[[q]])
    assert np.allclose(g[:, 0], z[2:5, 4:7].reshape(-1))
    assert np.allclose(MO.complex_to_group(g), Q[[q]])
    keys = np.array([q, 0], np.int32)
    idx, dist = G.match_topk(x, P, keys, 5, Q)
    zp = z[2:5, 4:7]
    for j in range(5):
        r, c = divmod(int(idx[0, j]), 8)
        assert np.isclose(dist[0, j], np.sum(np.abs(z[r:r + 3, c:c + 3] - zp) ** 2))


def test_mask_recipe():
    m = synth.cartesian_mask(synth.rng_for("mask"), 64, 32, 0.25, 8)
    rows = m[:, 0] > 0
    assert rows.sum() == 16 and np.all(m == m[:, :1])
    assert rows[[0, 1, 2, 3, 60, 61, 62, 63]].all()  # the 8 lowest frequencies


@pytest.mark.slow
def test_admm_improves_on_zero_filling():
    cfg = synth.mri_scaled(synth.MRI_SMALL, iters=4)
    p = synth.mri_problem(cfg)
    y = MO.planes_to_complex(p.y)
    gt = MO.planes_to_complex(p.truth)
    x0 = MO.ifft2c(y)
    x = MO.mri_reconstruct(y, p.mask, cfg.P, cfg.N, cfg.K, cfg.sigma_schedule(), cfg.c_wnnm, cfg.edge_th, cfg.rho)
    err0 = np.mean(np.abs(x0 - gt) ** 2)
    err = np.mean(np.abs(x - gt) ** 2)
    assert err < 0.9 * err0
    assert MO.dc_residual(x, y, p.mask) < np.linalg.norm(y)
