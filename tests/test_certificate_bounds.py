"""The mathematics the rank-1 certificate of the WNNM kernel rests on, checked on the CPU
against the oracle's WNNM (Eq. 5 with the weights of ref. [15]) and an FP64 SVD.

* WNNM removes a component exactly when s <= s_crit, s_crit^2 = sw^2 (K + sqrt(K^2 + 4 C^2)) / 2
  (the root of s = C sw^2 / sqrt(s^2 - K sw^2)): a rank-1 group just below s_crit returns
  rank 0, just above it rank 1.
* For any unit vector v and mu = ||Y v||^2:
    energy bound  s_2^2 <= ||Y||_F^2 - mu,
    Gram bound    s_2^2 <= lambda_max(R^T R) <= ||R^T R||_F,  R = Y (I - v v^T)
  (Cauchy interlacing: R^T R is Y^T Y compressed to the complement of v), also for a v
  that is only near the dominant right singular vector.
* When only the first component survives, X^ = s_1' u u^T Y with u = Y v / ||Y v||, i.e.
  X^ = coef y (y^T Y), y = Y v, coef = s_1' / (s_1 ||y||^2): the oracle's X^ on such groups.
"""
import math

import numpy as np
import pytest

from oracle import glr_oracle as O


def s_crit2(sw, K, C):
    return sw * sw * (K + math.sqrt(K * K + 4 * C * C)) / 2


@pytest.mark.parametrize("K,d", [(64, 64), (40, 64), (16, 36)])
def test_wnnm_threshold_is_s_crit(K, d):
    rng = np.random.default_rng(K + d)
    sw, C = 0.1, 2 * math.sqrt(K)
    sc = math.sqrt(s_crit2(sw, K, C))
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    v = rng.standard_normal(K)
    v /= np.linalg.norm(v)
    for f, want in ((1 - 1e-6, 0), (1 + 1e-6, 1)):
        Y = (f * sc) * np.outer(u, v)  # d x K, one singular value f s_crit
        _, r, s, s_new = O.wnnm(Y, sw, C, eps=1e-30)
        assert r == want, (f, s[0], s_new[0])


def _near_rank1(rng, d, K, noise, scale=1.0):
    u = rng.random(d)
    return scale * np.outer(u, 1 + 0.1 * rng.standard_normal(K)) + noise * rng.standard_normal((d, K))


@pytest.mark.parametrize("noise", [0.0, 0.01, 0.05, 0.3])
def test_energy_and_gram_bounds_hold_for_inexact_v(noise):
    rng = np.random.default_rng(int(noise * 1000) + 7)
    d = K = 64
    for trial in range(40):
        Y = _near_rank1(rng, d, K, noise)
        _, s, Vt = np.linalg.svd(Y)
        s2 = s[1] ** 2
        for eps in (0.0, 1e-4, 1e-2, 0.3):  # v at angle ~eps from the dominant vector
            v = Vt[0] + eps * rng.standard_normal(K)
            v /= np.linalg.norm(v)
            y = Y @ v
            mu = y @ y
            energy = (Y * Y).sum() - mu
            R = Y - np.outer(y, v)
            G = R.T @ R
            gram = math.sqrt((G * G).sum())
            lam_max = np.linalg.eigvalsh(G)[-1]
            tol = 1e-12 * (Y * Y).sum()
            assert s2 <= energy + tol
            assert s2 <= lam_max + tol
            assert lam_max <= gram + tol
            assert mu <= s[0] ** 2 + tol  # the Rayleigh quotient never exceeds s_1^2


def test_gram_bound_is_tighter_than_energy_on_spread_noise():
    """The case the Gram bound exists for: rank-1 plus noise spread over all components; the
    energy bound is about sqrt(K - 1) / sqrt(2) times larger (Marchenko-Pastur, ratio 1)."""
    rng = np.random.default_rng(3)
    d = K = 64
    ratios = []
    for _ in range(20):
        Y = _near_rank1(rng, d, K, 0.02, scale=1.0)
        _, s, Vt = np.linalg.svd(Y)
        v = Vt[0]
        y = Y @ v
        energy = (Y * Y).sum() - y @ y
        R = Y - np.outer(y, v)
        G = R.T @ R
        ratios.append(energy / math.sqrt((G * G).sum()))
    assert min(ratios) > 4.0, min(ratios)


@pytest.mark.parametrize("sw", [0.05, 0.1])
def test_rank1_output_formula_equals_the_oracle(sw):
    """Groups whose second singular value lies below s_crit: the oracle's X^ equals
    coef y (y^T Y) with y = Y v_1, coef = s_1' / (s_1 ||y||^2), s_1' the shrunk value."""
    rng = np.random.default_rng(int(sw * 100))
    d = K = 64
    C = 2 * math.sqrt(K)
    sc2 = s_crit2(sw, K, C)
    checked = 0
    for _ in range(30):
        Y = _near_rank1(rng, d, K, 0.005)
        X, r, s, s_new = O.wnnm(Y, sw, C, eps=1e-30)
        if s[1] ** 2 >= sc2:
            continue
        _, _, Vt = np.linalg.svd(Y)
        y = Y @ Vt[0]
        coef = s_new[0] / (s[0] * (y @ y))
        Xr = coef * np.outer(y, y @ Y)
        assert r == (1 if s_new[0] > 0 else 0)
        np.testing.assert_allclose(Xr, X, rtol=0, atol=1e-10 * s[0])
        checked += 1
    assert checked >= 20
