"""Pins of the FP64 encoder oracle (learned proposal) against independent facts."""
import numpy as np

from oracle import encoder_oracle as E
from paper_2301_03047_gb300 import synth


def _data(tag, n=24):
    rng = synth.rng_for(tag)
    Pm = rng.standard_normal((n, 64)) * 0.3
    Qm = Pm + rng.standard_normal((n, 64)) * 0.1
    d = ((Pm - Qm) ** 2).sum(1)
    return rng, Pm, Qm, d


def test_gradient_matches_central_differences():
    rng, Pm, Qm, d = _data("enc-fd")
    params = E.init_params(rng)
    g = E.pair_loss_grad(params, Pm, Qm, d)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2"):
        flat = params[name].reshape(-1)
        for j in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + h
            lp = E.pair_loss(params, Pm, Qm, d)
            flat[j] = old - h
            lm = E.pair_loss(params, Pm, Qm, d)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (name, j)


def test_linear_regime_closed_form():
    """W1 = I with a large bias keeps every ReLU open; W2 = [I_16 0], b2 = -b1[:16]: f(p) = p[:16]."""
    _, Pm, Qm, _ = _data("enc-lin")
    params = {"W1": np.eye(64), "b1": np.full(64, 10.0), "W2": np.hstack([np.eye(16), np.zeros((16, 48))]),
              "b2": np.full(16, -10.0)}
    Ep, _ = E.forward(params, Pm)
    assert np.allclose(Ep, Pm[:, :16])
    Eq, _ = E.forward(params, Qm)
    assert np.allclose(((Ep - Eq) ** 2).sum(1), ((Pm[:, :16] - Qm[:, :16]) ** 2).sum(1))


def test_perfect_fit_has_zero_loss_and_gradient():
    rng, Pm, Qm, _ = _data("enc-zero")
    params = E.init_params(rng)
    Ep, _ = E.forward(params, Pm)
    Eq, _ = E.forward(params, Qm)
    d = ((Ep - Eq) ** 2).sum(1)
    assert E.pair_loss(params, Pm, Qm, d) < 1e-28
    g = E.pair_loss_grad(params, Pm, Qm, d)
    assert all(np.abs(v).max() < 1e-12 for v in g.values())


def test_adamw_first_step_closed_form():
    """t = 1: bias-corrected moments are g and g^2, so the step is -lr g/(|g|+eps) - lr wd p (weights only)."""
    rng = synth.rng_for("adamw")
    params = {"W1": rng.standard_normal((3, 2)), "b1": rng.standard_normal(3)}
    grads = {"W1": rng.standard_normal((3, 2)), "b1": rng.standard_normal(3)}
    zeros = {k: np.zeros_like(v) for k, v in params.items()}
    lr, wd, eps = 1e-2, 0.1, 1e-8
    p1, m1, v1 = E.adamw_step(params, grads, zeros, zeros, 1, lr=lr, wd=wd, eps=eps)
    want_W = params["W1"] - lr * wd * params["W1"] - lr * grads["W1"] / (np.abs(grads["W1"]) + eps)
    want_b = params["b1"] - lr * grads["b1"] / (np.abs(grads["b1"]) + eps)
    assert np.allclose(p1["W1"], want_W) and np.allclose(p1["b1"], want_b)
    assert np.allclose(m1["W1"], 0.1 * grads["W1"]) and np.allclose(v1["b1"], 0.001 * grads["b1"] ** 2)


# ---- E4M3 rounding of the 8-bit proposal operands (pinned to the format's definition)
def _codes_positive():
    return [c for c in range(0x00, 0x7F)]  # 0x7F is NaN


def test_e4m3_every_finite_code_rounds_to_itself():
    vals = np.array([E.e4m3_decode(c) for c in _codes_positive()] + [E.e4m3_decode(0x80 | c) for c in _codes_positive()])
    np.testing.assert_array_equal(E.e4m3_round(vals), vals)
    assert E.e4m3_decode(0x7E) == 448.0 and E.e4m3_decode(0x01) == 2.0**-9 and E.e4m3_decode(0x38) == 1.0
    assert np.isnan(E.e4m3_decode(0x7F)) and np.isnan(E.e4m3_decode(0xFF))


def test_e4m3_midpoints_round_to_the_even_code():
    codes = _codes_positive()
    vals = [E.e4m3_decode(c) for c in codes]
    for c in range(len(codes) - 1):
        lo, hi = vals[c], vals[c + 1]
        mid = 0.5 * (lo + hi)
        want = lo if codes[c] % 2 == 0 else hi  # the even mantissa (lowest code bit 0)
        assert E.e4m3_round(mid) == want, (codes[c], lo, hi)
        assert E.e4m3_round(-mid) == -want
        # just off the midpoint: the nearer neighbour
        assert E.e4m3_round(mid - 1e-6 * (hi - lo)) == lo
        assert E.e4m3_round(mid + 1e-6 * (hi - lo)) == hi


def test_e4m3_saturates_and_flushes_below_half_the_smallest_subnormal():
    np.testing.assert_array_equal(E.e4m3_round([448.0, 464.0, 1e6, -1e6]), [448.0, 448.0, 448.0, -448.0])
    np.testing.assert_array_equal(E.e4m3_round([2.0**-11, -(2.0**-11)]), [0.0, 0.0])


def test_e4m3_scale_is_the_largest_fitting_power_of_two():
    rng = np.random.default_rng(5)
    for n2 in np.exp(rng.uniform(-10, 12, 200)):
        s = E.e4m3_scale(n2)
        assert np.log2(s) == np.round(np.log2(s))
        assert s * s * n2 <= 384.0 < 4 * s * s * n2
