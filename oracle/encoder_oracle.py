"""FP64 oracle of the learned matching proposal (patch encoder and its training loss).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the library never imports it.

The proposal replaces the exhaustive contraction over d = 64 patch values by
one over a 16-dimensional embedding f(p):

  f(p) = W2 relu(W1 p + b1) + b2,     W1: 64 x 64, W2: 16 x 64 (rows = outputs)

trained so that ||f(p) - f(q)||^2 matches the exact squared patch distance
d(p, q) = ||p - q||^2 on pairs the method itself produced (a key and its
exact nearest matches, plus random positions):

  L = (1/n) sum_i w_i (||f(p_i) - f(q_i)||^2 - d_i)^2,   w_i = 1 / (d_i + d0)^2

(relative squared error, so near pairs dominate; d0 = 0.05).  The optimiser is
AdamW (decoupled weight decay on W1 and W2, not on the biases).  Patches are
mean-shifted exactly as for the exhaustive matcher.  The paper has no such
component (its Outlook mentions low-rank networks); this follows the
project's description of the learned proposal.
"""
from __future__ import annotations

import numpy as np

D0 = 0.05


def init_params(rng: np.random.Generator, d_in: int = 64, d_hid: int = 64, d_out: int = 16) -> dict:
    """He-style initialisation; the biases start at zero."""
    return {
        "W1": rng.standard_normal((d_hid, d_in)) * np.sqrt(2.0 / d_in),
        "b1": np.zeros(d_hid),
        "W2": rng.standard_normal((d_out, d_hid)) * np.sqrt(1.0 / d_hid),
        "b2": np.zeros(d_out),
    }


def forward(params: dict, X: np.ndarray):
    """Embeddings of the rows of X [n][64]; returns (E [n][16], hidden pre-activation Z [n][64])."""
    Z = X @ params["W1"].T + params["b1"]
    H = np.maximum(Z, 0.0)
    return H @ params["W2"].T + params["b2"], Z


def pair_loss(params: dict, Pm: np.ndarray, Qm: np.ndarray, d: np.ndarray) -> float:
    Ep, _ = forward(params, Pm)
    Eq, _ = forward(params, Qm)
    s = ((Ep - Eq) ** 2).sum(1)
    w = 1.0 / (d + D0) ** 2
    return float(np.mean(w * (s - d) ** 2))


def pair_loss_grad(params: dict, Pm: np.ndarray, Qm: np.ndarray, d: np.ndarray):
    """Analytic gradient of pair_loss (backward pass written out by hand)."""
    n = Pm.shape[0]
    Ep, Zp = forward(params, Pm)
    Eq, Zq = forward(params, Qm)
    diff = Ep - Eq
    s = (diff * diff).sum(1)
    w = 1.0 / (d + D0) ** 2
    r = w * (s - d)  # dL/ds * n / 2
    gE = (4.0 / n) * r[:, None] * diff  # dL/dEp ; dL/dEq = -gE
    grads = {k: np.zeros_like(v) for k, v in params.items()}
    for sign, Z, X in ((1.0, Zp, Pm), (-1.0, Zq, Qm)):
        g_out = sign * gE
        H = np.maximum(Z, 0.0)
        grads["W2"] += g_out.T @ H
        grads["b2"] += g_out.sum(0)
        g_h = (g_out @ params["W2"]) * (Z > 0)
        grads["W1"] += g_h.T @ X
        grads["b1"] += g_h.sum(0)
    return grads


def adamw_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW update (bias-corrected moments; decay on the weight matrices only)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        g = grads[k]
        m_k = b1 * m[k] + (1 - b1) * g
        v_k = b2 * v[k] + (1 - b2) * g * g
        mh = m_k / (1 - b1**t)
        vh = v_k / (1 - b2**t)
        p = params[k]
        if k.startswith("W"):
            p = p - lr * wd * p
        out_p[k] = p - lr * mh / (np.sqrt(vh) + eps)
        out_m[k], out_v[k] = m_k, v_k
    return out_p, out_m, out_v


# ---------------------------------------------------------------------------
# 8-bit proposal operands: FP8 E4M3 rounding (the OCP 8-bit floating-point
# format's E4M3 encoding: 1 sign bit, 4 exponent bits with bias 7, 3 mantissa
# bits, no infinities, largest finite magnitude 1.75 x 2^8 = 448, normals down
# to 2^-6, subnormals m x 2^-9 for m = 1..7), written from that definition.
# ---------------------------------------------------------------------------
E4M3_MAX = 448.0


def e4m3_round(x) -> np.ndarray:
    """Round to the nearest E4M3 value, ties to even, saturating at +-448 (FP64 in and out)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6, 8)  # below 2^-6 the spacing stays at the subnormal 2^-9
    quantum = np.exp2(e - 3)
    q = np.round(a / quantum) * quantum  # numpy rounds halves to even
    q = np.minimum(q, E4M3_MAX)
    return np.where(x < 0, -q, q)


def e4m3_decode(code: int) -> float:
    """Value of an E4M3 byte (NaN for the two NaN codes)."""
    s = -1.0 if code & 0x80 else 1.0
    ex = (code >> 3) & 0xF
    m = code & 0x7
    if ex == 0xF and m == 0x7:
        return float("nan")
    if ex == 0:
        return s * m * 2.0**-9
    return s * (1.0 + m / 8.0) * 2.0 ** (ex - 7)


def e4m3_scale(n2max: float, target: float = 384.0) -> float:
    """The proposal's per-call scale: the largest power of two s with s^2 n2max <= target."""
    if not n2max > 0:
        return 1.0
    return float(2.0 ** np.floor(np.log2(np.sqrt(target / n2max))))
