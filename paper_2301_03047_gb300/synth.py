"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module only *makes data*: scenes, masks, noise and the simulated camera
measurement.  It contains none of the reconstruction method's arithmetic
(no edge maps, no matching, no low-rank step, no projection) and imports
neither the oracle nor the CUDA extension.

Scene model (stand-in for the paper's CACTI test videos, which are not
available): float32 frames in [0, 1] made of piecewise-smooth shapes
(ellipses, rectangles, triangles; each a constant plus a small linear ramp)
painted over a band-limited textured background.  Shapes translate by a
per-shape integer velocity of 1-3 px/frame; the background texture drifts by
1 px/frame.  Every frame is rendered analytically (no wrap-around).

Camera (Eq. 6, coded-aperture temporal imaging): Bernoulli(0.5) binary masks
per frame, y = sum_t M_t * x_t + N(0, sigma^2).

Seeds: numpy PCG64 with SeedSequence(20230107 + config_no), spawned into
(scene, masks, noise) streams.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20230107


# ----------------------------------------------------------------------------
# workload descriptions
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class SciConfig:
    """A video snapshot-compressive-imaging workload (Eq. 6)."""

    name: str
    config_no: int
    T: int  # frames summed into one snapshot
    H: int
    W: int
    P: int  # patch side
    N: int  # key patches per frame
    K: int  # matches per key
    iters: int
    noise_sigma: float = 0.01
    sigma_first: float = 0.5
    sigma_last: float = 0.1
    edge_th: float = 0.1

    @property
    def c_wnnm(self) -> float:
        return 2.0 * math.sqrt(self.K)

    def sigma_schedule(self) -> list[float]:
        """Geometric noise-level schedule sigma_w per outer iteration."""
        if self.iters == 1:
            return [self.sigma_last]
        r = (self.sigma_last / self.sigma_first) ** (1.0 / (self.iters - 1))
        return [float(self.sigma_first * r**k) for k in range(self.iters)]


SCI_SMALL = SciConfig("sci_8x128x128_P8_N200_K40", 1, T=8, H=128, W=128, P=8, N=200, K=40, iters=3)
SCI_LARGE = SciConfig("sci_16x512x512_P8_N4096_K64", 2, T=16, H=512, W=512, P=8, N=4096, K=64, iters=20)
SCI_HUGE = SciConfig("sci_24x2048x2048_P8_N16384_K64", 5, T=24, H=2048, W=2048, P=8, N=16384, K=64, iters=20)


def scaled(cfg: SciConfig, *, T=None, H=None, W=None, N=None, K=None, iters=None, name=None) -> SciConfig:
    """A smaller copy of a workload (same scene model, same seed stream)."""
    return SciConfig(
        name or cfg.name + "_scaled",
        cfg.config_no,
        T=T or cfg.T,
        H=H or cfg.H,
        W=W or cfg.W,
        P=cfg.P,
        N=N or cfg.N,
        K=K or cfg.K,
        iters=iters or cfg.iters,
        noise_sigma=cfg.noise_sigma,
        sigma_first=cfg.sigma_first,
        sigma_last=cfg.sigma_last,
        edge_th=cfg.edge_th,
    )


def streams(config_no: int, extra: int = 0):
    """(scene, masks, noise) generators for one workload."""
    ss = np.random.SeedSequence(SEED_BASE + config_no + 1000 * extra)
    a, b, c = ss.spawn(3)
    return np.random.Generator(np.random.PCG64(a)), np.random.Generator(np.random.PCG64(b)), np.random.Generator(np.random.PCG64(c))


# ----------------------------------------------------------------------------
# scene rendering
# ----------------------------------------------------------------------------
def _lowpass_noise(rng: np.random.Generator, h: int, w: int, sigma_px: float) -> np.ndarray:
    """White noise filtered by a Gaussian of std sigma_px (done in the Fourier domain)."""
    n = rng.standard_normal((h, w))
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    g = np.exp(-2.0 * (math.pi**2) * (sigma_px**2) * (fx**2 + fy**2))
    out = np.fft.irfft2(np.fft.rfft2(n) * g, s=(h, w))
    return out / (np.abs(out).max() + 1e-12)


@dataclass
class _Shape:
    kind: int  # 0 ellipse, 1 rectangle, 2 triangle
    cy: float
    cx: float
    a: float  # half extent (rows)
    b: float  # half extent (cols)
    theta: float
    tri: np.ndarray = field(default_factory=lambda: np.zeros((3, 2)))
    base: float = 0.5
    gy: float = 0.0
    gx: float = 0.0
    vy: int = 0
    vx: int = 0


def _make_shapes(rng: np.random.Generator, H: int, W: int) -> list[_Shape]:
    n = max(1, int(round(12 * math.sqrt(H * W / (128.0 * 128.0)))))
    scale = math.sqrt(H * W) / 128.0
    shapes = []
    for _ in range(n):
        kind = int(rng.integers(0, 3))
        a = float(rng.uniform(6, 22) * scale)
        b = float(rng.uniform(6, 22) * scale)
        cy = float(rng.uniform(0, H))
        cx = float(rng.uniform(0, W))
        theta = float(rng.uniform(0, math.pi))
        tri = rng.uniform(-1, 1, size=(3, 2)) * np.array([a, b])
        base = float(rng.uniform(0.2, 0.8))
        ext = max(a, b)
        g = 0.1 / (2.0 * ext)  # ramp keeps the shape inside base +- 0.1
        gy = float(rng.uniform(-g, g))
        gx = float(rng.uniform(-g, g))
        vy = int(rng.choice([-3, -2, -1, 1, 2, 3]))
        vx = int(rng.choice([-3, -2, -1, 1, 2, 3]))
        shapes.append(_Shape(kind, cy, cx, a, b, theta, tri, base, gy, gx, vy, vx))
    return shapes


def _paint(img: np.ndarray, s: _Shape, t: int) -> None:
    H, W = img.shape
    cy = s.cy + s.vy * t
    cx = s.cx + s.vx * t
    ext = math.hypot(s.a, s.b) + 1
    r0, r1 = max(0, int(cy - ext)), min(H, int(cy + ext) + 1)
    c0, c1 = max(0, int(cx - ext)), min(W, int(cx + ext) + 1)
    if r0 >= r1 or c0 >= c1:
        return
    rr = np.arange(r0, r1, dtype=np.float64)[:, None] + 0.5 - cy
    cc = np.arange(c0, c1, dtype=np.float64)[None, :] + 0.5 - cx
    ct, st = math.cos(s.theta), math.sin(s.theta)
    u = ct * rr + st * cc
    v = -st * rr + ct * cc
    if s.kind == 0:
        m = (u / s.a) ** 2 + (v / s.b) ** 2 <= 1.0
    elif s.kind == 1:
        m = (np.abs(u) <= s.a) & (np.abs(v) <= s.b)
    else:
        p = s.tri
        sgn = []
        for i in range(3):
            (y0, x0), (y1, x1) = p[i], p[(i + 1) % 3]
            sgn.append((x1 - x0) * (u - y0) - (y1 - y0) * (v - x0))
        m = ((sgn[0] >= 0) & (sgn[1] >= 0) & (sgn[2] >= 0)) | ((sgn[0] <= 0) & (sgn[1] <= 0) & (sgn[2] <= 0))
    val = s.base + s.gy * rr + s.gx * cc
    sub = img[r0:r1, c0:c1]
    sub[m] = val[m]


def render_scene(rng: np.random.Generator, T: int, H: int, W: int) -> np.ndarray:
    """T frames [T][H][W] float32 in [0,1] of the moving-shapes scene model."""
    tex = _lowpass_noise(rng, H, W + T + 1, sigma_px=2.0) * 0.08
    bg_base = float(rng.uniform(0.3, 0.7))
    gy, gx = rng.uniform(-0.15, 0.15, size=2) / np.array([H, W])
    rr = np.arange(H)[:, None].astype(np.float64)
    cc = np.arange(W)[None, :].astype(np.float64)
    background = bg_base + gy * (rr - H / 2) + gx * (cc - W / 2)
    shapes = _make_shapes(rng, H, W)
    frames = np.empty((T, H, W), dtype=np.float32)
    for t in range(T):
        img = background + tex[:, t : t + W]
        for s in shapes:
            _paint(img, s, t)
        frames[t] = np.clip(img, 0.0, 1.0)
    return frames


def bernoulli_masks(rng: np.random.Generator, T: int, H: int, W: int, p: float = 0.5) -> np.ndarray:
    return (rng.random((T, H, W)) < p).astype(np.float32)


@dataclass
class SciProblem:
    cfg: SciConfig
    truth: np.ndarray  # [T][H][W] float32
    masks: np.ndarray  # [T][H][W] float32 (0/1)
    y: np.ndarray  # [H][W] float32 measurement


def sci_problem(cfg: SciConfig, extra: int = 0) -> SciProblem:
    """Synthetic snapshot: scene, masks and y = sum_t M_t x_t + noise (Eq. 6 camera)."""
    rs, rm, rn = streams(cfg.config_no, extra)
    truth = render_scene(rs, cfg.T, cfg.H, cfg.W)
    masks = bernoulli_masks(rm, cfg.T, cfg.H, cfg.W)
    y = (masks.astype(np.float64) * truth).sum(0) + rn.standard_normal((cfg.H, cfg.W)) * cfg.noise_sigma
    return SciProblem(cfg, truth, masks, y.astype(np.float32))


# ----------------------------------------------------------------------------
# small generic helpers for tests
# ----------------------------------------------------------------------------
def rng_for(tag: str, salt: int = 0) -> np.random.Generator:
    """A deterministic generator for a named test case."""
    h = 0
    for ch in tag:
        h = (h * 131 + ord(ch)) % (2**31)
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, h, salt])))


def quantize8(x: np.ndarray) -> np.ndarray:
    """Round to multiples of 1/256 (an 8-bit image); keeps small sums exact in float32."""
    return (np.round(np.asarray(x, dtype=np.float64) * 256.0) / 256.0).astype(np.float32)


def textured_frames(rng: np.random.Generator, F: int, H: int, W: int) -> np.ndarray:
    """F independent frames [F][H][W] of the scene model (no motion coupling)."""
    out = np.empty((F, H, W), dtype=np.float32)
    for f in range(F):
        out[f] = render_scene(rng, 1, H, W)[0]
    return out


# ----------------------------------------------------------------------------
# MRI: complex images, Cartesian variable-density k-space sampling (Section 3, MRI)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class MriConfig:
    """A Fourier-domain compressive-imaging workload y = M F(x) (the paper's MRI model)."""

    name: str
    config_no: int
    H: int
    W: int
    P: int  # patch side (complex patches: d = 2 P^2 real values)
    N: int  # key patches
    K: int  # matches per key
    iters: int  # ADMM iterations
    line_frac: float = 0.2  # fraction of k-space rows sampled
    centre_lines: int = 32  # fully sampled low-frequency rows
    noise_sigma: float = 0.005  # std of the real and of the imaginary part of the k-space noise
    rho: float = 0.5  # ADMM penalty
    sigma_first: float = 0.5
    sigma_last: float = 0.02
    edge_th: float = 0.1

    @property
    def c_wnnm(self) -> float:
        return 2.0 * math.sqrt(self.K)

    def sigma_schedule(self) -> list[float]:
        if self.iters == 1:
            return [self.sigma_last]
        r = (self.sigma_last / self.sigma_first) ** (1.0 / (self.iters - 1))
        return [float(self.sigma_first * r**k) for k in range(self.iters)]


MRI_SMALL = MriConfig("mri_96x96_P6_N128_K24", 3, H=96, W=96, P=6, N=128, K=24, iters=3, centre_lines=8)
MRI_LARGE = MriConfig("mri_1024x1024_P6_N8192_K48", 3, H=1024, W=1024, P=6, N=8192, K=48, iters=30)


def mri_scaled(cfg: MriConfig, *, H=None, W=None, N=None, K=None, iters=None, centre_lines=None, name=None) -> MriConfig:
    return MriConfig(
        name or cfg.name + "_scaled", cfg.config_no, H=H or cfg.H, W=W or cfg.W, P=cfg.P, N=N or cfg.N,
        K=K or cfg.K, iters=iters or cfg.iters, line_frac=cfg.line_frac,
        centre_lines=centre_lines or cfg.centre_lines, noise_sigma=cfg.noise_sigma, rho=cfg.rho,
        sigma_first=cfg.sigma_first, sigma_last=cfg.sigma_last, edge_th=cfg.edge_th)


def complex_phantom(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    """Complex image [2][H][W] (real plane, imaginary plane), float32.

    Magnitude: 12-20 random ellipses whose intensities add (each in [0.1, 0.5])
    over band-limited texture of amplitude 0.03, clipped to [0, 1]; phase: a
    random quadratic polynomial of the normalised coordinates (|coefficients|
    <= pi/4)."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = 2.0 * xx / max(W - 1, 1) - 1.0
    v = 2.0 * yy / max(H - 1, 1) - 1.0
    mag = np.zeros((H, W))
    for _ in range(int(rng.integers(12, 21))):
        cx, cy = rng.uniform(-0.7, 0.7, 2)
        ax, ay = rng.uniform(0.08, 0.5, 2)
        th = rng.uniform(0, math.pi)
        ct, st = math.cos(th), math.sin(th)
        xr = (u - cx) * ct + (v - cy) * st
        yr = -(u - cx) * st + (v - cy) * ct
        mag[(xr / ax) ** 2 + (yr / ay) ** 2 <= 1.0] += rng.uniform(0.1, 0.5)
    tex = _lowpass_noise(rng, H, W, 2.0)
    tex = tex / max(np.abs(tex).max(), 1e-12) * 0.03
    mag = np.clip(mag + tex, 0.0, 1.0)
    c = rng.uniform(-math.pi / 4, math.pi / 4, 6)
    phase = c[0] + c[1] * u + c[2] * v + c[3] * u * u + c[4] * u * v + c[5] * v * v
    return np.stack([mag * np.cos(phase), mag * np.sin(phase)]).astype(np.float32)


def cartesian_mask(rng: np.random.Generator, H: int, W: int, frac: float, centre: int) -> np.ndarray:
    """0/1 k-space mask [H][W] (float32) of whole rows, in the unshifted FFT layout
    (row k holds frequency k for k < H/2 and k - H otherwise).  The `centre`
    lowest frequencies are always taken; the other rows are drawn without
    replacement with probability proportional to (1 - |k| / (H/2))^2 until
    round(frac * H) rows are chosen."""
    freq = np.where(np.arange(H) < H // 2, np.arange(H), np.arange(H) - H)
    chosen = np.abs(freq + 0.5) < centre / 2.0
    n_more = max(int(round(frac * H)) - int(chosen.sum()), 0)
    pdf = (1.0 - np.abs(freq) / (H / 2.0)) ** 2
    pdf[chosen] = 0.0
    pdf /= pdf.sum()
    pick = rng.choice(H, size=n_more, replace=False, p=pdf)
    chosen[pick] = True
    return np.repeat(chosen[:, None], W, axis=1).astype(np.float32)


@dataclass
class MriProblem:
    cfg: MriConfig
    truth: np.ndarray  # [2][H][W] float32 (real, imaginary planes)
    mask: np.ndarray  # [H][W] float32 (0/1)
    y: np.ndarray  # [2][H][W] float32 k-space measurement (zero off the mask)


def mri_problem(cfg: MriConfig, extra: int = 0) -> MriProblem:
    """Synthetic scan: y = M (F x + n), F the orthonormal 2-D DFT (unshifted),
    n complex Gaussian with std noise_sigma per real component (the MRI model
    of Section 3)."""
    rs, rm, rn = streams(cfg.config_no, extra)
    truth = complex_phantom(rs, cfg.H, cfg.W)
    mask = cartesian_mask(rm, cfg.H, cfg.W, cfg.line_frac, cfg.centre_lines)
    k = np.fft.fft2(truth[0].astype(np.float64) + 1j * truth[1].astype(np.float64), norm="ortho")
    k = k + cfg.noise_sigma * (rn.standard_normal(k.shape) + 1j * rn.standard_normal(k.shape))
    k = k * mask
    return MriProblem(cfg, truth, mask, np.stack([k.real, k.imag]).astype(np.float32))


# ----------------------------------------------------------------------------
# MSFA: multispectral filter-array demosaicing, uneven image sizes (Section 3, MSFA)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class MsfaConfig:
    """A batch of MSFA snapshots y = sum_b A_b x_b (Eq. 8) of uneven sizes."""

    name: str
    config_no: int
    sides: tuple  # image side of every image of the batch (square images)
    bands: int
    P: int
    K: int
    iters: int
    N_fixed: int = 0  # 0: N = min(8192, 1024 (side / 256)^2) per image
    sigma_first: float = 0.1
    sigma_last: float = 0.02
    edge_th: float = 0.1

    @property
    def c_wnnm(self) -> float:
        return 2.0 * math.sqrt(self.K)

    def N_of(self, side: int) -> int:
        if self.N_fixed:
            return self.N_fixed
        return int(min(8192, 1024 * (side / 256.0) ** 2))

    def sigma_schedule(self) -> list[float]:
        if self.iters == 1:
            return [self.sigma_last]
        r = (self.sigma_last / self.sigma_first) ** (1.0 / (self.iters - 1))
        return [float(self.sigma_first * r**k) for k in range(self.iters)]


def msfa_sides(n: int, seed_no: int = 4, choices=(256, 384, 512, 768, 1024)) -> tuple:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE + seed_no, 77])))
    return tuple(int(v) for v in rng.choice(np.asarray(choices), size=n))


MSFA_SMALL = MsfaConfig("msfa_3img_40-64_16band_P6_N48_K16", 4, sides=(40, 56, 64), bands=16, P=6, K=16, iters=2,
                        N_fixed=48)
MSFA_LARGE = MsfaConfig("msfa_32img_256-1024_16band_P6_K32", 4, sides=msfa_sides(32), bands=16, P=6, K=32, iters=10)


def mosaic_masks(H: int, W: int, bands: int = 16) -> np.ndarray:
    """Periodic square mosaic [bands][H][W] (0/1): pixel (r, c) sees band s*(r mod s) + (c mod s), s = sqrt(bands)."""
    s = int(round(math.sqrt(bands)))
    assert s * s == bands
    r = np.arange(H)[:, None] % s
    c = np.arange(W)[None, :] % s
    band = s * r + c
    return (band[None] == np.arange(bands)[:, None, None]).astype(np.float32)


def spectral_cube(rng: np.random.Generator, bands: int, H: int, W: int, materials: int = 6) -> np.ndarray:
    """Multispectral image [bands][H][W] in [0, 1]: `materials` spectra (each a sum of 4
    Gaussians over the band index, peak-normalised) mixed by abundance maps drawn from
    the scene model (independent textured frames, normalised to sum 1 per pixel),
    times a shading map from the scene model."""
    b = np.arange(bands, dtype=np.float64)
    spectra = np.zeros((materials, bands))
    for m in range(materials):
        for _ in range(4):
            spectra[m] += rng.uniform(0.2, 1.0) * np.exp(-0.5 * ((b - rng.uniform(0, bands - 1)) / rng.uniform(1.0, 4.0)) ** 2)
        spectra[m] /= spectra[m].max()
    ab = textured_frames(rng, materials, H, W).astype(np.float64) ** 3 + 1e-3
    ab /= ab.sum(0, keepdims=True)
    shade = 0.4 + 0.6 * textured_frames(rng, 1, H, W)[0].astype(np.float64)
    cube = np.einsum("mhw,mb->bhw", ab, spectra) * shade[None]
    return np.clip(cube, 0.0, 1.0).astype(np.float32)


@dataclass
class MsfaImage:
    truth: np.ndarray  # [bands][H][W]
    masks: np.ndarray  # [bands][H][W]
    y: np.ndarray  # [H][W]
    N: int


def msfa_problem(cfg: MsfaConfig, extra: int = 0) -> list:
    """Noiseless mosaic snapshots y = sum_b A_b x_b, one per image of the batch."""
    rs, _, _ = streams(cfg.config_no, extra)
    out = []
    for side in cfg.sides:
        truth = spectral_cube(rs, cfg.bands, side, side)
        masks = mosaic_masks(side, side, cfg.bands)
        y = (masks.astype(np.float64) * truth).sum(0).astype(np.float32)
        out.append(MsfaImage(truth, masks, y, cfg.N_of(side)))
    return out
