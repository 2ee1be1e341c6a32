"""Seeded synthetic frame pairs with the shapes of the method's workloads.

This module makes inputs only: images, ground-truth flows, gain fields and the
solver parameters a workload is run with.  It holds none of the solver's
arithmetic (no gradients, no element coefficients, no operator), so both the
CUDA path and the FP64 oracle can be fed from it.

Workloads (the datasets of the paper's experiments, Middlebury RubberWhale and
the Cerema HD sequences of Section 4, are not available; these stand in for
them with the same sizes and the same kinds of structure):

* ``blobs``     -- 64x48 float64, 40 Gaussian blobs, translated by (1.5,-0.75)
                   px (bicubic) with gain 1.1 and offset 0.02, alpha = 0.05.
* ``texture``   -- 640x480 float32 band-limited 1/f^2 noise, rotated 2 degrees
                   about the centre and translated by (3,1) px, gain ramp
                   0.9..1.2 across x (RubberWhale scale, Section 4).
* ``layers``    -- WxH (3840x2160 by default) float32: 4 textured layers (a
                   background and 3 random polygons) in painter's order with
                   distinct rigid translations up to 6 px, smooth random
                   degree-2 gain in [0.8, 1.25] (Cerema HD stand-in).
* ``batch``     -- 64 ``layers`` pairs with sizes drawn from 320x240,
                   640x480, 1280x720 and 1920x1080.
* ``smooth``    -- 8 pairs 512x512 with a smooth ground-truth flow (Gaussian
                   filtered noise, sigma 32 px, max 4 px) and gain 1.1.

Every generator is deterministic in its seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1508

# Solver parameters that the paper leaves open (Sections 1 and 2.3); the
# values are the ones every workload here is run with.
ALPHA0 = 0.05       # initial regularisation alpha (constant field)
LAMBDA = 1.0        # regularisation of the illumination field m
KAPPA = 4.0         # alpha-update control parameter kappa
ETA_THR = 0.25      # alpha-update threshold on eta_K / max eta
ALPHA_TH_FRAC = 1e-2  # alpha_th = ALPHA_TH_FRAC * ALPHA0


@dataclass
class Pair:
    """One frame pair and what is known about it."""
    f1: np.ndarray                      # [H][W]
    f2: np.ndarray                      # [H][W]
    alpha0: float = ALPHA0
    lam: float = LAMBDA
    flow_gt: np.ndarray | None = None   # [2][H][W] (u1 along x, u2 along y)
    gain_gt: np.ndarray | None = None   # [H][W]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def H(self) -> int:
        return int(self.f1.shape[0])

    @property
    def W(self) -> int:
        return int(self.f1.shape[1])


# ---------------------------------------------------------------- sampling --

def _keys(s: np.ndarray, a: float = -0.5) -> np.ndarray:
    """Keys' cubic convolution kernel (Keys 1981) with parameter a."""
    s = np.abs(s)
    out = np.zeros_like(s)
    m1 = s <= 1.0
    m2 = (s > 1.0) & (s < 2.0)
    out[m1] = (a + 2.0) * s[m1] ** 3 - (a + 3.0) * s[m1] ** 2 + 1.0
    out[m2] = a * s[m2] ** 3 - 5.0 * a * s[m2] ** 2 + 8.0 * a * s[m2] - 4.0 * a
    return out


def sample_bicubic(img: np.ndarray, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """Samples img (float64 [H][W], pixel centres at integer coordinates) at
    real positions (xs, ys) by Keys bicubic interpolation, edges clamped."""
    H, W = img.shape
    x0 = np.floor(xs).astype(np.int64)
    y0 = np.floor(ys).astype(np.int64)
    tx = xs - x0
    ty = ys - y0
    out = np.zeros(xs.shape, dtype=np.float64)
    for j in range(-1, 3):
        wy = _keys(ty - j)
        yy = np.clip(y0 + j, 0, H - 1)
        row = np.zeros(xs.shape, dtype=np.float64)
        for i in range(-1, 3):
            wx = _keys(tx - i)
            xx = np.clip(x0 + i, 0, W - 1)
            row += wx * img[yy, xx]
        out += wy * row
    return out


def band_limited_noise(W: int, H: int, rng: np.random.Generator,
                       cut: float = 0.25, spectrum: bool = False):
    """White noise shaped to amplitude ~ 1/|f| (power ~ 1/f^2), DC removed,
    zero above ``cut`` cycles/px, min-max normalised to [0, 1].

    With ``spectrum=True`` also returns (F, lo, hi) so that exact sub-pixel
    translates of the same texture can be made by a Fourier phase shift."""
    white = rng.standard_normal((H, W))
    F = np.fft.rfft2(white)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    fr = np.sqrt(fx * fx + fy * fy)
    shape = np.zeros_like(fr)
    keep = (fr > 0) & (fr <= cut)
    shape[keep] = 1.0 / fr[keep]
    F = F * shape
    img = np.fft.irfft2(F, s=(H, W))
    lo, hi = float(img.min()), float(img.max())
    out = (img - lo) / (hi - lo)
    if spectrum:
        return out, (F, lo, hi)
    return out


def translated_texture(spec, W: int, H: int, vx: float, vy: float) -> np.ndarray:
    """The texture of ``spec`` moved by (vx, vy): out(y) = tex(y - v), exact
    for the band-limited (periodic) texture."""
    F, lo, hi = spec
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    ph = np.exp(-2j * np.pi * (fx * vx + fy * vy))
    img = np.fft.irfft2(F * ph, s=(H, W))
    return (img - lo) / (hi - lo)


def _polygon_mask(px: np.ndarray, py: np.ndarray, vx: np.ndarray, vy: np.ndarray) -> np.ndarray:
    """Even-odd point-in-polygon test of points (px, py) against the polygon
    with vertices (vx, vy)."""
    inside = np.zeros(px.shape, dtype=bool)
    n = len(vx)
    for k in range(n):
        x1, y1 = vx[k], vy[k]
        x2, y2 = vx[(k + 1) % n], vy[(k + 1) % n]
        if y1 == y2:
            continue
        cond = (y1 > py) != (y2 > py)
        xcross = x1 + (py - y1) * (x2 - x1) / (y2 - y1)
        inside ^= cond & (px < xcross)
    return inside


def _gaussian_filter_periodic(a: np.ndarray, sigma: float) -> np.ndarray:
    H, W = a.shape
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (fx * fx + fy * fy))
    return np.fft.irfft2(np.fft.rfft2(a) * g, s=(H, W))


# --------------------------------------------------------------- workloads --

def blobs(W: int = 64, H: int = 48, seed: int = BASE_SEED + 1, nblobs: int = 40,
          shift=(1.5, -0.75), gain: float = 1.1, offset: float = 0.02) -> Pair:
    """Sum of Gaussian blobs; frame 2 = gain * frame1(x - d) + offset."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, W, nblobs)
    cy = rng.uniform(0, H, nblobs)
    sg = rng.uniform(2.0, 6.0, nblobs)
    am = rng.uniform(0.0, 1.0, nblobs)
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    f1 = np.zeros((H, W))
    for k in range(nblobs):
        f1 += am[k] * np.exp(-((X - cx[k]) ** 2 + (Y - cy[k]) ** 2) / (2.0 * sg[k] ** 2))
    f2 = gain * sample_bicubic(f1, X - shift[0], Y - shift[1]) + offset
    flow = np.stack([np.full((H, W), shift[0]), np.full((H, W), shift[1])])
    return Pair(f1=f1, f2=f2, flow_gt=flow, gain_gt=np.full((H, W), gain),
                name=f"blobs_{W}x{H}", meta=dict(seed=seed, dtype="f64"))


def texture(W: int = 640, H: int = 480, seed: int = BASE_SEED + 2,
            angle_deg: float = 2.0, shift=(3.0, 1.0), g0: float = 0.9,
            g1: float = 1.2) -> Pair:
    """Band-limited texture under rotation about the centre + translation,
    with a multiplicative gain ramp g0..g1 across x."""
    rng = np.random.default_rng(seed)
    tex = band_limited_noise(W, H, rng)
    cxc, cyc = (W - 1) / 2.0, (H - 1) / 2.0
    th = math.radians(angle_deg)
    c, s = math.cos(th), math.sin(th)
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    # forward map T(x) = R (x - c) + c + t ; flow = T(x) - x
    Tx = c * (X - cxc) - s * (Y - cyc) + cxc + shift[0]
    Ty = s * (X - cxc) + c * (Y - cyc) + cyc + shift[1]
    # inverse map for sampling frame 2 at its grid points
    dx, dy = X - cxc - shift[0], Y - cyc - shift[1]
    Sx = c * dx + s * dy + cxc
    Sy = -s * dx + c * dy + cyc
    gain_src = g0 + (g1 - g0) * Sx / (W - 1)
    f2 = gain_src * sample_bicubic(tex, Sx, Sy)
    flow = np.stack([Tx - X, Ty - Y])
    gain = g0 + (g1 - g0) * X / (W - 1)
    return Pair(f1=tex.astype(np.float32), f2=f2.astype(np.float32), flow_gt=flow,
                gain_gt=gain, name=f"texture_{W}x{H}", meta=dict(seed=seed, dtype="f32"))


def layers(W: int = 3840, H: int = 2160, seed: int = BASE_SEED + 3, nlayers: int = 4,
           vmax: float = 6.0, gmin: float = 0.8, gmax: float = 1.25) -> Pair:
    """Background + (nlayers-1) random polygons, each with its own band-limited
    texture and rigid translation, painter's order, smooth degree-2 gain."""
    rng = np.random.default_rng(seed)
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    f1 = np.zeros((H, W))
    f2 = np.zeros((H, W))
    flow = np.zeros((2, H, W))
    for k in range(nlayers):
        _, spec = band_limited_noise(W, H, rng, spectrum=True)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        mag = rng.uniform(1.0, vmax)
        vx, vy = mag * math.cos(ang), mag * math.sin(ang)
        t1 = translated_texture(spec, W, H, 0.0, 0.0)
        t2 = translated_texture(spec, W, H, vx, vy)
        if k == 0:
            m1 = np.ones((H, W), dtype=bool)
            m2 = m1
        else:
            nv = int(rng.integers(5, 9))
            pcx, pcy = rng.uniform(0.15 * W, 0.85 * W), rng.uniform(0.15 * H, 0.85 * H)
            rad = rng.uniform(0.12, 0.3) * min(W, H)
            angs = np.sort(rng.uniform(0.0, 2.0 * math.pi, nv))
            rr = rad * rng.uniform(0.6, 1.0, nv)
            pvx = pcx + rr * np.cos(angs)
            pvy = pcy + rr * np.sin(angs)
            m1 = _polygon_mask(X, Y, pvx, pvy)
            m2 = _polygon_mask(X - vx, Y - vy, pvx, pvy)
        f1[m1] = t1[m1]
        f2[m2] = t2[m2]
        flow[0][m1] = vx
        flow[1][m1] = vy
    c = rng.uniform(-1.0, 1.0, 6)
    xn, yn = X / max(W - 1, 1), Y / max(H - 1, 1)
    poly = c[0] + c[1] * xn + c[2] * yn + c[3] * xn * xn + c[4] * xn * yn + c[5] * yn * yn
    lo, hi = float(poly.min()), float(poly.max())
    gain = gmin + (gmax - gmin) * (poly - lo) / (hi - lo if hi > lo else 1.0)
    f2 = gain * f2
    return Pair(f1=f1.astype(np.float32), f2=f2.astype(np.float32), flow_gt=flow,
                gain_gt=gain, name=f"layers_{W}x{H}", meta=dict(seed=seed, dtype="f32"))


BATCH_SIZES = ((320, 240), (640, 480), (1280, 720), (1920, 1080))


def batch_sizes(npairs: int = 64, seed: int = BASE_SEED + 4, weights=(0.25, 0.25, 0.25, 0.25)):
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(BATCH_SIZES), size=npairs, p=np.asarray(weights) / np.sum(weights))
    return [BATCH_SIZES[i] for i in idx]


def batch(npairs: int = 64, seed: int = BASE_SEED + 4) -> list[Pair]:
    """Mixed-size batch of layered pairs (sizes from a seeded categorical)."""
    sizes = batch_sizes(npairs, seed)
    return [layers(W, H, seed=seed * 1000 + i) for i, (W, H) in enumerate(sizes)]


def smooth(W: int = 512, H: int = 512, npairs: int = 8, seed: int = BASE_SEED + 5,
           sigma: float = 32.0, umax: float = 4.0, gain: float = 1.1) -> list[Pair]:
    """Pairs with a smooth known flow: f2(x) = gain * f1(x - u(x))."""
    rng = np.random.default_rng(seed)
    out = []
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    for i in range(npairs):
        tex = band_limited_noise(W, H, rng)
        u = np.stack([_gaussian_filter_periodic(rng.standard_normal((H, W)), sigma)
                      for _ in range(2)])
        mag = np.sqrt(u[0] ** 2 + u[1] ** 2).max()
        u *= umax / mag
        f2 = gain * sample_bicubic(tex, X - u[0], Y - u[1])
        out.append(Pair(f1=tex.astype(np.float32), f2=f2.astype(np.float32), flow_gt=u,
                        gain_gt=np.full((H, W), gain), name=f"smooth_{W}x{H}_{i}",
                        meta=dict(seed=seed, dtype="f32")))
    return out


def random_alpha(W: int, H: int, seed: int, lo: float = 0.01, hi: float = 0.1) -> np.ndarray:
    """A random positive per-element alpha field [H-1][W-1][2] for tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(H - 1, W - 1, 2))


def random_frames(W: int, H: int, seed: int):
    """Two independent uniform random frames (non-degenerate data everywhere)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (H, W)), rng.uniform(0.0, 1.0, (H, W))
