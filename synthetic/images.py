"""Seeded synthetic images, video GOPs and request streams.

The paper evaluates on Kodak (768x512), UVG (1920x1080, GOP 8) and JPEG-XL
test images (Section 4). None of those are available here, so these
generators produce images with the same sizes and broadly similar structure
(smooth regions, edges, 1/f texture, global motion). Every generator takes an
explicit seed and uses numpy's PCG64 through ``default_rng``.
"""
from __future__ import annotations

import numpy as np


def gray_sinusoids(h: int = 256, w: int = 256, seed: int = 0) -> np.ndarray:
    """Grayscale uint8 image: 128 + sum of 8 random 2-D sinusoids + N(0, 8^2).

    Amplitudes ~ U(5, 20), spatial frequencies (u, v) ~ U(-8, 8) cycles per
    256 samples, phases ~ U(0, 2 pi); the sum is rounded and clipped to
    [0, 255]. Returns an (h, w) array.
    """
    rng = np.random.default_rng(seed)
    a = rng.uniform(5.0, 20.0, 8)
    u = rng.uniform(-8.0, 8.0, 8)
    v = rng.uniform(-8.0, 8.0, 8)
    ph = rng.uniform(0.0, 2.0 * np.pi, 8)
    ii, jj = np.meshgrid(np.arange(h, dtype=np.float64),
                         np.arange(w, dtype=np.float64), indexing="ij")
    x = np.full((h, w), 128.0)
    for k in range(8):
        x += a[k] * np.sin(2.0 * np.pi * (u[k] * ii + v[k] * jj) / 256.0 + ph[k])
    x += rng.normal(0.0, 8.0, (h, w))
    return np.clip(np.round(x), 0, 255).astype(np.uint8)


def _one_over_f(rng: np.random.Generator, h: int, w: int, std: float) -> np.ndarray:
    """White Gaussian noise shaped by 1/|f| in the 2-D FFT, scaled to `std`."""
    n = rng.normal(0.0, 1.0, (h, w))
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    f[0, 0] = 1.0
    spec = np.fft.rfft2(n) / f
    spec[0, 0] = 0.0
    t = np.fft.irfft2(spec, s=(h, w))
    s = t.std()
    return t * (std / s) if s > 0 else t


def rgb_natural(h: int = 512, w: int = 768, seed: int = 1) -> np.ndarray:
    """RGB uint8 image (h, w, 3): gradient + rectangles + 1/f texture.

    Per channel a linear gradient with a random direction and random end
    values; then 6 to 20 axis-aligned rectangles of random colour; then a
    1/f texture with standard deviation 12 added to all channels.
    """
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(0.0, 1.0, h), np.linspace(0.0, 1.0, w),
                         indexing="ij")
    img = np.empty((h, w, 3))
    for c in range(3):
        ang = rng.uniform(0.0, 2.0 * np.pi)
        t = np.cos(ang) * xx + np.sin(ang) * yy
        t = (t - t.min()) / max(t.max() - t.min(), 1e-9)
        lo, hi = rng.uniform(0.0, 255.0, 2)
        img[:, :, c] = lo + (hi - lo) * t
    for _ in range(int(rng.integers(6, 21))):
        y0 = int(rng.integers(0, h)); x0 = int(rng.integers(0, w))
        rh = int(rng.integers(h // 16 + 1, h // 3 + 2))
        rw = int(rng.integers(w // 16 + 1, w // 3 + 2))
        img[y0:y0 + rh, x0:x0 + rw, :] = rng.uniform(0.0, 255.0, 3)
    tex = _one_over_f(rng, h, w, 12.0)
    img += tex[:, :, None]
    return np.clip(np.round(img), 0, 255).astype(np.uint8)


def video_gop(h: int = 1080, w: int = 1920, nframes: int = 8,
              seed: int = 3) -> np.ndarray:
    """RGB uint8 frames (nframes, h, w, 3): a panned 1/f canvas + sprites.

    A 1/f texture canvas (plus a colour gradient) larger than the frame is
    panned by a random integer global motion in [-4, 4]^2 pixels per frame;
    3 to 6 rectangular sprites of random colour move with their own random
    integer velocities.
    """
    rng = np.random.default_rng(seed)
    pad = 4 * nframes + 8
    ch, cw = h + 2 * pad, w + 2 * pad
    base = rgb_natural(ch, cw, int(rng.integers(0, 2**31))).astype(np.float64)
    base += _one_over_f(rng, ch, cw, 10.0)[:, :, None]
    motion = rng.integers(-4, 5, (nframes, 2))
    nspr = int(rng.integers(3, 7))
    spr = []
    for _ in range(nspr):
        spr.append(dict(y=int(rng.integers(0, h)), x=int(rng.integers(0, w)),
                        hh=int(rng.integers(h // 20 + 2, h // 6 + 3)),
                        ww=int(rng.integers(w // 20 + 2, w // 6 + 3)),
                        vy=int(rng.integers(-6, 7)), vx=int(rng.integers(-6, 7)),
                        col=rng.uniform(0.0, 255.0, 3)))
    out = np.empty((nframes, h, w, 3), dtype=np.uint8)
    oy, ox = pad, pad
    for f in range(nframes):
        fr = base[oy:oy + h, ox:ox + w, :].copy()
        for s in spr:
            y0 = s["y"] + f * s["vy"]; x0 = s["x"] + f * s["vx"]
            ya, yb = max(y0, 0), min(y0 + s["hh"], h)
            xa, xb = max(x0, 0), min(x0 + s["ww"], w)
            if ya < yb and xa < xb:
                fr[ya:yb, xa:xb, :] = s["col"]
        out[f] = np.clip(np.round(fr), 0, 255).astype(np.uint8)
        oy += int(motion[f, 0]); ox += int(motion[f, 1])
    return out


def lossless_blobs(h: int = 2160, w: int = 3840, seed: int = 5,
                   bitdepth: int = 12) -> np.ndarray:
    """RGB uint16 image (h, w, 3) with values in [0, 2^bitdepth - 1].

    Sum of 20 to 60 isotropic Gaussian blobs (std 20 to 400 px, random
    colour amplitude) on a mid-grey background, plus N(0, 15^2) noise,
    rounded and clipped. Resembles smooth medical or scientific images.
    """
    rng = np.random.default_rng(seed)
    top = (1 << bitdepth) - 1
    yy = np.arange(h, dtype=np.float64)[:, None]
    xx = np.arange(w, dtype=np.float64)[None, :]
    nb = int(rng.integers(20, 61))
    gys, gxs, amps = [], [], []
    for _ in range(nb):
        cy = rng.uniform(0, h); cx = rng.uniform(0, w)
        s = rng.uniform(20.0, 400.0)
        amps.append(rng.uniform(-0.25, 0.5, 3) * top)
        gys.append(np.exp(-0.5 * ((yy[:, 0] - cy) / s) ** 2))
        gxs.append(np.exp(-0.5 * ((xx[0] - cx) / s) ** 2))
    gy = np.stack(gys, axis=1)          # [h, nb]
    gx = np.stack(gxs, axis=0)          # [nb, w]
    amp = np.stack(amps, axis=0)        # [nb, 3]
    img = np.empty((h, w, 3))
    for c in range(3):                  # separable blobs: one matrix product
        img[:, :, c] = top / 4.0 + (gy * amp[None, :, c]) @ gx
    img += rng.normal(0.0, 15.0, (h, w, 3))
    return np.clip(np.round(img), 0, top).astype(np.uint16)


def request_stream(n: int = 10000, rate: float = 200.0, seed: int = 7,
                   lo: int = 256, hi: int = 2048):
    """Decode-request descriptors for a Poisson stream.

    Inter-arrival times are exponential with the given rate (requests per
    second). Width and height are each log-uniform in [lo, hi] and rounded
    down to a multiple of 16; half the requests are grayscale, half RGB; the
    quantiser step is uniform over {4, 8, 16, 32}. Returns a list of dicts
    with keys t (arrival time, s), w, h, c (1 or 3), q and seed (image seed).
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        w = int(np.exp(rng.uniform(np.log(lo), np.log(hi)))) // 16 * 16
        h = int(np.exp(rng.uniform(np.log(lo), np.log(hi)))) // 16 * 16
        c = 1 if rng.uniform() < 0.5 else 3
        q = int(rng.choice([4, 8, 16, 32]))
        out.append(dict(t=float(t[i]), w=max(w, 16), h=max(h, 16), c=c, q=q,
                        seed=int(rng.integers(0, 2**31))))
    return out
