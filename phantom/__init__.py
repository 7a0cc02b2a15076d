"""Seeded synthetic inputs for Fuzzy C-Means image segmentation.

This module is shared by the FP64 oracle tests and the CUDA path. It holds
none of the clustering arithmetic: it only draws images, their label maps and
the random initial membership matrix, from numpy's seeded generators.

The paper segments skull-stripped BrainWeb slices into four classes
(background, CSF, GM, WM; Sec. 5.2). That dataset is not available, so the
images here stand in for it with the same structure:

* ``phantom2d``  nested seeded ellipses (background, CSF, GM, WM) with
  Gaussian noise, clipped to [0, 255] and rounded to uint8.
* ``phantom3d``  nested ellipsoids with a smooth multiplicative bias field
  (a degree <= 2 polynomial scaled to +/-20 %) and Rician-like noise
  (magnitude of a complex Gaussian), clipped and rounded to uint8.
* ``slice_spec`` / ``batch_slice``  per-slice random size (log-uniform side
  64..512), cluster count C in {3, 4, 5}, class means (sorted draws in
  [0, 235] with a minimum gap of 20) and noise sigma in [4, 12].
* ``dirichlet_u0``  the random initial membership of Algorithm 1 step 2: a
  per-pixel uniform Dirichlet(1, ..., 1) drawn as normalised -ln(U(0, 1])
  in FP64 and stored as FP32, cluster-major ``U0[j, i]``.
* ``philox_dirichlet_u0``  the same distribution from the counter-based
  generator Philox4x32-10, the definition the library's on-device start
  (``fcm_init_dirichlet``) implements on its own side.

Every draw is keyed by a tuple of integers through ``numpy.random.SeedSequence``
so that the same key gives the same array on any machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BRAIN_MEANS = (0.0, 40.0, 110.0, 150.0)  # background, CSF, GM, WM

# Seeds of the standard workloads.
SINGLE_IMAGE_SEEDS = {
    # name: (phantom seed, U0 seed)
    "phantom200": (1, 101),
    "phantom1024": (2, 102),
    "volume256": (3, 103),
}
BATCH_FAMILY = 4            # slice i of the 512-slice batch is keyed (4, i)
TRAIN_OFFSET = 1_000_000    # training slice i is keyed (4, 1_000_000 + i)
U0_FAMILY = 104             # U0 of batch slice i is keyed (104, i)


def rng(*key: int) -> np.random.Generator:
    """A numpy Generator keyed by a tuple of non-negative integers."""
    return np.random.default_rng(np.random.SeedSequence([int(k) for k in key]))


# ---------------------------------------------------------------------------
# 2-D phantom
# ---------------------------------------------------------------------------

def _ellipse_params(g: np.random.Generator, n_levels: int, H: int, W: int):
    """Centres, semi-axes and angles of ``n_levels - 1`` nested ellipses."""
    out = []
    cy = H / 2 + g.uniform(-0.05, 0.05) * H
    cx = W / 2 + g.uniform(-0.05, 0.05) * W
    a = g.uniform(0.36, 0.46) * W
    b = g.uniform(0.36, 0.46) * H
    th = g.uniform(-0.5, 0.5)
    for _ in range(1, n_levels):
        out.append((cy, cx, a, b, th))
        cy = cy + g.uniform(-0.1, 0.1) * b
        cx = cx + g.uniform(-0.1, 0.1) * a
        a = a * g.uniform(0.55, 0.8)
        b = b * g.uniform(0.55, 0.8)
        th = th + g.uniform(-0.3, 0.3)
    return out


def _label_map_2d(params, H: int, W: int) -> np.ndarray:
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64) + 0.5,
                         np.arange(W, dtype=np.float64) + 0.5, indexing="ij")
    lab = np.zeros((H, W), dtype=np.uint8)
    for level, (cy, cx, a, b, th) in enumerate(params, start=1):
        dy, dx = yy - cy, xx - cx
        c, s = math.cos(th), math.sin(th)
        p = (dx * c + dy * s) / a
        q = (-dx * s + dy * c) / b
        lab[p * p + q * q <= 1.0] = level
    return lab


def _to_uint8(v: np.ndarray) -> np.ndarray:
    return np.rint(np.clip(v, 0.0, 255.0)).astype(np.uint8)


def phantom2d(seed: int, H: int, W: int, sigma: float,
              means=BRAIN_MEANS, *, key=None):
    """Nested-ellipse phantom with Gaussian noise.

    Returns ``(image uint8 [H, W], labels uint8 [H, W])``; label k has mean
    ``means[k]`` before noise.
    """
    g = rng(*(key if key is not None else (seed,)))
    params = _ellipse_params(g, len(means), H, W)
    lab = _label_map_2d(params, H, W)
    mu = np.asarray(means, dtype=np.float64)[lab]
    img = _to_uint8(mu + g.normal(0.0, sigma, size=(H, W)))
    return img, lab


def multichannel2d(seed: int, H: int, W: int, sigma: float, contrasts):
    """One nested-ellipse layout rendered once per channel with that
    channel's class means (``contrasts[d]``) and its own Gaussian noise, as
    co-registered images of different tissue contrast.

    Returns ``(image uint8 [D, H*W], labels uint8 [H*W])``.
    """
    g = rng(seed)
    params = _ellipse_params(g, len(contrasts[0]), H, W)
    lab = _label_map_2d(params, H, W)
    chans = []
    for d, means in enumerate(contrasts):
        mu = np.asarray(means, dtype=np.float64)[lab]
        chans.append(_to_uint8(mu + rng(seed, 1000 + d).normal(0.0, sigma, size=(H, W))).reshape(-1))
    return np.stack(chans), lab.reshape(-1)


# ---------------------------------------------------------------------------
# 3-D phantom
# ---------------------------------------------------------------------------

def phantom3d(seed: int, D: int, H: int, W: int, sigma: float = 6.0,
              bias: float = 0.2, means=BRAIN_MEANS):
    """Nested-ellipsoid volume with a bias field and Rician-like noise.

    The bias is ``b = 1 + bias * p(z, y, x)`` with p a degree <= 2
    polynomial in coordinates scaled to [-1, 1], with seeded N(0, 1)
    coefficients, scaled so that max |p| over the grid is 1. The noisy
    value is ``|s * b + n1 + i n2|`` with n1, n2 ~ N(0, sigma^2).
    Returns ``(volume uint8 [D, H, W], labels uint8 [D, H, W])``.
    """
    g = rng(seed)
    L = len(means)
    # nested ellipsoids: centre, semi-axes (z, y, x), in-plane angle
    ells = []
    cz = D / 2 + g.uniform(-0.05, 0.05) * D
    cy = H / 2 + g.uniform(-0.05, 0.05) * H
    cx = W / 2 + g.uniform(-0.05, 0.05) * W
    az, ay, ax = (g.uniform(0.36, 0.46) * D, g.uniform(0.36, 0.46) * H,
                  g.uniform(0.36, 0.46) * W)
    th = g.uniform(-0.5, 0.5)
    for _ in range(1, L):
        ells.append((cz, cy, cx, az, ay, ax, th))
        cz += g.uniform(-0.1, 0.1) * az
        cy += g.uniform(-0.1, 0.1) * ay
        cx += g.uniform(-0.1, 0.1) * ax
        az *= g.uniform(0.7, 0.88)
        ay *= g.uniform(0.7, 0.88)
        ax *= g.uniform(0.7, 0.88)
        th += g.uniform(-0.3, 0.3)
    # bias polynomial: 1, z, y, x, z^2, y^2, x^2, zy, zx, yx
    coef = g.normal(0.0, 1.0, size=10)
    zs = np.linspace(-1.0, 1.0, D)
    ys = np.linspace(-1.0, 1.0, H)
    xs = np.linspace(-1.0, 1.0, W)

    def poly(z, y, x):
        return (coef[0] + coef[1] * z + coef[2] * y + coef[3] * x
                + coef[4] * z * z + coef[5] * y * y + coef[6] * x * x
                + coef[7] * z * y + coef[8] * z * x + coef[9] * y * x)

    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    pmax = 0.0
    for z in zs:
        pmax = max(pmax, float(np.max(np.abs(poly(z, yy, xx)))))
    scale = bias / pmax

    mu = np.asarray(means, dtype=np.float64)
    vol = np.empty((D, H, W), dtype=np.uint8)
    lab = np.empty((D, H, W), dtype=np.uint8)
    py, px = np.meshgrid(np.arange(H, dtype=np.float64) + 0.5,
                         np.arange(W, dtype=np.float64) + 0.5, indexing="ij")
    for k in range(D):
        pz = k + 0.5
        lk = np.zeros((H, W), dtype=np.uint8)
        for level, (ez, ey, ex, az_, ay_, ax_, th_) in enumerate(ells, start=1):
            c, s = math.cos(th_), math.sin(th_)
            dy, dx = py - ey, px - ex
            p = (dx * c + dy * s) / ax_
            q = (-dx * s + dy * c) / ay_
            r = (pz - ez) / az_
            lk[p * p + q * q + r * r <= 1.0] = level
        b = 1.0 + scale * poly(zs[k], yy, xx)
        sig = mu[lk] * b
        n1 = g.normal(0.0, sigma, size=(H, W))
        n2 = g.normal(0.0, sigma, size=(H, W))
        vol[k] = _to_uint8(np.sqrt((sig + n1) ** 2 + n2 ** 2))
        lab[k] = lk
    return vol, lab


# ---------------------------------------------------------------------------
# Batches of uneven slices
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class SliceSpec:
    index: int
    side: int
    C: int
    means: tuple
    sigma: float


def slice_spec(i: int, family: int = BATCH_FAMILY) -> SliceSpec:
    """Size, cluster count, class means and noise of batch slice ``i``."""
    g = rng(family, i)
    side = int(round(math.exp(g.uniform(math.log(64.0), math.log(512.0)))))
    C = int(g.integers(3, 6))
    while True:
        m = np.sort(g.uniform(0.0, 235.0, size=C))
        if C == 1 or np.min(np.diff(m)) >= 20.0:
            break
    perm = g.permutation(C)
    means = tuple(float(m[p]) for p in perm)
    sigma = float(g.uniform(4.0, 12.0))
    return SliceSpec(i, side, C, means, sigma)


def batch_slice(i: int, family: int = BATCH_FAMILY):
    """Image and labels of batch slice ``i``: ``(spec, image uint8, labels)``."""
    sp = slice_spec(i, family)
    img, lab = phantom2d(0, sp.side, sp.side, sp.sigma, sp.means,
                         key=(family, i, 1))
    return sp, img, lab


# ---------------------------------------------------------------------------
# Random initial membership (Algorithm 1, step 2)
# ---------------------------------------------------------------------------

def dirichlet_u0(key, C: int, n: int) -> np.ndarray:
    """Uniform Dirichlet(1, ..., 1) membership per pixel, FP32 ``[C, n]``.

    Drawn as E_j = -ln(1 - r_j) with r_j ~ U[0, 1) (so E_j is standard
    exponential), normalised per pixel in FP64, then rounded to FP32.
    """
    if isinstance(key, int):
        key = (key,)
    g = rng(*key)
    out = np.empty((C, n), dtype=np.float32)
    chunk = 1 << 22
    for s in range(0, n, chunk):
        e = -np.log1p(-g.random((C, min(chunk, n - s))))
        out[:, s:s + e.shape[1]] = (e / e.sum(axis=0, keepdims=True)).astype(np.float32)
    return out


def single_image(name: str):
    """One of the standard single-image workloads.

    Returns ``(x uint8 flat, labels flat, u0 FP32 [C, n], C)``:
    ``phantom200`` (200 x 200, sigma 8), ``phantom1024`` (1024 x 1024,
    sigma 10), ``volume256`` (256^3 with bias and Rician noise, sigma 6).
    """
    seed, useed = SINGLE_IMAGE_SEEDS[name]
    if name == "phantom200":
        img, lab = phantom2d(seed, 200, 200, 8.0)
    elif name == "phantom1024":
        img, lab = phantom2d(seed, 1024, 1024, 10.0)
    elif name == "volume256":
        img, lab = phantom3d(seed, 256, 256, 256, 6.0)
    else:
        raise KeyError(name)
    x = img.reshape(-1)
    C = 4
    return x, lab.reshape(-1), dirichlet_u0(useed, C, x.size), C


# ---------------------------------------------------------------------------
# Counter-based random initial membership (the library's on-device start)
# ---------------------------------------------------------------------------

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57   # round multipliers
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85   # key increments (Weyl sequence)


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
    as easy as 1, 2, 3", SC'11): ten rounds on a 128-bit counter ``ctr`` (four
    uint32 arrays) under a 64-bit key ``(k0, k1)``. A round multiplies words 0
    and 2 by the two multipliers (64-bit products), and gives
    (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the two
    increments between rounds. Returns four uint32 arrays."""
    mask = np.uint64(0xFFFFFFFF)
    c = [np.asarray(v, dtype=np.uint64) & mask for v in ctr]
    k0, k1 = np.uint64(key[0]) & mask, np.uint64(key[1]) & mask
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(PHILOX_W0)) & mask
            k1 = (k1 + np.uint64(PHILOX_W1)) & mask
        p0 = c[0] * np.uint64(PHILOX_M0)
        p1 = c[2] * np.uint64(PHILOX_M1)
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & mask, (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & mask]
    return [v.astype(np.uint32) for v in c]


def philox_dirichlet_u0(seed: int, C: int, n: int) -> np.ndarray:
    """Uniform Dirichlet(1, ..., 1) membership per pixel, FP32 ``[C, n]``, from
    Philox4x32-10 — the definition the library's on-device start implements.

    Pixel i draws counter (i mod 2^32, i div 2^32, b, 0) for blocks b = 0, 1
    under key (seed mod 2^32, seed div 2^32); cluster j takes word j mod 4 of
    block j div 4. A word w gives r = (2 floor(w / 512) + 1) / 2^24 in (0, 1),
    E_j = -ln r_j (standard exponential), u_j = E_j / sum_k E_k (FP64, then
    rounded to FP32)."""
    seed = int(seed)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.empty((C, n), dtype=np.float32)
    chunk = 1 << 22
    for s in range(0, n, chunk):
        i = np.arange(s, min(n, s + chunk), dtype=np.uint64)
        lo, hi = i & np.uint64(0xFFFFFFFF), i >> np.uint64(32)
        words = []
        for b in range((C + 3) // 4):
            words += philox4x32_10([lo, hi, np.full(i.size, b, dtype=np.uint64), np.zeros(i.size, np.uint64)], key)
        E = np.stack([-np.log((2.0 * (w >> np.uint32(9)).astype(np.float64) + 1.0) / 16777216.0) for w in words[:C]])
        out[:, s:s + i.size] = (E / E.sum(axis=0, keepdims=True)).astype(np.float32)
    return out
