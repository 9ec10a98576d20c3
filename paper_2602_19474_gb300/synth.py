"""Seeded synthetic label bitmaps for the five workloads.

This module only makes input images (numpy, scipy); it holds none of the
meshing arithmetic.  Both the CUDA path and the CPU oracle consume the same
arrays.  The paper meshes private domains (a stomach MR slice, a star, a
droplet, a handwritten "Y"); these generators stand in for them with the
shapes, sizes and value distributions of the five workloads:

  disk64      64x64 u8, filled disk r=20 at (32,32) (1257 px), h=2
  ellipses    2048x2048 u8, union of 200 filled ellipses, h=4
  voronoi16   8192x8192 u16, 16 labels on the Voronoi cells of 4096 seeds,
              5x5 majority filter, h=2
  noise_batch 512 u8 bitmaps, sides log-uniform in [128, 2048], thresholded
              Gaussian-filtered white noise (sigma ~ U[4, 32]), h=2
  serving     pool of square noise bitmaps, side log-uniform in [256, 4096],
              h drawn from {2, 4, 8}

Seeds are 260219474 + workload number (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

SEED0 = 260219474


def rng_for(k: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED0 + k + 1000003 * salt))


def disk(size: int = 64, cx: float = 32, cy: float = 32, r: float = 20) -> np.ndarray:
    """Filled disk: foreground where the pixel centre satisfies (x-cx)^2+(y-cy)^2 <= r^2."""
    yy, xx = np.mgrid[0:size, 0:size]
    return (((xx - cx) ** 2 + (yy - cy) ** 2) <= r * r).astype(np.uint8)


def star(size: int = 256, points: int = 5, r_out: float = 100.0, r_in: float = 40.0, rot: float = 0.3) -> np.ndarray:
    """Filled five-pointed star (a stand-in for the paper's synthetic star):
    foreground where the pixel centre lies inside the polygon whose vertices
    alternate between radius r_out and r_in about the image centre."""
    c = (size - 1) / 2.0
    ang = rot + np.arange(2 * points) * math.pi / points
    rad = np.where(np.arange(2 * points) % 2 == 0, r_out, r_in)
    px, py = c + rad * np.cos(ang), c + rad * np.sin(ang)
    yy, xx = np.mgrid[0:size, 0:size].astype(float)
    inside = np.zeros((size, size), bool)
    j = len(px) - 1
    for i in range(len(px)):  # even-odd rule over the polygon's edges
        cond = (py[i] > yy) != (py[j] > yy)
        xint = (px[j] - px[i]) * (yy - py[i]) / np.where(py[j] != py[i], py[j] - py[i], 1.0) + px[i]
        inside ^= cond & (xx < xint)
        j = i
    return inside.astype(np.uint8)


def blob(size: int = 256, seed_k: int = 6, n: int = 7) -> np.ndarray:
    """A smooth blob (a stand-in for the paper's droplet): the union of n
    overlapping disks with seeded centres near the image centre."""
    rng = rng_for(seed_k)
    c = size / 2.0
    yy, xx = np.mgrid[0:size, 0:size].astype(float)
    img = np.zeros((size, size), bool)
    for _ in range(n):
        cx, cy = c + rng.uniform(-0.2, 0.2) * size, c + rng.uniform(-0.2, 0.2) * size
        r = rng.uniform(0.12, 0.25) * size
        img |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    return img.astype(np.uint8)


def ellipses(size: int = 2048, n: int = 200, seed_k: int = 2, amin: float = 10.0, amax: float = 150.0) -> np.ndarray:
    """Union of n filled ellipses: centres uniform over the image, semi-axes
    uniform in [amin, amax], rotation uniform in [0, pi)."""
    rng = rng_for(seed_k)
    cx = rng.uniform(0, size, n)
    cy = rng.uniform(0, size, n)
    a = rng.uniform(amin, amax, n)
    b = rng.uniform(amin, amax, n)
    th = rng.uniform(0, math.pi, n)
    img = np.zeros((size, size), np.uint8)
    for k in range(n):
        r = max(a[k], b[k])
        x0, x1 = max(0, int(cx[k] - r) - 1), min(size, int(cx[k] + r) + 2)
        y0, x1y = max(0, int(cy[k] - r) - 1), min(size, int(cy[k] + r) + 2)
        if x0 >= x1 or y0 >= x1y:
            continue
        yy, xx = np.mgrid[y0:x1y, x0:x1]
        dx, dy = xx - cx[k], yy - cy[k]
        c, s = math.cos(th[k]), math.sin(th[k])
        u = (c * dx + s * dy) / a[k]
        v = (-s * dx + c * dy) / b[k]
        img[y0:x1y, x0:x1] |= (u * u + v * v <= 1.0).astype(np.uint8)
    return img


def _mode_filter(lab: np.ndarray, nlabels: int, w: int) -> np.ndarray:
    """w x w majority filter with the window clipped at the border.  Ties keep
    the centre label when it is among the most frequent, else the smallest.
    Only pixels whose window holds more than one label can change."""
    from scipy.ndimage import maximum_filter, minimum_filter

    r = w // 2
    mixed = minimum_filter(lab, size=w, mode="nearest") != maximum_filter(lab, size=w, mode="nearest")
    ys, xs = np.nonzero(mixed)
    out = lab.copy()
    if len(ys) == 0:
        return out
    sentinel = nlabels  # pixels outside the image match no label
    pad = np.pad(lab.astype(np.int64), r, mode="constant", constant_values=sentinel)
    chunk = 1 << 20
    for c0 in range(0, len(ys), chunk):
        y, x = ys[c0:c0 + chunk], xs[c0:c0 + chunk]
        n = len(y)
        counts = np.zeros((nlabels + 1) * n, np.int32)
        ar = np.arange(n)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                nb = pad[y + r + dy, x + r + dx]
                counts += np.bincount(nb * n + ar, minlength=(nlabels + 1) * n).astype(np.int32)
        counts = counts.reshape(nlabels + 1, n)[:nlabels]
        best = np.argmax(counts, axis=0)
        centre = lab[y, x].astype(np.int64)
        keep = counts[centre, ar] == counts[best, ar]
        out[y, x] = np.where(keep, centre, best).astype(lab.dtype)
    return out


def voronoi_labels(size: int = 8192, nseeds: int = 4096, nlabels: int = 16, window: int = 5,
                   seed_k: int = 3, block_rows: int = 512) -> np.ndarray:
    """Multi-label map: each pixel takes the label of the nearest of nseeds
    uniform seeds (labels uniform in 0..nlabels-1), then a majority filter."""
    from scipy.spatial import cKDTree

    rng = rng_for(seed_k)
    seeds = rng.uniform(0, size, (nseeds, 2))
    labels = rng.integers(0, nlabels, nseeds).astype(np.uint16)
    tree = cKDTree(seeds)
    out = np.empty((size, size), np.uint16)
    xs = np.arange(size, dtype=np.float64)
    for y0 in range(0, size, block_rows):
        y1 = min(size, y0 + block_rows)
        yy, xx = np.meshgrid(np.arange(y0, y1, dtype=np.float64), xs, indexing="ij")
        _, idx = tree.query(np.stack([xx.ravel(), yy.ravel()], axis=1), k=1, workers=-1)
        out[y0:y1] = labels[idx].reshape(y1 - y0, size)
    # the filter needs a halo of window//2 rows; run it on overlapping bands
    res = np.empty_like(out)
    r = window // 2
    band = 1024
    for y0 in range(0, size, band):
        y1 = min(size, y0 + band)
        a0, a1 = max(0, y0 - r), min(size, y1 + r)
        f = _mode_filter(out[a0:a1], nlabels, window)
        res[y0:y1] = f[y0 - a0:y0 - a0 + (y1 - y0)]
    return res.astype(np.uint16)


def _gauss_kernel(sigma: float, truncate: float = 4.0) -> np.ndarray:
    rad = int(truncate * sigma + 0.5)
    x = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def _filter_axis_fft(a: np.ndarray, k: np.ndarray, axis: int) -> np.ndarray:
    """Correlate along one axis with boundary mode 'reflect' (d c b a | a b c d),
    via FFT over the reflect-padded signal."""
    import scipy.fft as sfft

    rad = (len(k) - 1) // 2
    n = a.shape[axis]
    pad = [(0, 0), (0, 0)]
    pad[axis] = (rad, rad)
    ap = np.pad(a, pad, mode="symmetric")
    m = ap.shape[axis]
    L = sfft.next_fast_len(m + len(k) - 1, real=True)
    fa = sfft.rfft(ap, n=L, axis=axis, workers=-1)
    fk = sfft.rfft(k[::-1], n=L)
    shape = [1, 1]
    shape[axis] = -1
    full = sfft.irfft(fa * fk.reshape(shape), n=L, axis=axis, workers=-1)
    sl = [slice(None), slice(None)]
    sl[axis] = slice(2 * rad, 2 * rad + n)
    return full[tuple(sl)]


def noise_bitmap(rng: np.random.Generator, width: int, height: int, sigma: float) -> np.ndarray:
    """Threshold at 0 of white noise filtered by a Gaussian (sigma px, reflect
    boundary, truncated at 4 sigma): foreground where the filtered value > 0."""
    z = rng.standard_normal((height, width))
    k = _gauss_kernel(sigma)
    f = _filter_axis_fft(_filter_axis_fft(z, k, 0), k, 1)
    return (f > 0).astype(np.uint8)


def noise_batch_specs(n: int = 512, lo: int = 128, hi: int = 2048, seed_k: int = 4):
    """(width, height, sigma, image seed) for each bitmap of the batch."""
    rng = rng_for(seed_k)
    w = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(int)
    h = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(int)
    s = rng.uniform(4.0, 32.0, n)
    return [(int(w[i]), int(h[i]), float(s[i]), i) for i in range(n)]


def noise_batch_item(spec, seed_k: int = 4) -> np.ndarray:
    """One bitmap of the batch from its (width, height, sigma, index) spec."""
    w, h, s, i = spec
    return noise_bitmap(rng_for(seed_k, salt=1 + i), w, h, s)


def noise_batch(n: int = 512, lo: int = 128, hi: int = 2048, seed_k: int = 4, first: int | None = None):
    """The batch of thresholded-noise bitmaps (optionally only the first few)."""
    specs = noise_batch_specs(n, lo, hi, seed_k)
    if first is not None:
        specs = specs[:first]
    return [noise_batch_item(sp, seed_k) for sp in specs]


def serving_specs(n: int = 128, lo: int = 256, hi: int = 4096, seed_k: int = 5):
    """(side, sigma, h, image seed) for the pool of square serving bitmaps."""
    rng = rng_for(seed_k)
    side = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(int)
    s = rng.uniform(4.0, 32.0, n)
    h = rng.choice(np.array([2, 4, 8]), n)
    return [(int(side[i]), float(s[i]), int(h[i]), i) for i in range(n)]


def serving_image(spec, seed_k: int = 5) -> np.ndarray:
    side, s, _, i = spec
    return noise_bitmap(rng_for(seed_k, salt=1 + i), side, side, s)


# workload name -> (generator, h_num, h_den)
WORKLOADS = {
    "disk64": (lambda: disk(), 2, 1),
    "ellipses2048": (lambda: ellipses(), 4, 1),
    "voronoi8192": (lambda: voronoi_labels(), 2, 1),
}


def delaunay_mesh(width: int, height: int, n: int = 900, seed_k: int = 7, spacing: float = 2.0):
    """A conforming counter-clockwise triangle mesh of the image rectangle
    [-1/2, W - 1/2] x [-1/2, H - 1/2] that is no lattice: the Delaunay
    triangulation of the rectangle's corners, points every `spacing` px along
    its sides (edges lying on the border's pixel lines) and n seeded points.
    Returns (xy (m, 2) float64, tri (t, 3) int32)."""
    from scipy.spatial import Delaunay

    rng = rng_for(seed_k)
    sx = np.arange(-0.5 + spacing, width - 0.5, spacing)
    sy = np.arange(-0.5 + spacing, height - 0.5, spacing)
    pts = np.concatenate([
        [[-0.5, -0.5], [width - 0.5, -0.5], [width - 0.5, height - 0.5], [-0.5, height - 0.5]],
        np.stack([sx, np.full_like(sx, -0.5)], 1), np.stack([sx, np.full_like(sx, height - 0.5)], 1),
        np.stack([np.full_like(sy, -0.5), sy], 1), np.stack([np.full_like(sy, width - 0.5), sy], 1),
        rng.uniform([-0.5, -0.5], [width - 0.5, height - 0.5], (n, 2))])
    tri = Delaunay(pts).simplices.astype(np.int32)
    P = pts[tri]
    o = (P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0])
    tri[o < 0] = tri[o < 0][:, [0, 2, 1]]
    return pts, np.ascontiguousarray(tri)
