"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's 80-cloud dataset and its trained weights are not available, so every
input here is generated from a seed: clouds (a sum of Gaussian blobs, or
thresholded fractal gradient noise), cameras, light directions, query sets and
He-initialised network parameters.  This module holds none of the method's
arithmetic; both the CUDA path (through the tests and the benchmark) and the
CPU oracle consume what it returns.  numpy only.
"""
from __future__ import annotations

import math

import numpy as np

K, S, DIN, H, NTAIL = 10, 225, 226, 200, 3


# --------------------------------------------------------------------------- clouds
def blob_cloud(n: int = 64, nblobs: int = 8, seed: int = 1, peak: float = 50.0) -> np.ndarray:
    """Sum of `nblobs` isotropic Gaussian blobs in the unit box, sampled at voxel
    centres of an n^3 grid and rescaled so the largest voxel equals `peak`
    (extinction per unit of the unit box).  Centres U[0.25,0.75]^3, widths
    U[0.06,0.14], amplitudes U[0.5,1]."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.25, 0.75, size=(nblobs, 3))
    s = rng.uniform(0.06, 0.14, size=nblobs)
    a = rng.uniform(0.5, 1.0, size=nblobs)
    t = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    dens = np.zeros((n, n, n), np.float64)
    for i in range(nblobs):
        r2 = (X - c[i, 0]) ** 2 + (Y - c[i, 1]) ** 2 + (Z - c[i, 2]) ** 2
        dens += a[i] * np.exp(-r2 / (2.0 * s[i] ** 2))
    dens *= peak / dens.max()
    return dens.astype(np.float32)


def _perm(seed: int) -> np.ndarray:
    p = np.random.default_rng(seed).permutation(256).astype(np.int64)
    return np.concatenate([p, p, p[:1]])


def _grad(h, x, y, z):
    # the 12 edge directions of a cube (Perlin 2002), 16 cases via h & 15
    h = h & 15
    u = np.where(h < 8, x, y)
    v = np.where(h < 4, y, np.where((h == 12) | (h == 14), x, z))
    return np.where(h & 1, -u, u) + np.where(h & 2, -v, v)


def gradient_noise(x, y, z, perm) -> np.ndarray:
    """Lattice gradient noise following Perlin's improved-noise construction
    (SIGGRAPH 2002): quintic fade, hashed gradients from a permutation table."""
    fx, fy, fz = np.floor(x), np.floor(y), np.floor(z)
    X = fx.astype(np.int64) & 255
    Y = fy.astype(np.int64) & 255
    Z = fz.astype(np.int64) & 255
    x, y, z = x - fx, y - fy, z - fz
    fade = lambda t: t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    u, v, w = fade(x), fade(y), fade(z)
    A = perm[X] + Y
    AA = perm[A] + Z
    AB = perm[A + 1] + Z
    B = perm[X + 1] + Y
    BA = perm[B] + Z
    BB = perm[B + 1] + Z
    lerp = lambda t, a, b: a + t * (b - a)
    return lerp(w,
                lerp(v, lerp(u, _grad(perm[AA], x, y, z), _grad(perm[BA], x - 1, y, z)),
                     lerp(u, _grad(perm[AB], x, y - 1, z), _grad(perm[BB], x - 1, y - 1, z))),
                lerp(v, lerp(u, _grad(perm[AA + 1], x, y, z - 1), _grad(perm[BA + 1], x - 1, y, z - 1)),
                     lerp(u, _grad(perm[AB + 1], x, y - 1, z - 1),
                          _grad(perm[BB + 1], x - 1, y - 1, z - 1))))


def _grad_t(h, x, y, z):
    import torch
    h = h & 15
    u = torch.where(h < 8, x, y)
    v = torch.where(h < 4, y, torch.where((h == 12) | (h == 14), x, z))
    return torch.where((h & 1) != 0, -u, u) + torch.where((h & 2) != 0, -v, v)


def _noise_t(x, y, z, perm):
    """gradient_noise() on torch tensors (same construction, any device)."""
    import torch
    fx, fy, fz = torch.floor(x), torch.floor(y), torch.floor(z)
    X, Y, Z = fx.long() & 255, fy.long() & 255, fz.long() & 255
    x, y, z = x - fx, y - fy, z - fz
    fade = lambda t: t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    u, v, w = fade(x), fade(y), fade(z)
    A = perm[X] + Y
    AA, AB = perm[A] + Z, perm[A + 1] + Z
    B = perm[X + 1] + Y
    BA, BB = perm[B] + Z, perm[B + 1] + Z
    lerp = lambda t, a, b: a + t * (b - a)
    return lerp(w,
                lerp(v, lerp(u, _grad_t(perm[AA], x, y, z), _grad_t(perm[BA], x - 1, y, z)),
                     lerp(u, _grad_t(perm[AB], x, y - 1, z), _grad_t(perm[BB], x - 1, y - 1, z))),
                lerp(v, lerp(u, _grad_t(perm[AA + 1], x, y, z - 1), _grad_t(perm[BA + 1], x - 1, y, z - 1)),
                     lerp(u, _grad_t(perm[AB + 1], x, y - 1, z - 1),
                          _grad_t(perm[BB + 1], x - 1, y - 1, z - 1))))


def fbm_cloud(n: int = 256, seed: int = 7, octaves: int = 6, coverage: float = 0.30,
              peak: float = 50.0, base_freq: float = 4.0, shape=None, device=None) -> np.ndarray:
    """Cumulus-like cloud: 6-octave fBm (lacunarity 2, gain 0.5) of gradient noise
    added to a spherical falloff, thresholded so that `coverage` of the voxels are
    non-zero, rescaled so the largest voxel equals `peak`.  shape=(nz, ny, nx)
    allows non-cubic grids (the longest edge spans the unit box).  Evaluated with
    torch in FP64 on `device` (default: CUDA when available, else CPU); returns a
    float32 numpy array."""
    import torch
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    nz, ny, nx = shape if shape is not None else (n, n, n)
    m = max(nx, ny, nz)
    perm = torch.as_tensor(_perm(seed), device=device)
    off = np.random.default_rng(seed + 1).uniform(0, 64, size=3)
    f64 = dict(dtype=torch.float64, device=device)
    tx = (torch.arange(nx, **f64) + 0.5) / m
    ty = (torch.arange(ny, **f64) + 0.5) / m
    cx, cy, cz = 0.5 * nx / m, 0.5 * ny / m, 0.5 * nz / m
    Y, X = torch.meshgrid(ty, tx, indexing="ij")
    out = torch.empty((nz, ny, nx), **f64)
    slab = max(1, (1 << 22) // (nx * ny))
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        tz = ((torch.arange(k0, k1, **f64) + 0.5) / m)[:, None, None]
        Xs, Ys = X[None].expand(k1 - k0, -1, -1), Y[None].expand(k1 - k0, -1, -1)
        Zs = tz.expand_as(Xs)
        f = torch.zeros_like(Xs)
        amp, freq = 1.0, base_freq
        for _ in range(octaves):
            f += amp * _noise_t(Xs * freq + off[0], Ys * freq + off[1], Zs * freq + off[2], perm)
            amp *= 0.5
            freq *= 2.0
        r = torch.sqrt((Xs - cx) ** 2 + (Ys - cy) ** 2 + (Zs - cz) ** 2) / (0.45 * min(nx, ny, nz) / m)
        out[k0:k1] = 0.7 * f + (1.0 - r * r)
    a = out.cpu().numpy().astype(np.float32)
    kth = int(round((1.0 - coverage) * (a.size - 1)))
    tau = np.partition(a.ravel(), kth)[kth]
    a = np.maximum(a - tau, 0.0)
    a *= peak / a.max()
    return a.astype(np.float32)


# --------------------------------------------------------------------------- scene
def unit_sphere_dir(seed: int) -> np.ndarray:
    """Direction uniform on the sphere (seeded)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    r = math.sqrt(max(0.0, 1.0 - z * z))
    return np.array([r * math.cos(phi), r * math.sin(phi), z])


def camera(shape, width: int, height: int, spp: int = 1, seed: int = 3, light_seed: int = 4,
           fov_y_deg: float = 30.0, dist: float = 1.7, light_dir=None) -> dict:
    """Pinhole camera orbiting the unit-box cloud (seeded azimuth, elevation in
    [-20, 40] degrees), looking at the box centre, y up."""
    nz, ny, nx = shape
    m = max(nx, ny, nz)
    centre = np.array([0.5 * nx / m, 0.5 * ny / m, 0.5 * nz / m])
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 2.0 * math.pi)
    el = math.radians(rng.uniform(-20.0, 40.0))
    pos = centre + dist * np.array([math.cos(el) * math.sin(az), math.sin(el),
                                    math.cos(el) * math.cos(az)])
    fwd = centre - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    wl = unit_sphere_dir(light_seed) if light_dir is None else np.asarray(light_dir, np.float64)
    wl = wl / np.linalg.norm(wl)
    return {
        "cam_pos": pos, "cam_fwd": fwd, "cam_right": right, "cam_up": up,
        "tan_half_fov_y": math.tan(math.radians(fov_y_deg) / 2.0),
        "width": int(width), "height": int(height), "spp": int(spp),
        "seed": int(seed) * 7919 + 17, "light_dir": wl, "light_E": 1.0,
    }


def random_queries(shape, q: int, seed: int = 5, margin: float = 0.0):
    """q shading positions uniform in the unit-box grid extent and q unit tracing
    directions uniform on the sphere (float64)."""
    nz, ny, nx = shape
    m = max(nx, ny, nz)
    ext = np.array([nx / m, ny / m, nz / m])
    rng = np.random.default_rng(seed)
    x = rng.uniform(margin, 1.0 - margin, size=(q, 3)) * ext
    z = rng.uniform(-1.0, 1.0, size=q)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=q)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return x, d


# --------------------------------------------------------------------------- network
def param_shapes(K_: int = K, din: int = DIN, H_: int = H, ntail: int = NTAIL):
    """(name, shape, fan_in) of the flat parameter vector, in its documented order:
    per block V [H][din], W1 [H][H] (blocks 2..K), b1 [H], W2 [H][H], b2 [H];
    then the standard layers [H][H], [H], ..., [1][H], [1]."""
    out = []
    for k in range(K_):
        fan1 = din + (H_ if k > 0 else 0)
        out.append((f"V{k + 1}", (H_, din), fan1))
        if k > 0:
            out.append((f"W1_{k + 1}", (H_, H_), fan1))
        out.append((f"b1_{k + 1}", (H_,), 0))
        out.append((f"W2_{k + 1}", (H_, H_), H_))
        out.append((f"b2_{k + 1}", (H_,), 0))
    for t in range(ntail):
        o = 1 if t == ntail - 1 else H_
        out.append((f"T{t + 1}", (o, H_), H_))
        out.append((f"bT{t + 1}", (o,), 0))
    return out


def param_count(**kw) -> int:
    return int(sum(int(np.prod(s)) for _, s, _ in param_shapes(**kw)))


def he_init(seed: int = 2, bias: float = 0.0, positive_head: bool = True, **kw) -> np.ndarray:
    """He-normal weights (std sqrt(2/fan_in)), constant biases, float32 flat.  With
    positive_head the output layer's weights are taken in absolute value, so the
    (non-negative, ReLU) hidden state maps to a positive prediction instead of an
    output ReLU that is dead for every input of a similar-looking batch."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = param_shapes(**kw)
    for i, (_, shp, fan) in enumerate(shapes):
        if fan:
            w = rng.normal(0.0, math.sqrt(2.0 / fan), size=shp)
            if positive_head and i == len(shapes) - 2:
                w = np.abs(w)
            parts.append(w.ravel())
        else:
            parts.append(np.full(shp, bias).ravel())
    return np.concatenate(parts).astype(np.float32)


def split_params(flat, **kw) -> dict:
    out, o = {}, 0
    for name, shp, _ in param_shapes(**kw):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n]).reshape(shp)
        o += n
    return out


def join_params(parts: dict, **kw) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).ravel()
                           for name, _, _ in param_shapes(**kw)])


# architectures of the comparison in Sec. 7 (Fig. 10): hidden widths of the plain MLPs
SHALLOW_WIDE = (400, 400, 200, 200, 200)
DEEP_NARROW = (200,) * 22


def dense_he_init(widths, din: int, seed: int = 2, bias: float = 0.0, positive_head: bool = True) -> np.ndarray:
    """He-normal weights for a plain MLP with hidden widths `widths` on din inputs (flat
    layout: W_i [w_i][w_{i-1}], b_i per layer, then the output row and bias), float32."""
    rng = np.random.default_rng(seed)
    parts, prev = [], din
    for w in widths:
        parts.append(rng.normal(0.0, math.sqrt(2.0 / prev), size=w * prev))
        parts.append(np.full(w, bias))
        prev = w
    wo = rng.normal(0.0, math.sqrt(2.0 / prev), size=prev)
    parts.append(np.abs(wo) if positive_head else wo)
    parts.append(np.full(1, bias))
    return np.concatenate(parts).astype(np.float32)
