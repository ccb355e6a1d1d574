"""Seeded design fields and request streams (see the package docstring)."""

import numpy as np


def _cone_smooth(x, radius=1.5):
    """Normalised cone-kernel smoothing of a (nz, ny, nx) array, zero-flux at the box faces."""
    r = int(np.floor(radius))
    offs = []
    for dk in range(-r, r + 1):
        for dj in range(-r, r + 1):
            for di in range(-r, r + 1):
                wgt = radius - np.sqrt(di * di + dj * dj + dk * dk)
                if wgt > 0:
                    offs.append((dk, dj, di, wgt))
    acc = np.zeros_like(x)
    norm = np.zeros_like(x)
    nz, ny, nx = x.shape
    for dk, dj, di, wgt in offs:
        src = [slice(max(0, d), n + min(0, d)) for d, n in zip((dk, dj, di), (nz, ny, nx))]
        dst = [slice(max(0, -d), n + min(0, -d)) for d, n in zip((dk, dj, di), (nz, ny, nx))]
        acc[tuple(dst)] += wgt * x[tuple(src)]
        norm[tuple(dst)] += wgt
    return acc / norm


def filtered_random(nx, ny, nz, seed, volfrac=None):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nz, ny, nx))
    x = _cone_smooth(x, 1.5)
    x = (x - x.min()) / (x.max() - x.min())
    if volfrac is not None:
        lo, hi = -1.0, 1.0
        for _ in range(100):
            c = 0.5 * (lo + hi)
            if np.clip(x + c, 0.0, 1.0).mean() < volfrac:
                lo = c
            else:
                hi = c
        x = np.clip(x + 0.5 * (lo + hi), 0.0, 1.0)
    return np.ascontiguousarray(x.ravel(), dtype=np.float64)


def fin_plates(nx, ny, nz, seed, heated_layers=2, n_plates=8, thickness=2, top=0.75):
    rng = np.random.default_rng(seed)
    x = np.zeros((nz, ny, nx))
    spacing = nx / n_plates
    ztop = int(round(top * nz))
    for p in range(n_plates):
        c = int(round((p + 0.5) * spacing - thickness / 2))
        x[heated_layers:ztop, :, max(0, c):min(nx, c + thickness)] = 1.0
    x = np.clip(x + 0.05 * rng.standard_normal(x.shape), 0.0, 1.0)
    return np.ascontiguousarray(x.ravel(), dtype=np.float64)


def request_stream(n=300, rate=20.0, seed=12345, sizes=(32, 48, 64, 96, 128),
                   alpha_range=(1e3, 1e5)):
    """List of dicts: t_arrival, n (grid edge), alpha, adjoint (bool), design_seed."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    edge = rng.choice(np.asarray(sizes), size=n)
    la = rng.uniform(np.log(alpha_range[0]), np.log(alpha_range[1]), size=n)
    adj = rng.random(n) < 0.5
    seeds = rng.integers(0, 2**31 - 1, size=n)
    return [dict(t_arrival=float(t[i]), n=int(edge[i]), alpha=float(np.exp(la[i])),
                 adjoint=bool(adj[i]), design_seed=int(seeds[i])) for i in range(n)]


def filtered_random_torch(nx, ny, nz, seed, volfrac=None, device="cpu", noise=None):
    """The filtered_random recipe computed with torch on `device` (for streams of many designs that
    should be drawn in milliseconds on the device): N(0, 1) per element from torch's generator seeded
    with `seed` (or the given (nz, ny, nx) `noise`), the same cone smoothing, min-max map and
    volume-fraction bisection (on the device, no host round trips). Not byte-identical to
    filtered_random, whose normals come from NumPy's PCG64."""
    import torch
    if noise is None:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        x = torch.randn((nz, ny, nx), generator=gen, device=device, dtype=torch.float64)
    else:
        x = torch.as_tensor(noise, dtype=torch.float64, device=device)
    radius, r = 1.5, 1
    acc = torch.zeros_like(x)
    norm = torch.zeros_like(x)
    for dk in range(-r, r + 1):
        for dj in range(-r, r + 1):
            for di in range(-r, r + 1):
                wgt = radius - float(np.sqrt(di * di + dj * dj + dk * dk))
                if wgt <= 0:
                    continue
                src = tuple(slice(max(0, d), n + min(0, d)) for d, n in zip((dk, dj, di), (nz, ny, nx)))
                dst = tuple(slice(max(0, -d), n + min(0, -d)) for d, n in zip((dk, dj, di), (nz, ny, nx)))
                acc[dst] += wgt * x[src]
                norm[dst] += wgt
    x = acc / norm
    x = (x - x.min()) / (x.max() - x.min())
    if volfrac is not None:
        lo = torch.full((), -1.0, dtype=torch.float64, device=device)
        hi = torch.full((), 1.0, dtype=torch.float64, device=device)
        for _ in range(100):
            c = 0.5 * (lo + hi)
            below = torch.clamp(x + c, 0.0, 1.0).mean() < volfrac
            lo = torch.where(below, c, lo)
            hi = torch.where(below, hi, c)
        x = torch.clamp(x + 0.5 * (lo + hi), 0.0, 1.0)
    return x.reshape(-1).contiguous()
