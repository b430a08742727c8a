"""Seeded synthetic volumes shared by the tests, the benchmark and the oracle
checks.  Holds none of the transform's arithmetic: only random fields.

Volume b of a batch is drawn from ``numpy.random.default_rng(seed + b)`` so a
single volume can be regenerated without the rest of its batch.

Recipes (the paper's only workload, an artificial voxel "sword" of opacities
in [0, 1], is not available; these stand in for it):

* ``uniform``        i.i.d. U[-1, 1] coefficients.
* ``smoothed_noise`` periodic Gaussian smoothing of N(0,1) white noise,
                     sigma in lattice spacings (frequency-domain multiply),
                     rescaled to unit sample variance.
* ``phantom``        CT-like phantom: K ~ U{10..30} ellipsoids, centres
                     U[0, n)^3, semi-axes U[0.05 n, 0.35 n], uniformly random
                     rotations, densities U[0, 1] added up, plus N(0, noise^2).
"""
import numpy as np


def _rng(seed, b):
    return np.random.default_rng(int(seed) + int(b))


def uniform(n, batch=1, seed=0, complex_=False):
    out = np.empty((batch, n, n, n), dtype=np.complex128 if complex_ else np.float64)
    for b in range(batch):
        g = _rng(seed, b)
        v = g.uniform(-1.0, 1.0, size=(n, n, n))
        if complex_:
            v = v + 1j * g.uniform(-1.0, 1.0, size=(n, n, n))
        out[b] = v
    return out


def smoothed_noise(n, batch=1, seed=0, sigma=2.0):
    out = np.empty((batch, n, n, n), dtype=np.float64)
    f = np.fft.fftfreq(n)
    f2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2
    gain = np.exp(-2.0 * np.pi ** 2 * sigma ** 2 * f2)
    for b in range(batch):
        w = _rng(seed, b).standard_normal((n, n, n))
        v = np.fft.ifftn(np.fft.fftn(w) * gain).real
        v -= v.mean()
        sd = v.std()
        out[b] = v / sd if sd > 0 else v
    return out


def _rotation(g):
    q = g.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def phantom(n, batch=1, seed=0, noise=1e-3):
    out = np.zeros((batch, n, n, n), dtype=np.float64)
    for b in range(batch):
        g = _rng(seed, b)
        vol = out[b]
        for _ in range(int(g.integers(10, 31))):
            c = g.uniform(0.0, n, size=3)
            ax = g.uniform(0.05 * n, 0.35 * n, size=3)
            R = _rotation(g)
            rho = g.uniform(0.0, 1.0)
            half = np.sqrt(((R * ax[None, :]) ** 2).sum(1))
            lo = np.maximum(np.floor(c - half).astype(int), 0)
            hi = np.minimum(np.ceil(c + half).astype(int) + 1, n)
            if np.any(hi <= lo):
                continue
            grids = np.meshgrid(*[np.arange(lo[i], hi[i]) for i in range(3)], indexing="ij")
            p = np.stack(grids, -1) - c
            q = (p @ R) / ax
            inside = (q * q).sum(-1) <= 1.0
            vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += rho * inside
        vol += noise * g.standard_normal((n, n, n))
    return out


def ragged_orders(count, seed=0, choices=tuple(range(8, 97, 8))):
    g = np.random.default_rng(int(seed))
    return [int(v) for v in g.choice(np.asarray(choices), size=count)]


def bernoulli_mask(n, batch=1, seed=0, p=0.1):
    out = np.empty((batch, n, n, n), dtype=bool)
    for b in range(batch):
        out[b] = _rng(seed, b).random((n, n, n)) < p
    return out


def phantom_device(n, batch, seed=0, noise=1e-3, device="cuda"):
    """Same recipe as ``phantom`` evaluated with torch on `device` (used for
    benchmark-sized batches).  Ellipsoid parameters come from
    ``default_rng(seed + b)``; the N(0, noise^2) term from a torch generator
    seeded with seed + b.  Returns a float32 tensor of batch * n^3 values."""
    import torch
    out = torch.zeros(batch, n, n, n, dtype=torch.float32, device=device)
    ax1 = torch.arange(n, device=device, dtype=torch.float32)
    gen = torch.Generator(device=device)
    for b in range(batch):
        g = _rng(seed, b)
        vol = out[b]
        for _ in range(int(g.integers(10, 31))):
            c = g.uniform(0.0, n, size=3)
            ax = g.uniform(0.05 * n, 0.35 * n, size=3)
            R = _rotation(g)
            rho = g.uniform(0.0, 1.0)
            half = np.sqrt(((R * ax[None, :]) ** 2).sum(1))
            lo = np.maximum(np.floor(c - half).astype(int), 0)
            hi = np.minimum(np.ceil(c + half).astype(int) + 1, n)
            if np.any(hi <= lo):
                continue
            A = torch.tensor(R / ax[None, :], dtype=torch.float32, device=device)
            p = torch.stack(torch.meshgrid(ax1[lo[0]:hi[0]], ax1[lo[1]:hi[1]], ax1[lo[2]:hi[2]],
                                           indexing="ij"), -1) - torch.tensor(c, dtype=torch.float32, device=device)
            q = p @ A
            vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += float(rho) * ((q * q).sum(-1) <= 1.0).float()
        gen.manual_seed(int(seed) + b)
        vol += noise * torch.randn(n, n, n, generator=gen, device=device)
    return out.reshape(-1)
