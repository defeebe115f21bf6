"""Seeded synthetic inputs shaped like the paper's hyperspectral workloads.

This module draws random numbers only: the sensing matrix Phi, the per-pixel
sparse coefficient vectors x (the paper's x in f = Psi x, Section II), the
additive measurement noise e and per-pixel sparsity levels.  It holds none of
the recovery method's arithmetic (no dictionary, no measurement, no solver), so
both the GPU library's tests and the FP64 oracle can consume the same inputs.

Host arrays come from numpy's PCG64 generator (bit-reproducible across
machines).  The ``*_torch`` variants draw the same distributions with a seeded
``torch.Generator`` on a chosen device, for cubes too large to build on the
host; their values differ from the numpy ones but are reproducible for a
given seed and device type.

Recipes (sizes and distributions of the cubes this library is exercised on):
  * Phi ~ N(0, 1/M) i.i.d.
  * "sparse": exactly S-sparse x, uniform random support; amplitudes N(0,1)
    ("normal") or +-(0.5 + |N(0,1)|) ("separated", bounded away from zero).
  * "powerlaw": compressible x with |x_k| = k^-decay for DCT index k = 1..N
    (low frequencies largest), random signs; optionally a random permutation.
  * noise e ~ N(0, var) i.i.d. per measurement.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def gaussian_phi(M: int, N: int, seed: int) -> np.ndarray:
    """Random sensing matrix Phi (M x N), entries N(0, 1/M), float64."""
    return _rng(seed, 1).standard_normal((M, N)) / np.sqrt(M)


def sparse_coeffs(P: int, N: int, S, seed: int, amplitude: str = "normal") -> np.ndarray:
    """P x N coefficient vectors, pixel p exactly S[p]-sparse (S scalar or per-pixel)."""
    rng = _rng(seed, 2)
    S = np.broadcast_to(np.asarray(S, dtype=np.int64), (P,))
    order = rng.random((P, N)).argsort(axis=1)
    if amplitude == "normal":
        amp = rng.standard_normal((P, N))
    elif amplitude == "separated":
        amp = (0.5 + np.abs(rng.standard_normal((P, N)))) * rng.choice([-1.0, 1.0], size=(P, N))
    else:
        raise ValueError(amplitude)
    X = np.zeros((P, N))
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(N)[None, :].repeat(P, 0), axis=1)
    mask = rank < S[:, None]
    X[mask] = amp[mask]
    return X


def powerlaw_coeffs(P: int, N: int, seed: int, decay: float = 1.5,
                    permute: bool = False) -> np.ndarray:
    """P x N compressible vectors, |x_k| = k^-decay (k = 1..N), random signs."""
    rng = _rng(seed, 3)
    mag = np.arange(1, N + 1, dtype=np.float64) ** (-decay)
    X = mag[None, :] * rng.choice([-1.0, 1.0], size=(P, N))
    if permute:
        perm = rng.random((P, N)).argsort(axis=1)
        X = np.take_along_axis(X, perm, axis=1)
    return X


def noise(P: int, M: int, var: float, seed: int) -> np.ndarray:
    """P x M measurement noise, i.i.d. N(0, var)."""
    if var == 0.0:
        return np.zeros((P, M))
    return _rng(seed, 4).standard_normal((P, M)) * np.sqrt(var)


def kappa_per_pixel(P: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Per-pixel sparsity levels, uniform on {lo, ..., hi}."""
    return _rng(seed, 5).integers(lo, hi + 1, size=P).astype(np.int16)


# --------------------------------------------------------------------------
# device-side variants (torch) for large cubes
# --------------------------------------------------------------------------
def _tgen(seed: int, stream: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + int(stream))
    return g


def powerlaw_coeffs_torch(P: int, N: int, seed: int, device, decay: float = 1.5):
    """Device tensor (float32) of P x N power-law vectors with random signs."""
    import torch
    g = _tgen(seed, 3, device)
    mag = torch.arange(1, N + 1, device=device, dtype=torch.float64).pow(-decay)
    sign = torch.randint(0, 2, (P, N), generator=g, device=device, dtype=torch.int8)
    return (mag[None, :] * (sign.double() * 2 - 1)).float()


def sparse_coeffs_torch(P: int, N: int, S, seed: int, device):
    """Device tensor (float32) of exactly S-sparse vectors (S scalar or per-pixel tensor)."""
    import torch
    g = _tgen(seed, 2, device)
    keys = torch.rand((P, N), generator=g, device=device)
    rank = keys.argsort(dim=1).argsort(dim=1)
    amp = torch.randn((P, N), generator=g, device=device)
    S_t = torch.as_tensor(S, device=device).reshape(-1, 1) if not np.isscalar(S) else S
    return torch.where(rank < S_t, amp, torch.zeros_like(amp)).float()


def noise_torch(P: int, M: int, var: float, seed: int, device):
    import torch
    g = _tgen(seed, 4, device)
    return (torch.randn((P, M), generator=g, device=device, dtype=torch.float32) *
            float(np.sqrt(var)))


# --------------------------------------------------------------------------
# workload recipes
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class CubeRecipe:
    name: str
    X: int            # spatial width
    Y: int            # spatial height
    N: int            # bands
    M: int            # measurements per pixel (0.4 N, i.e. 2.5x compression)
    coeffs: str       # "sparse" or "powerlaw"
    S: int = 8        # sparsity for "sparse"
    noise_var: float = 0.0

    @property
    def P(self) -> int:
        return self.X * self.Y


RECIPES = {
    # 32x32 pixels, N=120, M=48, exactly 8-sparse N(0,1) amplitudes, noiseless
    "small_sparse": CubeRecipe("small_sparse", 32, 32, 120, 48, "sparse", 8, 0.0),
    # 512x512 pixels, N=200, M=80, power-law spectra plus N(0, 1e-3) noise
    "fp32_powerlaw": CubeRecipe("fp32_powerlaw", 512, 512, 200, 80, "powerlaw", 0, 1e-3),
    # 1024x1024 pixels, N=224, M=90, same generator
    "precision_powerlaw": CubeRecipe("precision_powerlaw", 1024, 1024, 224, 90, "powerlaw", 0,
                                     1e-3),
    # 2048x2048 pixels, N=256, M=102, same generator
    "large_powerlaw": CubeRecipe("large_powerlaw", 2048, 2048, 256, 102, "powerlaw", 0, 1e-3),
}


def batch_recipe(seed: int = 1, n_cubes: int = 64):
    """64 cubes of uneven sizes: square side U{64..512}, N in {120, 200, 224},
    M = round(0.4 N), per-pixel sparsity S ~ U{4..32} (exactly sparse, noiseless)."""
    rng = _rng(seed, 6)
    sides = rng.integers(64, 513, size=n_cubes)
    bands = rng.choice([120, 200, 224], size=n_cubes)
    return [dict(side=int(s), N=int(n), M=int(round(0.4 * n))) for s, n in zip(sides, bands)]
