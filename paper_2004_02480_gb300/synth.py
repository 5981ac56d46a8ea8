"""Seeded synthetic inputs for CSK workloads.

The paper's experiments draw A and x* with MATLAB's ``randn`` and set
b = A x* (Section 3).  This module produces inputs with the same distribution
from a seeded numpy generator (PCG64); it holds none of the method's own
arithmetic (no hashing, sketching or iteration) and is the one module shared
by the oracle-side tests and the CUDA-side tests and benchmark.

Recipes (sizes are the caller's):

* :func:`gaussian_system`      -- A, x* iid N(0, 1), b = A x* formed in binary64,
                                  then stored in the requested dtype.
* :func:`conditioned_system`   -- A = G diag(sigma) Q with G iid N(0, 1), Q Haar
                                  orthogonal (QR of a Gaussian, column signs
                                  fixed by sign(diag R)), sigma log-spaced
                                  between 1 and ``kappa``.
* :func:`gaussian_multi_rhs`   -- A iid N(0, 1), X* (n x R) iid N(0, 1), B = A X*.
* :func:`batched_shapes`       -- (m, n) pairs with m log-uniform and n
                                  uniform-integer.
* :func:`noisy_system`         -- an inconsistent system: A, x* as in
                                  :func:`gaussian_system`, b = A x* + e with e
                                  iid N(0, (noise * rms(A x*))^2) from a second
                                  stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    A: np.ndarray          # (m, n) row-major, dtype as requested
    b: np.ndarray          # (m,) or (m, R)
    x_star: np.ndarray     # (n,) or (n, R), binary64


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), 0x2004_02480]))


def gaussian_system(m: int, n: int, seed: int, dtype=np.float64) -> System:
    """A, x* iid N(0,1); b = A x* computed in binary64 then cast to ``dtype``."""
    g = _rng(seed)
    A = g.standard_normal((m, n), dtype=np.float64 if dtype == np.float64 else np.float32)
    xs = g.standard_normal(n)
    b = A.astype(np.float64, copy=False) @ xs
    return System(np.ascontiguousarray(A, dtype=dtype), b.astype(dtype), xs)


def noisy_system(m: int, n: int, seed: int, noise: float, dtype=np.float64) -> System:
    """A, x* as gaussian_system(m, n, seed); b = A x* + e, e iid Gaussian with
    standard deviation noise * rms(A x*), drawn from a stream of its own; b in
    binary64 then cast.  x_star is the x* the noise was added to (no longer a
    solution)."""
    s = gaussian_system(m, n, seed, dtype)
    g = np.random.default_rng(np.random.SeedSequence([int(seed), 0x2004_02480, 1]))
    ax = s.A.astype(np.float64, copy=False) @ s.x_star
    b = ax + noise * np.sqrt(np.mean(ax * ax)) * g.standard_normal(m)
    return System(s.A, b.astype(dtype), s.x_star)


def gaussian_multi_rhs(m: int, n: int, R: int, seed: int, dtype=np.float32) -> System:
    """A iid N(0,1), X* (n x R) iid N(0,1), B = A X* in binary64 then cast."""
    g = _rng(seed)
    A = g.standard_normal((m, n), dtype=np.float64 if dtype == np.float64 else np.float32)
    X = g.standard_normal((n, R))
    B = A.astype(np.float64, copy=False) @ X
    return System(np.ascontiguousarray(A, dtype=dtype), np.ascontiguousarray(B.astype(dtype)), X)


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    Z = g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def conditioned_system(m: int, n: int, seed: int, kappa: float = 1e3,
                       dtype=np.float32, block: int = 65536) -> System:
    """A = G diag(sigma) Q, sigma_i = kappa^(i/(n-1)); b = A x* (binary64)."""
    g = _rng(seed)
    Q = haar_orthogonal(n, g)
    sig = kappa ** (np.arange(n) / max(n - 1, 1))
    M = sig[:, None] * Q                      # diag(sigma) Q
    xs = g.standard_normal(n)
    A = np.empty((m, n), dtype)
    b = np.empty(m, dtype)
    for s in range(0, m, block):
        e = min(m, s + block)
        Gb = g.standard_normal((e - s, n))
        Ab = Gb @ M
        A[s:e] = Ab
        b[s:e] = Ab.astype(dtype).astype(np.float64) @ xs
    return System(A, b, xs)


def batched_shapes(S: int, m_lo: int, m_hi: int, n_lo: int, n_hi: int, seed: int):
    """S shapes: m log-uniform in [m_lo, m_hi], n uniform integer in [n_lo, n_hi]."""
    g = _rng(seed)
    m = np.exp(g.uniform(np.log(m_lo), np.log(m_hi), S)).astype(np.int64)
    n = g.integers(n_lo, n_hi + 1, S)
    return [(int(a), int(c)) for a, c in zip(m, n)]


def conditioned_system_device(m: int, n: int, seed: int, kappa: float = 1e3, device="cuda",
                              block: int = 131072):
    """conditioned_system() drawn on a torch device (for sizes where host
    generation is slow): A = G diag(sigma) Q in FP32, G from a seeded torch
    generator on the device, Q Haar (host QR), x* N(0,1), b = A x* with
    binary64 accumulation.  Returns (A, b, x_star) torch tensors."""
    import torch
    g = _rng(seed)
    Q = haar_orthogonal(n, g)
    sig = kappa ** (np.arange(n) / max(n - 1, 1))
    M = torch.from_numpy(sig[:, None] * Q).to(device=device, dtype=torch.float32)
    xs = torch.from_numpy(g.standard_normal(n)).to(device)
    tg = torch.Generator(device=device).manual_seed(int(seed) * 7919 + 17)
    A = torch.empty((m, n), dtype=torch.float32, device=device)
    b = torch.empty(m, dtype=torch.float32, device=device)
    for s in range(0, m, block):
        e = min(m, s + block)
        Gb = torch.randn((e - s, n), generator=tg, device=device, dtype=torch.float32)
        A[s:e] = Gb @ M
        b[s:e] = (A[s:e].double() @ xs).float()
    return A, b, xs
