"""Seeded synthetic inputs for the stochastic Henry problem.

This module is the only code shared between the CUDA path's tests and the
FP64 oracle. It holds no arithmetic of the method: it only draws the random
vector xi ~ U[-1, 1]^M (the paper draws its xi_1..xi_3 independently and
uniformly on [-1, 1], section "Uncertain porosity and recharge") and builds
small synthetic per-cell log-permeability perturbations.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition: the state advances by the golden-ratio increment
0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 64-bit finaliser (shifts 30, 27, 31). One stream per
(seed, level, sample): the initial state is seed ^ (level << 40) ^ sample.

For quasi-Monte Carlo it also builds the Halton sequence (Halton, Numer.
Math. 2, 1960): coordinate j of point n is the radical inverse of n in the
j-th prime base (the base-b digits of n mirrored about the radix point),
optionally shifted modulo 1 by a seeded uniform vector (Cranley-Patterson
rotation) for independent randomised replicates.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 2403017018

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray, n: int) -> np.ndarray:
    """Return n outputs per stream; `state` is a uint64 array of stream states.

    Output shape is state.shape + (n,). Arithmetic wraps modulo 2**64.
    """
    s = np.array(state, dtype=np.uint64, copy=True)
    out = np.empty(s.shape + (n,), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for k in range(n):
            s = s + _GAMMA
            z = s.copy()
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            out[..., k] = z ^ (z >> np.uint64(31))
    return out


def uniform_pm1(bits: np.ndarray) -> np.ndarray:
    """Map 64-bit words to doubles in [-1, 1) using their top 53 bits."""
    u = (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def xi_batch(level: int, first_sample: int, count: int, n_xi: int = 3,
             seed: int = DEFAULT_SEED) -> np.ndarray:
    """xi for samples [first_sample, first_sample+count) of one MLMC level.

    Returns a C-contiguous float64 array of shape [count, n_xi]. Sample i of
    level l always gets the same xi, whatever batch it is drawn in.
    """
    if count < 0 or first_sample < 0 or level < 0:
        raise ValueError("level, first_sample and count must be >= 0")
    idx = np.arange(first_sample, first_sample + count, dtype=np.uint64)
    state = np.uint64(seed) ^ (np.uint64(level) << np.uint64(40)) ^ idx
    return np.ascontiguousarray(uniform_pm1(splitmix64(state, n_xi)))


def logk_perturbation(ny: int, nx: int, count: int, amplitude: float = 0.1,
                      seed: int = DEFAULT_SEED + 7) -> np.ndarray:
    """Per-cell log-permeability perturbations theta, shape [count, ny, nx].

    Uniform on [-amplitude, amplitude), one independent stream per cell and
    sample. Used to exercise the d/dlogK adjoint and field-dependent paths.
    """
    idx = np.arange(count * ny * nx, dtype=np.uint64)
    state = np.uint64(seed) ^ (np.uint64(0xA5) << np.uint64(48)) ^ idx
    vals = uniform_pm1(splitmix64(state, 1))[..., 0]
    return np.ascontiguousarray((amplitude * vals).reshape(count, ny, nx))


_PRIMES = (2, 3, 5, 7, 11, 13, 17, 19)


def radical_inverse(n: np.ndarray, base: int) -> np.ndarray:
    """phi_b(n) = sum_k d_k b^-(k+1) for n = sum_k d_k b^k, accumulated digit
    by digit (n >= 0 integers)."""
    n = np.array(n, dtype=np.int64, copy=True)
    out = np.zeros(n.shape, dtype=np.float64)
    f = 1.0 / base
    while np.any(n > 0):
        out += f * (n % base)
        n //= base
        f /= base
    return out


def halton(first: int, count: int, dim: int, shift_seed=None) -> np.ndarray:
    """Halton points with indices first..first+count-1 in [0,1)^dim, shape
    [count, dim]; with shift_seed, every coordinate is shifted by one seeded
    uniform number modulo 1 (the same shift for all points of a replicate)."""
    if dim > len(_PRIMES):
        raise ValueError(f"at most {len(_PRIMES)} dimensions")
    if first < 0 or count < 0:
        raise ValueError("first and count must be >= 0")
    idx = np.arange(first, first + count, dtype=np.int64)
    u = np.stack([radical_inverse(idx, _PRIMES[j]) for j in range(dim)], axis=1)
    if shift_seed is not None:
        sh = (uniform_pm1(splitmix64(np.array([np.uint64(shift_seed)]), dim)[0]) + 1.0) / 2.0
        u = np.mod(u + sh, 1.0)
    return np.ascontiguousarray(u)


def xi_halton(first: int, count: int, n_xi: int = 3, shift_seed=None) -> np.ndarray:
    """xi = 2u - 1 from Halton points u (indices from `first`; index 0, the
    corner xi = (-1, ..., -1), is usually skipped by starting at 1)."""
    return np.ascontiguousarray(2.0 * halton(first, count, n_xi, shift_seed) - 1.0)
