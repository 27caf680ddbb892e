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
