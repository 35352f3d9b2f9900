"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module draws numbers and arranges them; it holds none of the step's
arithmetic. Actions are uniform on [-1, 1) on a 2^-23 grid, so a float32 value
is exact in both FP32 and FP64.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 0x4D47


def class_counts(n_envs: int, n_classes: int, multiple: int = 4) -> list:
    """Split n_envs uniformly over n_classes in multiples of `multiple` (last
    class takes the remainder)."""
    base = (n_envs // n_classes) // multiple * multiple
    counts = [base] * n_classes
    counts[-1] = n_envs - base * (n_classes - 1)
    return counts


def env_classes(counts) -> np.ndarray:
    """Class index per env, envs grouped contiguously by class."""
    return np.repeat(np.arange(len(counts), dtype=np.int32), counts)


def actions(seed: int, n_steps: int, n_envs: int, width: int = 8, lo: float = -1.0,
            hi: float = 1.0) -> np.ndarray:
    """[n_steps, n_envs, width] float32 uniform on [lo, hi) on a 2^-23 grid
    (lo, hi in [-1, 1])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, 1 << 24, size=(n_steps, n_envs, width), dtype=np.int64)
    a = (k.astype(np.float64) / float(1 << 23) - 1.0)
    a = lo + (hi - lo) * (a + 1.0) * 0.5 if (lo, hi) != (-1.0, 1.0) else a
    return a.astype(np.float32)


def random_states(seed: int, n_envs: int, n_thr: np.ndarray, pos_scale: float = 3.0,
                  vel_scale: float = 0.5, rate_scale: float = 0.8) -> np.ndarray:
    """[n_envs, 21] float32 states: p, unit-norm q (w, x, y, z), nu, rotor
    speeds n in [-1, 1] for the first n_thr entries, zeros after."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.zeros((n_envs, 21))
    s[:, 0:3] = rng.uniform(-pos_scale, pos_scale, (n_envs, 3))
    q = rng.normal(size=(n_envs, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    s[:, 3:7] = q
    s[:, 7:10] = rng.uniform(-vel_scale, vel_scale, (n_envs, 3))
    s[:, 10:13] = rng.uniform(-rate_scale, rate_scale, (n_envs, 3))
    n = rng.uniform(-1.0, 1.0, (n_envs, 8))
    n[np.arange(8)[None, :] >= np.asarray(n_thr)[:, None]] = 0.0
    s[:, 13:21] = n
    return s.astype(np.float32)


def random_params(seed: int, classes, counts, spread: float = 0.2, current: float = 0.5,
                  target_half: float = 5.0) -> dict:
    """Per-env physical parameters drawn around the class values, rounded to
    float32 so that FP32 and FP64 consumers read identical numbers.

    Returns a dict of arrays keyed mass, Ig, rb, W, B, Ma, dl, dq, Vc, target
    and cls (env order, envs grouped by class)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cls = env_classes(counts)
    n = len(cls)
    f = lambda shape: rng.uniform(1.0 - spread, 1.0 + spread, shape)
    pick = lambda key: np.array([classes[c][key] for c in cls], dtype=np.float64).reshape(n, -1)
    out = {}
    fm = f((n, 1))
    out["mass"] = (pick("mass") * fm)[:, 0]
    out["Ig"] = pick("Ig") * fm
    out["rb"] = pick("rb") * f((n, 1))
    # Weight and buoyancy near the class's nominal weight (slightly non-neutral).
    w0 = pick("mass")[:, 0] * 9.81
    out["W"] = out["mass"] * 9.81
    out["B"] = w0 * rng.uniform(0.97, 1.03, n)
    out["Ma"] = pick("Ma") * f((n, 6))
    out["dl"] = pick("dl") * f((n, 6))
    out["dq"] = pick("dq") * f((n, 6))
    psi = rng.uniform(0.0, 2.0 * np.pi, n)
    sp = rng.uniform(0.0, current, n)
    out["Vc"] = np.stack([sp * np.cos(psi), sp * np.sin(psi), np.zeros(n)], axis=1)
    out["target"] = rng.uniform(-target_half, target_half, (n, 3))
    for k in list(out):
        out[k] = out[k].astype(np.float32).astype(np.float64)
    out["cls"] = cls
    out["rg"] = np.zeros((n, 3))
    return out
