"""Shared helpers of the test-suite (comparison metrics, input plumbing)."""
import numpy as np


def align_q(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Flip the quaternion (entries 3:7) of gpu states to the sign of ref (q and -q
    are the same attitude)."""
    g = np.array(gpu, dtype=np.float64, copy=True)
    s = np.sign(np.sum(g[..., 3:7] * ref[..., 3:7], axis=-1, keepdims=True))
    s[s == 0] = 1.0
    g[..., 3:7] *= s
    return g


def rel_state_err(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-env ||x_gpu - x_ref|| / max(||x_ref||, 1) over the sign-aligned state."""
    g = align_q(gpu, ref)
    return np.linalg.norm(g - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1.0)


def oracle_env_arrays(p: dict) -> dict:
    """Per-env parameter dict (workloads.random_params keys) -> oracle env arrays."""
    keys = ("mass", "Ig", "rg", "rb", "W", "B", "Ma", "dl", "dq", "Vc", "target", "cls")
    return {k: p[k] for k in keys}
