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


def adjoint_vs_oracle_tangents(classes, sub_envs, s0, a, dt, K, g, go, gr, nthr, ids, rng, tol=1e-3, integ=0):
    """Per env: <gpu gradient, d> against the oracle's tangent of
    sum_t <g_obs, obs_t> + <g_rew, rew_t> along d, for three directions per
    gradient group (g: the GPU gradients of all envs; sub_envs: the oracle's
    records of the envs `ids`). Per env the relative error over the directions
    is at most `tol`. integ: the integrator (0 semi-implicit Euler, 1 RK4)."""
    import oracle
    n = len(ids)
    T = a.shape[0]
    thr_mask = (np.arange(8)[None, :] < nthr[ids][:, None]).astype(np.float64)
    st_mask = (np.arange(21)[None, :] < (13 + nthr[ids])[:, None]).astype(np.float64)
    groups = {"act": lambda: dict(d_actions=rng.normal(size=(T, n, 8)) * thr_mask[None]),
              "A": lambda: dict(d_Ma=rng.normal(size=(n, 6))),
              "dl": lambda: dict(d_dl=rng.normal(size=(n, 6))),
              "dq": lambda: dict(d_dq=rng.normal(size=(n, 6))),
              "s0": lambda: dict(d_state0=rng.normal(size=(n, 21)) * st_mask * 0.1)}
    for name, mk in groups.items():
        got, want = [], []
        for _ in range(3):
            d = mk()
            j = oracle.rollout_jvp(classes, sub_envs, s0[ids].astype(np.float64), a[:, ids], dt, K, integ=integ, **d)
            want.append(np.einsum("te,te->e", gr[:, ids], j["d_reward"]) +
                        np.einsum("tek,tek->e", go[:, ids], j["d_obs"]))
            if name == "act":
                got.append(np.einsum("tek,tek->e", g["act"][:, ids], d["d_actions"]))
            elif name == "s0":
                got.append(np.einsum("ek,ek->e", g["s0"][ids], d["d_state0"]))
            else:
                key = {"A": "d_Ma", "dl": "d_dl", "dq": "d_dq"}[name]
                got.append(np.einsum("ek,ek->e", g[name][ids], d[key]))
        gv, rv = np.stack(got, 1), np.stack(want, 1)
        err = np.linalg.norm(gv - rv, axis=1) / np.maximum(np.linalg.norm(rv, axis=1), 1e-6)
        assert err.max() <= tol, (name, err.max(), int(ids[np.argmax(err)]))


def fp64_reward_differences(sim, a_dev, T, dA, ddl, ddq, eps=1e-6):
    """Per env, the central difference of the summed rewards of the FP64
    check path (mg_rollout_fp64) along (dA, ddl, ddq) [n_envs][6] each, from
    the simulator's current state."""
    import torch
    from paper_2503_09203_b300 import binding as B
    slots = sim.slots_of_envs()

    def to_slots(x):
        out = np.zeros((sim.n_slots, 6))
        out[slots] = x
        return torch.from_numpy(out).cuda()

    d = [to_slots(x) for x in (dA, ddl, ddq)]
    r_p = torch.zeros(T, sim.n_slots, dtype=torch.float64, device="cuda")
    r_m = torch.zeros_like(r_p)
    B.mg_rollout_fp64(sim.handle, a_dev, T, d[0], d[1], d[2], eps, r_p)
    B.mg_rollout_fp64(sim.handle, a_dev, T, d[0], d[1], d[2], -eps, r_m)
    torch.cuda.synchronize()
    return ((r_p - r_m).cpu().numpy()[:, slots] / (2 * eps)).sum(0)
