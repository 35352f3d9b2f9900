"""Long-horizon GPU parity at the sizes of the heterogeneous, sweep and
differentiable-rollout workloads, against the FP64 oracle on the same seeded
inputs.

Tolerances (the stated trajectory bound): per env, the trajectory-relative
state error max_t |x_gpu(t) - x_ref(t)| / max(max_t |x_ref(t)|, 1) <= 1e-3
over 1000 control steps, with the observation and the reward held to the same
relative bound at every step compared; adjoint <= 1e-3 relative per env
against the oracle's forward-mode tangents over random directions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import align_q, oracle_env_arrays

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-3
DT, K = 0.01, 4


class TrajErr:
    """Running max over time of |gpu - ref| and |ref| per env (states,
    observations, rewards), for the trajectory-relative error."""

    def __init__(self, n):
        self.num = {k: np.zeros(n) for k in ("s", "o", "r")}
        self.den = {k: np.ones(n) for k in ("s", "o", "r")}

    def add(self, key, gpu, ref, axis=-1):
        g = np.asarray(gpu, np.float64)
        r = np.asarray(ref, np.float64)
        if key == "s":
            g = align_q(g, r)
        d = np.abs(g - r) if g.ndim == 1 else np.linalg.norm(g - r, axis=axis)
        m = np.abs(r) if r.ndim == 1 else np.linalg.norm(r, axis=axis)
        self.num[key] = np.maximum(self.num[key], d)
        self.den[key] = np.maximum(self.den[key], m)

    def err(self, key):
        return self.num[key] / self.den[key]


def test_heterogeneous_batch_1000_steps_through_the_captured_graph():
    """16,384 envs over the five classes, per-env DR and ocean current, hover
    initial poses, K = 4: 1000 steps as 20 replays of one captured 50-step
    rollout graph (the multi-step kernels that prefetch the next step's
    actions, one launch per class), observations and rewards every step."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(16384, 5)
    cfg = dict(vehicles.HOVER_DR)
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=True, reset=cfg)
    sim.reset(seed=0x4D47)
    E, S = sim.n_envs, 50
    slots = sim.slots_of_envs()
    a_dev = torch.zeros(S, sim.action_floats, device="cuda")
    obs = torch.zeros(S, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(S, sim.n_slots, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = B.mg_graph_capture(sim.handle, a_dev, S, obs, rew, stream=st)
    envs, s_ref = oracle.reset(classes, workloads.env_classes(counts), cfg, 0x4D47)
    te = TrajErr(E)
    for chunk in range(1000 // S):
        a = workloads.actions(1000 + chunk, S, E)
        with torch.cuda.stream(st):
            a_dev.copy_(sim.pack_actions(a))
            B.mg_graph_launch(g, stream=st)
        st.synchronize()
        s_ref, o_ref, r_ref = oracle.rollout(classes, envs, s_ref, a, DT, K)
        o = obs.cpu().numpy()[:, slots]
        r = rew.cpu().numpy()[:, slots]
        for t in range(S):
            te.add("o", o[t], o_ref[t])
            te.add("r", r[t], r_ref[t])
        te.add("s", sim.get_state(), s_ref)
    B.mg_graph_destroy(g)
    sim.status()
    sim.close()
    for key in ("s", "o", "r"):
        assert te.err(key).max() <= TRAJ_TOL, (key, te.err(key).max(), int(np.argmax(te.err(key))))


def test_sweep_size_1000_steps_multi_step_launches_sampled():
    """1,048,576 envs, five classes, class-constant hover step, K = 4: 1000
    steps as 20 launches of 50 steps; 2048 sampled envs (every class boundary
    included) run on the oracle with the same actions and reset draws."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(1 << 20, 5)
    cfg = dict(vehicles.HOVER)
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=False, reset=cfg)
    sim.reset(seed=77)
    E, S = sim.n_envs, 50
    rng = np.random.default_rng(78)
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 2048, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    ec = workloads.env_classes(counts)[ids]
    # Flat action index of (sampled env, thruster) in the per-class layout.
    lay = sim.layout
    env_off = np.array([lay.cls[c].env_offset for c in range(5)])
    act_off = np.array([lay.cls[c].action_offset for c in range(5)])
    nthr = np.array([classes[c]["n_thr"] for c in ec])
    local = ids - env_off[ec]
    rows, cols = np.nonzero(np.arange(8)[None, :] < nthr[:, None])
    flat = act_off[ec][rows] + local[rows] * nthr[rows] + cols
    flat_t = torch.from_numpy(flat).cuda()
    slots = sim.slots_of_envs()[ids]
    envs, s_ref = oracle.reset(classes, ec, cfg, 77, env_ids=ids)
    te = TrajErr(len(ids))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(79)
    for chunk in range(1000 // S):
        a_dev = torch.rand(S, sim.action_floats, device="cuda", generator=gen) * 2 - 1
        a_s = workloads.actions(2000 + chunk, S, len(ids))
        a_dev[:, flat_t] = torch.from_numpy(a_s[:, rows, cols]).cuda()
        B.mg_step(sim.handle, a_dev, S, sim.obs, sim.reward)
        torch.cuda.synchronize()
        s_ref, o_ref, r_ref = oracle.rollout(classes, envs, s_ref, a_s, DT, K)
        te.add("s", sim.get_state()[ids], s_ref)
        te.add("o", sim.obs.cpu().numpy()[slots], o_ref[-1])
        te.add("r", sim.reward.cpu().numpy()[slots], r_ref[-1])
    sim.status()
    sim.close()
    for key in ("s", "o", "r"):
        assert te.err(key).max() <= TRAJ_TOL, (key, te.err(key).max(), int(ids[np.argmax(te.err(key))]))


def test_adjoint_at_the_differentiable_rollout_size():
    """8192 envs over the five classes, per-env DR and current, T = 200,
    K = 4, a checkpoint every 20 steps: the launch shape of the full size
    (warp-sized blocks, class groups side by side). Gradients of 96 sampled
    envs (every class and every class boundary) against the oracle's tangents
    with the same parameters, states and actions."""
    from tests.test_gpu_adjoint import gpu_gradients
    classes = vehicles.five_classes()
    counts = workloads.class_counts(8192, 5)
    T = 200
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                record_steps=T, ckpt_every=20)
    sim.reset(seed=91)
    E = sim.n_envs
    s0 = sim.get_state()
    p_all = B.params_to_dict(sim.get_params())
    rng = np.random.default_rng(92)
    a = workloads.actions(93, T, E, lo=-0.99, hi=0.99)
    g_obs = (rng.normal(size=(T, E, 13)) * 0.1).astype(np.float32)
    g_rew = (-1.0 + 0.2 * rng.normal(size=(T, E))).astype(np.float32)
    g = gpu_gradients(sim, a, T, g_obs, g_rew, np.zeros((E, 21)))
    sim.close()
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 80, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    ec = workloads.env_classes(counts)[ids]
    assert set(ec.tolist()) == set(range(5)) and len(ids) >= 64
    p = {k: np.asarray(v)[ids] for k, v in p_all.items()}
    p["cls"], p["rg"] = ec, np.zeros((len(ids), 3))
    envs = oracle.make_envs(oracle_env_arrays(p))
    n = len(ids)
    nthr = np.array([classes[c]["n_thr"] for c in ec])
    thr_mask = (np.arange(8)[None, :] < nthr[:, None]).astype(np.float64)
    st_mask = (np.arange(21)[None, :] < (13 + nthr)[:, None]).astype(np.float64)
    go, gr = g_obs[:, ids].astype(np.float64), g_rew[:, ids].astype(np.float64)
    a_s = a[:, ids]
    groups = {"act": lambda: dict(d_actions=rng.normal(size=(T, n, 8)) * thr_mask[None]),
              "A": lambda: dict(d_Ma=rng.normal(size=(n, 6))),
              "dl": lambda: dict(d_dl=rng.normal(size=(n, 6))),
              "dq": lambda: dict(d_dq=rng.normal(size=(n, 6))),
              "s0": lambda: dict(d_state0=rng.normal(size=(n, 21)) * st_mask * 0.1)}
    for name, mk in groups.items():
        got, want = [], []
        for _ in range(3):
            d = mk()
            j = oracle.rollout_jvp(classes, envs, s0[ids].astype(np.float64), a_s, DT, K, **d)
            want.append(np.einsum("te,te->e", gr, j["d_reward"]) + np.einsum("tek,tek->e", go, j["d_obs"]))
            if name == "act":
                got.append(np.einsum("tek,tek->e", g["act"][:, ids], d["d_actions"]))
            elif name == "s0":
                got.append(np.einsum("ek,ek->e", g["s0"][ids], d["d_state0"]))
            else:
                key = {"A": "d_Ma", "dl": "d_dl", "dq": "d_dq"}[name]
                got.append(np.einsum("ek,ek->e", g[name][ids], d[key]))
        gv, rv = np.stack(got, 1), np.stack(want, 1)
        err = np.linalg.norm(gv - rv, axis=1) / np.maximum(np.linalg.norm(rv, axis=1), 1e-6)
        assert err.max() <= 1e-3, (name, err.max(), int(ids[np.argmax(err)]))
