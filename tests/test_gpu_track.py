"""Trajectory-tracking task on the GPU (Sec. IV-B): reset draws of the
reference, observations and rewards against p*(t), the per-env step counter
and the adjoint, all against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import oracle_env_arrays

pytestmark = pytest.mark.gpu


def make(counts, cfg, K=4, per_env=True, **kw):
    classes = vehicles.five_classes()[:len(counts)]
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=per_env, reset=cfg, task=B.TASK_TRACK, **kw)
    return classes, sim


@pytest.mark.parametrize("cfg", [vehicles.TRACK_HELIX, vehicles.TRACK_LISSAJOUS, vehicles.TRACK_HELIX_DR])
def test_reset_and_rollout_match_oracle(cfg):
    counts = [9, 4, 13, 6, 5]
    per_env = bool(cfg.get("dr_enabled"))
    classes, sim = make(counts, cfg, per_env=per_env)
    sim.reset(seed=31)
    envs, s0 = oracle.reset(classes, workloads.env_classes(counts), cfg, 31)
    ref = oracle.envs_to_arrays(envs)
    task = sim.get_task()
    for name, sl in (("target", slice(0, 3)), ("traj_a", slice(3, 6)), ("traj_w", slice(6, 9)),
                     ("traj_phi", slice(9, 12)), ("traj_v", slice(12, 15))):
        np.testing.assert_allclose(task[:, sl], ref[name], rtol=2e-7, atol=2e-7, err_msg=name)
    assert np.all(task[:, 15] == 0.0)
    T = 40
    a = workloads.actions(5, T, sim.n_envs)
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    sim.rollout(sim.pack_actions(a), T, obs, rew)
    torch.cuda.synchronize()
    _, o_ref, r_ref = oracle.rollout(classes, envs, s0, a, 0.01, 4)
    slots = sim.slots_of_envs()
    np.testing.assert_allclose(obs.cpu().numpy()[:, slots], o_ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(rew.cpu().numpy()[:, slots], r_ref, rtol=1e-4, atol=1e-3)
    assert np.all(sim.get_task()[:, 15] == T)
    sim.status()
    sim.close()


def test_step_counter_continues_time_across_calls():
    counts = [8, 8, 8, 8, 8]
    classes, sim = make(counts, vehicles.TRACK_LISSAJOUS, per_env=False)
    sim.reset(seed=4)
    envs, s = oracle.reset(classes, workloads.env_classes(counts), vehicles.TRACK_LISSAJOUS, 4)
    arr = oracle.envs_to_arrays(envs)
    a = workloads.actions(8, 30, sim.n_envs)
    a_dev = sim.pack_actions(a)
    B.mg_step(sim.handle, a_dev[:20], 20, None, None)
    sim.step(a_dev[20:30], n_steps=10)
    torch.cuda.synchronize()
    s, _, _ = oracle.rollout(classes, envs, s, a[:20], 0.01, 4, obs=False)
    arr["k0"] = np.full(sim.n_envs, 20.0)
    s, o, r = oracle.rollout(classes, oracle.make_envs(arr), s, a[20:30], 0.01, 4)
    slots = sim.slots_of_envs()
    last = sim.obs.cpu().numpy()[slots].copy()
    np.testing.assert_allclose(last, o[-1], rtol=1e-4, atol=1e-4)
    assert np.all(sim.get_task()[:, 15] == 30)
    # Observation without a step reads the reference at the current counter:
    # identical to the last step's observation.
    o0 = sim.observe().cpu().numpy()[slots]
    np.testing.assert_array_equal(o0, last)
    sim.close()


def test_task_roundtrip_and_validation():
    counts = [4, 4, 4, 4, 4]
    classes, sim = make(counts, vehicles.TRACK_HELIX, per_env=True)
    sim.reset(seed=2)
    t = sim.get_task()
    t[:, 15] = 123.0
    sim.set_task(t)
    p = sim.get_params()
    sim.set_params(p)                       # keeps the step counter
    assert np.array_equal(sim.get_task(), t)
    hover = B.Sim(classes, counts, dt=0.01, K=1, per_env_params=False, reset=dict(vehicles.HOVER))
    th = hover.get_task()
    th[0, 4] = 1.0
    with pytest.raises(B.MGError) as e:
        hover.set_task(th)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    sim.close()
    hover.close()


def test_adjoint_in_tracking_mode_matches_oracle_tangents():
    counts = [3, 3, 3, 3, 3]
    T, K = 25, 2
    classes, sim = make(counts, vehicles.TRACK_HELIX, K=K, per_env=True, record_steps=T, ckpt_every=7)
    sim.reset(seed=9)
    p = workloads.random_params(3, classes, counts)
    task = sim.get_task()
    p["target"] = task[:, 0:3]
    sim.set_params(B.dict_to_params(p, sim.n_envs))
    nthr = np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])
    s0 = workloads.random_states(4, sim.n_envs, nthr, pos_scale=2.0, vel_scale=0.3, rate_scale=0.4)
    sim.set_state(s0)
    a = workloads.actions(5, T, sim.n_envs, lo=-0.99, hi=0.99)
    a_dev = sim.pack_actions(a)
    E, ns = sim.n_envs, sim.n_slots
    slots = sim.slots_of_envs()
    B.mg_rollout(sim.handle, a_dev, T, None, None, True)
    rng = np.random.default_rng(1)
    g_obs = rng.normal(size=(T, E, 13)) * 0.1
    g_rew = -np.ones((T, E))
    go = torch.zeros(T, ns, 13); go[:, slots] = torch.from_numpy(g_obs).float()
    gr = torch.zeros(T, ns); gr[:, slots] = torch.from_numpy(g_rew).float()
    g_act = torch.zeros(T, sim.action_floats, device="cuda")
    gA = torch.zeros(ns, 6, device="cuda")
    B.mg_step_backward(sim.handle, a_dev, go.cuda(), gr.cuda(), None, g_act, gA, None, None)
    torch.cuda.synchronize()
    ga = sim.unpack_actions(g_act).astype(np.float64)
    gAn = gA.cpu().numpy()[slots].astype(np.float64)
    arr = oracle_env_arrays(p)
    for k in ("traj_a", "traj_w", "traj_phi", "traj_v"):
        arr[k] = task[:, {"traj_a": 3, "traj_w": 6, "traj_phi": 9, "traj_v": 12}[k]:][:, :3]
    envs = oracle.make_envs(arr)
    thr_mask = (np.arange(8)[None, :] < nthr[:, None]).astype(np.float64)
    for _ in range(2):
        da = rng.normal(size=(T, E, 8)) * thr_mask[None]
        dA = rng.normal(size=(E, 6))
        j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, 0.01, K, d_actions=da, d_Ma=dA)
        ref = np.einsum("te,te->e", g_rew, j["d_reward"]) + np.einsum("tek,tek->e", g_obs, j["d_obs"])
        got = np.einsum("tek,tek->e", ga, da) + np.einsum("ek,ek->e", gAn, dA)
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)
        assert err.max() <= 1e-3, err.max()
    sim.close()
