"""GPU parity of the lane-pair step kernel (two lanes per env: the linear and
the angular rows of Eq. 1-3 on two lanes) against the FP64 oracle, and its
agreement with the one-lane kernel.

Tolerances as for the one-lane kernel: one-step relative state error
<= 1e-5; observations and rewards of a 25-step rollout within 1e-4. The two
kernels sum the equation's terms in different orders, so they agree to
rounding, not bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import rel_state_err

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = 1e-5


def classes_with_dead_zone():
    cl = vehicles.five_classes()
    cl[4] = dict(cl[4], deadzone=[0.25] * 6)   # one class takes the dead-zone path
    return cl


@pytest.mark.parametrize("per_env", [False, True])
def test_pair_one_step_matches_oracle(per_env):
    """540k envs: large enough for one launch per class even for a single
    step, so every launch runs on the lane-pair kernel; sampled envs (every
    class boundary included) against the oracle."""
    classes = classes_with_dead_zone()
    counts = [300001, 3, 240001, 5, 9]
    cfg = dict(vehicles.HOVER_DR if per_env else vehicles.HOVER)
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=per_env, reset=cfg)
    assert sim.launches_per_step() == 5
    sim.reset(seed=61)
    s0 = sim.get_state()
    E = sim.n_envs
    rng = np.random.default_rng(62)
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 1500, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    a_s = workloads.actions(63, 1, len(ids))
    a_env = np.zeros((1, E, 8), np.float32)
    a_env[:, ids] = a_s
    a_dev = sim.pack_actions(a_env)
    out = {}
    for lanes in (1, 2):
        B.mg_set_launch_shape(sim.handle, lanes, 0)
        sim.set_state(s0)
        sim.step(a_dev)
        torch.cuda.synchronize()
        out[lanes] = (sim.get_state(), sim.obs.cpu().numpy().copy(), sim.reward.cpu().numpy().copy())
    sim.status()
    assert B.mg_get_launch_shape(sim.handle)["envs_per_block"] == 64
    slots = sim.slots_of_envs()
    sim.close()
    envs, s_ref0 = oracle.reset(classes, workloads.env_classes(counts)[ids], cfg, 61, env_ids=ids)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0[ids].astype(np.float64), a_s, 0.01, 4)
    gpu2 = out[2][0][ids]
    err = rel_state_err(gpu2, ref)
    assert err.max() <= ONE_STEP_TOL, (err.max(), int(ids[np.argmax(err)]))
    np.testing.assert_allclose(out[2][1][slots[ids]], o_ref[0], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(out[2][2][slots[ids]], r_ref[0], rtol=1e-5, atol=1e-4)
    # Every env (not only the sampled ones) agrees with the one-lane kernel to
    # rounding; the kernels differ (not bit-identical), so the pair one ran.
    e12 = rel_state_err(out[2][0], out[1][0].astype(np.float64))
    assert e12.max() <= 2e-6 and not np.array_equal(out[2][0], out[1][0])
    pad = np.setdiff1d(np.arange(len(out[2][2])), slots)
    assert np.all(out[2][1][pad] == 0) and np.all(out[2][2][pad] == 0)


def test_pair_rollout_with_observations_every_step_matches_oracle():
    """The heterogeneous batch (16,384 envs, five classes, DR and current,
    K = 4): a 25-step rollout with observations and rewards every step takes
    one launch per class (multi-step launches), on the lane-pair kernel."""
    classes = classes_with_dead_zone()
    counts = workloads.class_counts(16384, 5)
    cfg = dict(vehicles.HOVER_DR)
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=cfg)
    sim.reset(seed=64)
    B.mg_set_launch_shape(sim.handle, 2, 0)
    T = 25
    a = workloads.actions(65, T, sim.n_envs)
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    sim.rollout(sim.pack_actions(a), T, obs, rew)
    torch.cuda.synchronize()
    gpu = sim.get_state()
    sim.status()
    slots = sim.slots_of_envs()
    sim.close()
    envs, s0 = oracle.reset(classes, workloads.env_classes(counts), cfg, 64)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0, a, 0.01, 4)
    np.testing.assert_allclose(obs.cpu().numpy()[:, slots], o_ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(rew.cpu().numpy()[:, slots], r_ref, rtol=1e-4, atol=1e-3)
    assert rel_state_err(gpu, ref).max() <= 25 * ONE_STEP_TOL


def test_autotune_shape_keeps_results_within_rounding():
    """The autotuner's choice (lanes per env and grid) changes where the
    arithmetic runs, not what it computes."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(16384, 5)
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=66)
    s0 = sim.get_state()
    T = 20
    a_dev = sim.pack_actions(workloads.actions(67, T, sim.n_envs))
    sim.rollout(a_dev, T)
    torch.cuda.synchronize()
    ref = sim.get_state()
    sim.set_state(s0)
    shape = B.mg_autotune(sim.handle, T)
    assert np.array_equal(sim.get_state(), s0)
    sim.rollout(a_dev, T)
    torch.cuda.synchronize()
    assert rel_state_err(sim.get_state(), ref.astype(np.float64)).max() <= 20 * 2e-6, shape
    with pytest.raises(B.MGError) as e:
        B.mg_set_launch_shape(sim.handle, 4, 0)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    sim.status()
    sim.close()


def test_gradients_of_a_rollout_recorded_on_the_pair_kernel():
    """A rollout recorded with two lanes per env (its checkpoints come from
    the lane-pair kernel) differentiates to the oracle's tangents."""
    from tests.test_gpu_adjoint import gpu_gradients
    from tests.helpers import oracle_env_arrays
    classes = vehicles.five_classes()
    counts = [5, 4, 6, 3, 4]
    T, K = 24, 4
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                record_steps=T, ckpt_every=8)
    B.mg_set_launch_shape(sim.handle, 2, 0)
    p = workloads.random_params(71, classes, counts)
    sim.set_params(B.dict_to_params(p, sim.n_envs))
    nthr = np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])
    s0 = workloads.random_states(72, sim.n_envs, nthr, pos_scale=2.0, vel_scale=0.3, rate_scale=0.4)
    sim.set_state(s0)
    a = workloads.actions(73, T, sim.n_envs, lo=-0.99, hi=0.99)
    E = sim.n_envs
    rng = np.random.default_rng(74)
    g_rew = -np.ones((T, E))
    g = gpu_gradients(sim, a, T, np.zeros((T, E, 13)), g_rew, np.zeros((E, 21)))
    envs = oracle.make_envs(oracle_env_arrays(p))
    thr_mask = (np.arange(8)[None, :] < nthr[:, None]).astype(np.float64)
    for name in ("act", "A", "dq"):
        got, want = [], []
        for _ in range(3):
            if name == "act":
                d = dict(d_actions=rng.normal(size=(T, E, 8)) * thr_mask[None])
            elif name == "A":
                d = dict(d_Ma=rng.normal(size=(E, 6)))
            else:
                d = dict(d_dq=rng.normal(size=(E, 6)))
            j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, 0.01, K, **d)
            want.append(np.einsum("te,te->e", g_rew, j["d_reward"]))
            key = {"act": "d_actions", "A": "d_Ma", "dq": "d_dq"}[name]
            got.append(np.einsum("tek,tek->e", g[name], d[key]) if name == "act"
                       else np.einsum("ek,ek->e", g[name], d[key]))
        gv, rv = np.stack(got, 1), np.stack(want, 1)
        err = np.linalg.norm(gv - rv, axis=1) / np.maximum(np.linalg.norm(rv, axis=1), 1e-6)
        assert err.max() <= 1e-3, (name, err.max())
    sim.close()
