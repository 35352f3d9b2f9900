"""Rudder-propeller and tiltrotor classes (Sec. III-D actuator kinds: fins
with angle-of-attack lift and drag, servo-tilted propellers) and the RK4
variant on the GPU, against the FP64 oracle through the C-ABI.

Tolerances as for the plain step: per-env relative state error <= 1e-5 after
one control step from an identical FP32 state, <= 1e-3 over a trajectory.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import align_q, oracle_env_arrays, rel_state_err

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = 1e-5
TRAJ_TOL = 1e-3


def mixed_classes():
    """The three propulsion types plus two multirotor classes; heavy8 and the
    tiltrotor share 8 channels but not the step variant."""
    return vehicles.actuated_classes() + [vehicles.five_classes()[1], vehicles.five_classes()[3]]


def n_thr_of(classes, counts):
    return np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])


def integ_of(integrator):
    return 1 if integrator == B.MG_INTEG_RK4 else 0


@pytest.mark.parametrize("integrator", [B.MG_INTEG_EULER, B.MG_INTEG_RK4])
@pytest.mark.parametrize("counts,K,per_env", [([37, 50, 29, 5, 130], 4, True), ([64, 3, 128, 0, 9], 1, False),
                                              ([1, 129, 127, 4, 2], 8, True)])
def test_one_step_matches_oracle(counts, K, per_env, integrator):
    classes = mixed_classes()
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=per_env, reset=dict(vehicles.NO_DR),
                integrator=integrator)
    p = workloads.random_params(61 + K, classes, counts)
    if per_env:
        sim.set_params(B.dict_to_params(p, sim.n_envs))
    else:
        p = B.params_to_dict(sim.get_params())   # class values, no current
        p["rg"] = np.zeros((sim.n_envs, 3))
        p["cls"] = workloads.env_classes(counts)
    # Moving start: fins see a flow, servos and fins start deflected.
    s0 = workloads.random_states(62 + K, sim.n_envs, n_thr_of(classes, counts))
    sim.set_state(s0)
    a = workloads.actions(63, 1, sim.n_envs)
    sim.step(sim.pack_actions(a))
    torch.cuda.synchronize()
    gpu = sim.get_state()
    envs = oracle.make_envs(oracle_env_arrays(p))
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0.astype(np.float64), a, 0.01, K, integ=integ_of(integrator))
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, (err.max(), int(np.argmax(err)))
    slots = sim.slots_of_envs()
    np.testing.assert_allclose(sim.obs.cpu().numpy()[slots], o_ref[0], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(sim.reward.cpu().numpy()[slots], r_ref[0], rtol=1e-5, atol=1e-4)
    sim.status()
    sim.close()


@pytest.mark.parametrize("integrator", [B.MG_INTEG_EULER, B.MG_INTEG_RK4])
def test_trajectory_with_dr_and_current_matches_oracle(integrator):
    """300 steps from the hover-task reset with DR and current, K=4."""
    classes = mixed_classes()
    counts = [9, 12, 7, 5, 6]
    cfg = vehicles.HOVER_DR
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=dict(cfg), integrator=integrator)
    sim.reset(seed=19)
    envs, _ = oracle.reset(classes, workloads.env_classes(counts), cfg, 19)
    s_ref = sim.get_state().astype(np.float64)
    T, every = 300, 50
    a = workloads.actions(20, T, sim.n_envs)
    a_dev = sim.pack_actions(a)
    obs = torch.zeros(every, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(every, sim.n_slots, device="cuda")
    slots = sim.slots_of_envs()
    g_traj, r_traj = [], []
    for t0 in range(0, T, every):
        B.mg_rollout(sim.handle, a_dev[t0:t0 + every], every, obs, rew, False)
        torch.cuda.synchronize()
        g_traj.append(sim.get_state().astype(np.float64))
        s_ref, o_ref, r_ref = oracle.rollout(classes, envs, s_ref, a[t0:t0 + every], 0.01, 4,
                                             integ=integ_of(integrator))
        r_traj.append(s_ref.copy())
        np.testing.assert_allclose(obs.cpu().numpy()[:, slots], o_ref, rtol=1e-3, atol=1e-3)
        np.testing.assert_allclose(rew.cpu().numpy()[:, slots], r_ref, rtol=1e-3, atol=1e-2)
    g = align_q(np.stack(g_traj, 1), np.stack(r_traj, 1))
    r = np.stack(r_traj, 1)
    traj_err = np.linalg.norm(g - r, axis=-1).max(1) / np.maximum(np.linalg.norm(r, axis=-1).max(1), 1.0)
    assert traj_err.max() <= TRAJ_TOL, traj_err.max()
    sim.status()
    sim.close()


@pytest.mark.parametrize("integrator", [B.MG_INTEG_EULER, B.MG_INTEG_RK4])
def test_full_size_sampled(integrator):
    """1,048,576 envs of the three propulsion types (hover + DR, K=4): sampled
    envs after reset + one step against the oracle run on those envs alone."""
    classes = vehicles.actuated_classes()
    counts = workloads.class_counts(1 << 20, 3)
    cfg = vehicles.HOVER_DR
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=dict(cfg), integrator=integrator)
    sim.reset(seed=5)
    rng = np.random.default_rng(3)
    ids = np.sort(rng.choice(sim.n_envs, 1024, replace=False))
    ids = np.unique(np.concatenate([ids, [0, sim.n_envs - 1, counts[0], counts[0] + counts[1]]]))
    a_s = workloads.actions(9, 1, len(ids))
    a_env = np.zeros((1, sim.n_envs, 8), np.float32)
    a_env[:, ids] = a_s
    sim.step(sim.pack_actions(a_env))
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids]
    envs, s0 = oracle.reset(classes, workloads.env_classes(counts)[ids], cfg, 5, env_ids=ids)
    ref, o_ref, _ = oracle.rollout(classes, envs, s0, a_s, 0.01, 4, integ=integ_of(integrator))
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, err.max()
    slots = sim.slots_of_envs()[ids]
    np.testing.assert_allclose(sim.obs.cpu().numpy()[slots], o_ref[0], rtol=2e-5, atol=2e-5)
    sim.status()
    sim.close()


def test_rest_stays_rest_bit_exact_for_every_type_and_integrator():
    classes = vehicles.actuated_classes()
    for c in classes:
        c["rb"] = (0.0, 0.0, -0.02)
    counts = [5, 7, 9]
    for integrator in (B.MG_INTEG_EULER, B.MG_INTEG_RK4):
        sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=False, reset=dict(vehicles.NO_DR),
                    integrator=integrator)
        s0 = sim.get_state()
        sim.step(sim.new_actions(1) * 0.0, n_steps=1)
        B.mg_step(sim.handle, torch.zeros(30, sim.action_floats, device="cuda"), 30, None, None)
        torch.cuda.synchronize()
        assert np.array_equal(sim.get_state(), s0)
        sim.close()


@pytest.mark.parametrize("integrator", [B.MG_INTEG_EULER, B.MG_INTEG_RK4])
def test_fp64_check_path_matches_oracle(integrator):
    """The FP64 rollout of the check path (fins and tilted propellers with
    their FP64 tables, Euler or RK4) equals the oracle's FP64 rollout to near
    machine precision, from the same state and per-env parameters (current
    included)."""
    classes = mixed_classes()
    counts = [5, 6, 4, 3, 3]
    T, K = 30, 4
    cfg = vehicles.HOVER
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(cfg), integrator=integrator)
    # Parameters both sides hold exactly (the GPU stores them in FP32).
    p = workloads.random_params(23, classes, counts)
    sim.set_params(B.dict_to_params(p, sim.n_envs))
    envs = oracle.make_envs(oracle_env_arrays(p))
    s0 = workloads.random_states(24, sim.n_envs, n_thr_of(classes, counts), pos_scale=2.0, vel_scale=0.3)
    sim.set_state(s0)
    a = workloads.actions(25, T, sim.n_envs)
    rew = torch.zeros(T, sim.n_slots, dtype=torch.float64, device="cuda")
    s_end = torch.zeros(sim.n_slots, 21, dtype=torch.float64, device="cuda")
    B.mg_rollout_fp64(sim.handle, sim.pack_actions(a), T, reward=rew, state=s_end)
    torch.cuda.synchronize()
    slots = sim.slots_of_envs()
    ref_s, _, ref_r = oracle.rollout(classes, envs, s0.astype(np.float64), a, 0.01, K, integ=integ_of(integrator))
    np.testing.assert_allclose(rew.cpu().numpy()[:, slots], ref_r, rtol=1e-10, atol=1e-10)
    got = align_q(s_end.cpu().numpy()[slots], ref_s)
    np.testing.assert_allclose(got, ref_s, rtol=1e-10, atol=1e-10)
    sim.close()