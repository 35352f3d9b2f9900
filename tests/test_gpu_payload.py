"""Payload disturbance on the GPU (Sec. III-B mission payloads, Table 2 payload
mass): reset draws, the full-inertia step (off-origin CoG, 6x6 inverse) and
the payload setters, all against the FP64 oracle through the C-ABI.

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
from tests.helpers import align_q, rel_state_err

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = 1e-5
TRAJ_TOL = 1e-3


def make(counts, cfg, K=4, **kw):
    classes = vehicles.five_classes()[:len(counts)]
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(cfg), payload=True, **kw)
    return classes, sim


def n_thr_of(classes, counts):
    return np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])


@pytest.mark.parametrize("counts,K,cfg", [([37, 1, 0, 130, 5], 4, vehicles.PAYLOAD_DR),
                                          ([129, 128, 127, 4, 256], 2, vehicles.PAYLOAD),
                                          ([1024], 1, vehicles.PAYLOAD_DR)])
def test_one_step_with_payload_matches_oracle(counts, K, cfg):
    classes, sim = make(counts, cfg, K=K)
    sim.reset(seed=41)
    envs, _ = oracle.reset(classes, workloads.env_classes(counts), cfg, 41)
    ref_par = oracle.envs_to_arrays(envs)
    # The combined body: vehicle (mg_get_params) plus payload (mg_get_payload).
    veh = B.params_to_dict(sim.get_params())
    pay = sim.get_payload()
    assert pay[:, 0].max() > 0
    np.testing.assert_allclose(veh["mass"] + pay[:, 0], ref_par["mass"], rtol=1e-6)
    np.testing.assert_allclose(pay[:, :1] * pay[:, 1:] / ref_par["mass"][:, None], ref_par["rg"], rtol=1e-5, atol=1e-8)
    # Moving start (velocities and rotor speeds), identical FP32 state on both sides.
    s0 = workloads.random_states(43, sim.n_envs, n_thr_of(classes, counts))
    sim.set_state(s0)
    a = workloads.actions(7, 1, sim.n_envs)
    sim.step(sim.pack_actions(a))
    torch.cuda.synchronize()
    gpu = sim.get_state()
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0.astype(np.float64), a, 0.01, K)
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, (err.max(), np.argmax(err))
    slots = sim.slots_of_envs()
    np.testing.assert_allclose(sim.obs.cpu().numpy()[slots], o_ref[0], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(sim.reward.cpu().numpy()[slots], r_ref[0], rtol=1e-5, atol=1e-4)
    sim.status()
    sim.close()


def test_payload_trajectory_matches_oracle():
    """300 steps from the hover-task reset with payload and DR (current on)."""
    counts = [9, 4, 13, 6, 5]
    cfg = vehicles.PAYLOAD_DR
    classes, sim = make(counts, cfg, K=4)
    sim.reset(seed=7)
    envs, s_ref = oracle.reset(classes, workloads.env_classes(counts), cfg, 7)
    s0 = sim.get_state().astype(np.float64)
    np.testing.assert_allclose(s0[:, :13], s_ref[:, :13], rtol=2e-7, atol=1e-7)
    s_ref = s0.copy()
    T, every = 300, 50
    a = workloads.actions(8, T, sim.n_envs)
    a_dev = sim.pack_actions(a)
    obs = torch.zeros(every, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(every, sim.n_slots, device="cuda")
    slots = sim.slots_of_envs()
    g_traj, r_traj = [], []
    for t0 in range(0, T, every):
        B.mg_rollout(sim.handle, a_dev[t0:t0 + every], every, obs, rew, False)
        torch.cuda.synchronize()
        g_traj.append(sim.get_state().astype(np.float64))
        s_ref, o_ref, r_ref = oracle.rollout(classes, envs, s_ref, a[t0:t0 + every], 0.01, 4)
        r_traj.append(s_ref.copy())
        np.testing.assert_allclose(obs.cpu().numpy()[:, slots], o_ref, rtol=1e-3, atol=1e-3)
        np.testing.assert_allclose(rew.cpu().numpy()[:, slots], r_ref, rtol=1e-3, atol=1e-2)
    g = np.stack(g_traj, 1)
    r = np.stack(r_traj, 1)
    g = align_q(g, r)
    traj_err = np.linalg.norm(g - r, axis=-1).max(1) / np.maximum(np.linalg.norm(r, axis=-1).max(1), 1.0)
    assert traj_err.max() <= TRAJ_TOL, traj_err.max()
    sim.status()
    sim.close()


def test_full_size_payload_sampled():
    """1,048,576 envs, 5 classes, payload + DR, K=4: a sampled set of envs after
    reset + one step against the oracle run on those envs alone."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(1 << 20, 5)
    cfg = vehicles.PAYLOAD_DR
    _, sim = make(counts, cfg, K=4)
    sim.reset(seed=5)
    rng = np.random.default_rng(1)
    ids = np.sort(rng.choice(sim.n_envs, 2048, replace=False))
    ids = np.unique(np.concatenate([ids, [0, sim.n_envs - 1] + [sum(counts[:c]) for c in range(1, 5)]]))
    a_s = workloads.actions(9, 1, len(ids))
    a_env = np.zeros((1, sim.n_envs, 8), np.float32)
    a_env[:, ids] = a_s
    sim.step(sim.pack_actions(a_env))
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids]
    ec = workloads.env_classes(counts)[ids]
    envs, s0 = oracle.reset(classes, ec, cfg, 5, env_ids=ids)
    ref, o_ref, _ = oracle.rollout(classes, envs, s0, a_s, 0.01, 4)
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, err.max()
    slots = sim.slots_of_envs()[ids]
    np.testing.assert_allclose(sim.obs.cpu().numpy()[slots], o_ref[0], rtol=2e-5, atol=2e-5)
    sim.status()
    sim.close()


def test_zero_payload_equals_plain_per_env_step():
    """m_p = 0 through the full-inertia path gives the diagonal path's result."""
    counts = [64, 33, 1, 40, 70]
    cfg = dict(vehicles.PAYLOAD_DR, payload_lo=0.0, payload_hi=0.0)
    classes, sim = make(counts, cfg, K=4)
    plain = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=dict(vehicles.HOVER_DR))
    s0 = workloads.random_states(3, sim.n_envs, n_thr_of(classes, counts))
    for s in (sim, plain):
        s.reset(seed=11)
        s.set_state(s0)
    a = workloads.actions(12, 50, sim.n_envs)
    for s in (sim, plain):
        s.rollout(s.pack_actions(a), 50)
    torch.cuda.synchronize()
    assert np.all(sim.get_payload()[:, 0] == 0.0)
    err = rel_state_err(sim.get_state(), plain.get_state().astype(np.float64))
    assert err.max() <= 1e-5, err.max()
    sim.close()
    plain.close()


def test_set_payload_and_set_params_recompute_the_combined_body():
    counts = [17, 5, 9, 3, 6]
    cfg = vehicles.PAYLOAD_DR
    classes, sim = make(counts, cfg, K=4)
    sim.reset(seed=23)
    n = sim.n_envs
    rng = np.random.default_rng(2)
    veh = B.params_to_dict(sim.get_params())
    pay = np.zeros((n, 4))
    pay[:, 0] = veh["mass"] * rng.uniform(0.0, 0.4, n)
    pay[:, 1:] = rng.uniform(-0.15, 0.15, (n, 3))
    sim.set_payload(pay)
    np.testing.assert_allclose(sim.get_payload(), pay, rtol=1e-7, atol=1e-8)
    # New hydrodynamics through set_params: the payload stays attached.
    p = sim.get_params()
    p[:, 9:15] *= rng.uniform(0.8, 1.2, (n, 6))
    sim.set_params(p)
    np.testing.assert_allclose(sim.get_payload(), pay, rtol=1e-7, atol=1e-8)
    s0 = workloads.random_states(29, n, n_thr_of(classes, counts))
    sim.set_state(s0)
    a = workloads.actions(30, 1, n)
    sim.step(sim.pack_actions(a))
    torch.cuda.synchronize()
    # Oracle: the vehicle as stored (FP32 values), then the same payload.
    d = B.params_to_dict(sim.get_params())
    arr = {k: d[k] for k in ("mass", "Ig", "rb", "W", "B", "Ma", "dl", "dq", "Vc", "target")}
    arr["rg"] = np.zeros((n, 3))   # the vehicle's own CoG is the body origin
    arr["cls"] = workloads.env_classes(counts)
    envs = oracle.attach_payload(oracle.make_envs(arr), sim.get_payload())
    ref, _, _ = oracle.rollout(classes, envs, s0.astype(np.float64), a, 0.01, 4)
    err = rel_state_err(sim.get_state(), ref)
    assert err.max() <= ONE_STEP_TOL, err.max()
    sim.status()
    sim.close()


def test_payload_api_errors():
    counts = [8, 4]
    classes, sim = make(counts, vehicles.PAYLOAD)
    n = sim.n_envs
    bad = np.zeros((n, 4))
    bad[0, 0] = -1.0
    with pytest.raises(B.MGError) as e:
        sim.set_payload(bad)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    bad[0, 0] = np.nan
    with pytest.raises(B.MGError):
        sim.set_payload(bad)
    with pytest.raises(B.MGError):
        sim.set_payload(np.zeros((n - 1, 4)))
    z = torch.zeros(sim.n_slots, 6, device="cuda")
    with pytest.raises(B.MGError) as e:
        B.mg_set_hydro(sim.handle, z, None, None)
    assert "payload" in str(e.value)
    sim.close()
    plain = B.Sim(classes, counts, dt=0.01, K=1, per_env_params=True, reset=dict(vehicles.HOVER))
    with pytest.raises(B.MGError) as e:
        plain.get_payload()
    assert e.value.code == B.MG_ERR_INVALID_ARG
    plain.close()
