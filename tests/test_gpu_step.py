"""GPU parity of the batched step (CUDA path through the C-ABI) against the
FP64 oracle on the same seeded inputs.

Tolerances: per-env relative state error <= 1e-5 after one control step from
an identical FP32 state, and trajectory-relative error <= 1e-3 over 1000 steps
(error = ||x_gpu - x_ref|| / max(||x_ref||, 1), quaternion sign-aligned).
"""
import math
import time

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


def make_sim(classes, counts, K=1, dt=0.01, reset=None, per_env=True, **kw):
    return B.Sim(classes, counts, dt=dt, K=K, per_env_params=per_env, reset=reset or dict(vehicles.NO_DR), **kw)


def set_inputs(sim, classes, counts, seed, n_thr_of_env):
    p = workloads.random_params(seed, classes, counts)
    sim.set_params(B.dict_to_params(p, sim.n_envs))
    s0 = workloads.random_states(seed + 1, sim.n_envs, n_thr_of_env)
    sim.set_state(s0)
    return p, s0


def n_thr_of(classes, counts):
    return np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])


@pytest.mark.parametrize("counts,K", [([1024], 1), ([37, 1, 0, 130, 5], 4), ([3, 5, 7, 9, 11], 8),
                                      ([129, 128, 127, 4, 256], 2)])
def test_one_step_matches_oracle(counts, K):
    classes = vehicles.five_classes()[:len(counts)]
    sim = make_sim(classes, counts, K=K)
    nthr = n_thr_of(classes, counts)
    p, s0 = set_inputs(sim, classes, counts, 100 + K, nthr)
    a = workloads.actions(7, 1, sim.n_envs)
    sim.step(sim.pack_actions(a))
    torch.cuda.synchronize()
    gpu = sim.get_state()
    envs = oracle.make_envs(oracle_env_arrays(p))
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0.astype(np.float64), a, 0.01, K)
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, (err.max(), np.argmax(err))
    # Fused observation and reward of the same step.
    slots = sim.slots_of_envs()
    obs = sim.obs.cpu().numpy()[slots]
    rew = sim.reward.cpu().numpy()[slots]
    np.testing.assert_allclose(obs, o_ref[0], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(rew, r_ref[0], rtol=1e-5, atol=1e-4)
    sim.status()
    sim.close()


def test_reset_matches_oracle_draws():
    classes = vehicles.five_classes()
    counts = [64, 33, 1, 40, 70]
    sim = make_sim(classes, counts, K=4, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=0x4D47)
    torch.cuda.synchronize()
    envs, ref_state = oracle.reset(classes, workloads.env_classes(counts), vehicles.HOVER_DR, 0x4D47)
    ref = oracle.envs_to_arrays(envs)
    got = B.params_to_dict(sim.get_params())
    for k in ("mass", "Ig", "rb", "W", "B", "Ma", "dl", "dq", "Vc", "target"):
        np.testing.assert_allclose(got[k], ref[k], rtol=2e-7, atol=1e-7, err_msg=k)
    st = sim.get_state()
    np.testing.assert_allclose(st[:, :13], ref_state[:, :13], rtol=2e-7, atol=1e-7)
    sim.close()


def test_reset_subset_and_full_size_sampled():
    """The benchmark workload size (1,048,576 envs, 5 classes, hover + DR, K=4):
    a sampled set of envs after reset + one step against the oracle run on
    those envs alone (draws are keyed by env id)."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(1 << 20, 5)
    sim = make_sim(classes, counts, K=4, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=5)
    a_full = torch.zeros(1, sim.action_floats, device="cuda")
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(sim.n_envs, 2048, replace=False))
    ids = np.unique(np.concatenate([ids, [0, sim.n_envs - 1] + [sum(counts[:c]) for c in range(1, 5)]]))
    # Actions for the sampled envs; zeros elsewhere.
    a_s = workloads.actions(9, 1, len(ids))
    a_env = np.zeros((1, sim.n_envs, 8), np.float32)
    a_env[:, ids] = a_s
    a_full = sim.pack_actions(a_env)
    sim.step(a_full)
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids]
    ec = workloads.env_classes(counts)[ids]
    envs, s0 = oracle.reset(classes, ec, vehicles.HOVER_DR, 5, env_ids=ids)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0, a_s, 0.01, 4)
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, err.max()
    slots = sim.slots_of_envs()[ids]
    np.testing.assert_allclose(sim.obs.cpu().numpy()[slots], o_ref[0], rtol=2e-5, atol=2e-5)
    sim.close()


@pytest.mark.parametrize("E,launches", [(1 << 20, 5), (65536, 3)])
def test_class_constant_step_in_both_launch_shapes(E, launches):
    """Class-constant hover step, 5 classes, K=4, sampled envs after reset +
    one step against the oracle. At 1,048,576 envs (the benchmark workload)
    the step runs one launch per class with the class constants as the kernel
    parameter; at 65,536 envs one side-by-side launch per thruster count with
    the constants in shared memory."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(E, 5)
    sim = make_sim(classes, counts, K=4, reset=dict(vehicles.HOVER), per_env=False)
    assert sim.launches_per_step() == launches
    sim.reset(seed=7)
    rng = np.random.default_rng(8)
    bounds = np.cumsum(counts)
    ids = np.sort(rng.choice(E, 1024, replace=False))
    ids = np.unique(np.concatenate([ids, [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    a_s = workloads.actions(11, 1, len(ids))
    a_env = np.zeros((1, E, 8), np.float32)
    a_env[:, ids] = a_s
    sim.step(sim.pack_actions(a_env))
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids]
    envs, s0 = oracle.reset(classes, workloads.env_classes(counts)[ids], vehicles.HOVER, 7, env_ids=ids)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0, a_s, 0.01, 4)
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, (err.max(), int(ids[np.argmax(err)]))
    slots = sim.slots_of_envs()[ids]
    np.testing.assert_allclose(sim.obs.cpu().numpy()[slots], o_ref[0], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(sim.reward.cpu().numpy()[slots], r_ref[0], rtol=1e-5, atol=1e-4)
    sim.status()
    sim.close()


def test_thousand_step_trajectory_plain_workload():
    """Plain workload: 1024 envs of class 0, no DR, zero current, K=1, dt=0.01,
    1000 steps of uniform actions from rest."""
    classes = [vehicles.heavy8()]
    sim = make_sim(classes, [1024], K=1, per_env=False)
    sim.reset(seed=0x4D47)
    T, every = 1000, 50
    a = workloads.actions(0x4D47, T, 1024)
    a_dev = sim.pack_actions(a)
    envs, s_ref = oracle.reset(classes, np.zeros(1024, np.int32), vehicles.NO_DR, 0x4D47)
    gpu_traj, ref_traj = [], []
    for t0 in range(0, T, every):
        B.mg_step(sim.handle, a_dev[t0:t0 + every], every, None, None)
        torch.cuda.synchronize()
        gpu_traj.append(sim.get_state().astype(np.float64))
        s_ref, _, _ = oracle.rollout(classes, envs, s_ref, a[t0:t0 + every], 0.01, 1, obs=False)
        ref_traj.append(s_ref.copy())
    g = np.stack(gpu_traj, 1)
    r = np.stack(ref_traj, 1)
    g = align_q(g, r)
    num = np.linalg.norm(g - r, axis=-1).max(1)
    den = np.maximum(np.linalg.norm(r, axis=-1).max(1), 1.0)
    traj_err = num / den
    assert traj_err.max() <= TRAJ_TOL, traj_err.max()
    sim.status()
    sim.close()


def test_rollout_obs_reward_every_step_and_multi_step_equivalence():
    classes = vehicles.five_classes()
    counts = [20, 12, 8, 16, 4]
    sim = make_sim(classes, counts, K=4, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=3)
    s_init = sim.get_state()
    T = 25
    a = workloads.actions(11, T, sim.n_envs)
    a_dev = sim.pack_actions(a)
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    sim.rollout(a_dev, T, obs, rew)
    torch.cuda.synchronize()
    s_roll = sim.get_state()
    # Same rollout as one multi-step launch and as T single-step launches.
    sim.set_state(s_init)
    B.mg_step(sim.handle, a_dev, T, None, None)
    torch.cuda.synchronize()
    assert np.array_equal(sim.get_state(), s_roll)
    sim.set_state(s_init)
    for t in range(T):
        sim.step(a_dev[t:t + 1])
    torch.cuda.synchronize()
    assert np.array_equal(sim.get_state(), s_roll)
    np.testing.assert_array_equal(sim.obs.cpu().numpy(), obs[-1].cpu().numpy())
    # Against the oracle from its own reset draws.
    envs, s0 = oracle.reset(classes, workloads.env_classes(counts), vehicles.HOVER_DR, 3)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0, a, 0.01, 4)
    slots = sim.slots_of_envs()
    o = obs.cpu().numpy()[:, slots]
    r = rew.cpu().numpy()[:, slots]
    np.testing.assert_allclose(o, o_ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(r, r_ref, rtol=1e-4, atol=1e-3)
    # Padding slots read zero.
    pad = np.setdiff1d(np.arange(sim.n_slots), slots)
    assert np.all(obs.cpu().numpy()[:, pad] == 0) and np.all(rew.cpu().numpy()[:, pad] == 0)
    sim.close()


def test_rest_stays_rest_bit_exact_on_gpu():
    classes = vehicles.five_classes()
    counts = [8, 4, 4, 8, 4]
    sim = make_sim(classes, counts, K=4, per_env=False)
    sim.reset(seed=1)
    s0 = sim.get_state()
    s0[:, 0:3] = np.random.default_rng(0).uniform(-3, 3, (sim.n_envs, 3)).astype(np.float32)
    sim.set_state(s0)
    a = sim.new_actions(50)
    B.mg_step(sim.handle, a, 50, None, None)
    torch.cuda.synchronize()
    assert np.array_equal(sim.get_state(), s0)
    sim.close()


def test_env_result_independent_of_co_resident_classes():
    """Class-3 envs alone vs inside a 5-class mix with the same inputs:
    bit-identical states (permutation / class-mix invariance)."""
    classes = vehicles.five_classes()
    counts_mix = [30, 17, 9, 21, 13]
    sim = make_sim(classes, counts_mix, K=4)
    nthr = n_thr_of(classes, counts_mix)
    p, s0 = set_inputs(sim, classes, counts_mix, 5, nthr)
    a = workloads.actions(5, 10, sim.n_envs)
    sim.step(sim.pack_actions(a), n_steps=10)
    torch.cuda.synchronize()
    mixed = sim.get_state()
    lo, hi = sum(counts_mix[:3]), sum(counts_mix[:4])
    solo = make_sim([classes[3]], [counts_mix[3]], K=4)
    ps = {k: v[lo:hi] for k, v in p.items()}
    ps["cls"] = np.zeros(hi - lo, np.int32)
    solo.set_params(B.dict_to_params(ps, hi - lo))
    solo.set_state(s0[lo:hi])
    solo.step(solo.pack_actions(a[:, lo:hi]), n_steps=10)
    torch.cuda.synchronize()
    assert np.array_equal(solo.get_state(), mixed[lo:hi])
    sim.close()
    solo.close()


def test_env_result_independent_of_env_order():
    """Permuting the envs of a class (their parameters, states and actions)
    permutes the results bit-exactly: no env sees another."""
    classes = vehicles.five_classes()
    counts = [300, 7, 140, 0, 65]
    sims = [make_sim(classes, counts, K=4) for _ in range(2)]
    n = sims[0].n_envs
    p, s0 = set_inputs(sims[0], classes, counts, 31, n_thr_of(classes, counts))
    a = workloads.actions(32, 3, n)
    perm = np.arange(n)
    rng = np.random.default_rng(33)
    lo = 0
    for c in counts:   # shuffle within each class block
        perm[lo:lo + c] = lo + rng.permutation(c)
        lo += c
    pp = {k: np.asarray(v)[perm] for k, v in p.items()}
    sims[1].set_params(B.dict_to_params(pp, n))
    sims[1].set_state(s0[perm])
    sims[0].rollout(sims[0].pack_actions(a), 3)
    sims[1].rollout(sims[1].pack_actions(a[:, perm]), 3)
    torch.cuda.synchronize()
    assert np.array_equal(sims[1].get_state(), sims[0].get_state()[perm])
    for s in sims:
        s.status()
        s.close()


def test_nonfinite_state_is_reported_and_cleared():
    sim = make_sim([vehicles.heavy8()], [64], K=1)
    a = np.zeros((1, 64, 8), np.float32)
    a[0, 5, 2] = np.nan
    sim.step(sim.pack_actions(a))
    with pytest.raises(B.MGError) as e:
        sim.status()
    assert e.value.code == B.MG_ERR_NONFINITE
    sim.status()  # cleared
    sim.close()


def test_wait_that_runs_out_is_reported_and_the_simulator_stays_usable():
    """A step launch whose copies are never issued: every warp's bounded wait
    gives up after 20 ms, the status reports a timeout, the state is untouched
    and the next normal step matches a simulator that never saw the failure."""
    classes = vehicles.five_classes()
    counts = [300, 5, 130, 0, 64]
    sims = [make_sim(classes, counts, K=4, reset=dict(vehicles.HOVER_DR)) for _ in range(2)]
    for s in sims:
        s.reset(seed=8)
    s0 = sims[0].get_state()
    t0 = time.perf_counter()
    B.mg_test_wait_timeout(sims[0].handle, 20_000_000)
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(B.MGError) as e:
        sims[0].status()
    assert e.value.code == B.MG_ERR_TIMEOUT
    sims[0].status()   # cleared
    assert np.array_equal(sims[0].get_state(), s0)
    a = sims[0].pack_actions(workloads.actions(4, 1, sims[0].n_envs))
    for s in sims:
        s.step(a)
    torch.cuda.synchronize()
    assert np.array_equal(sims[0].get_state(), sims[1].get_state())
    assert torch.equal(sims[0].obs, sims[1].obs)
    for s in sims:
        s.status()
        s.close()


def test_state_and_params_roundtrip_byte_exact():
    classes = vehicles.five_classes()
    counts = [5, 6, 7, 8, 9]
    sim = make_sim(classes, counts, K=2, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=77)
    s = sim.get_state()
    p = sim.get_params()
    sim.step(sim.new_actions(1) + 0.3)
    sim.set_state(s)
    sim.set_params(p)
    assert np.array_equal(sim.get_state(), s)
    p2 = sim.get_params()
    assert np.array_equal(p2, p)
    sim.close()


def test_error_paths():
    sim = make_sim([vehicles.heavy8()], [16], K=1, record_steps=0)
    with pytest.raises(B.MGError) as e:
        B.mg_step(sim.handle, None, 1, None, None)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    with pytest.raises(B.MGError) as e:
        B.mg_step(sim.handle, sim.new_actions(1), 0, None, None)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    with pytest.raises(B.MGError) as e:
        B.mg_step_backward(sim.handle, sim.new_actions(1))
    assert e.value.code == B.MG_ERR_STATE
    with pytest.raises(B.MGError) as e:
        B.mg_rollout(sim.handle, sim.new_actions(2), 2, record=True)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    with pytest.raises(B.MGError) as e:
        B.mg_create([vehicles.heavy8()], [1 << 20], 0.01, 1, True, None, mem_budget=1 << 20)
    assert e.value.code == B.MG_ERR_OOM
    sim.close()


def test_host_buffer_step_equals_device_step():
    classes = vehicles.five_classes()
    counts = [10, 10, 10, 10, 10]
    sim = make_sim(classes, counts, K=4, reset=dict(vehicles.HOVER_DR))
    sim.reset(seed=2)
    s0 = sim.get_state()
    a = workloads.actions(2, 1, sim.n_envs)
    a_dev = sim.pack_actions(a)
    sim.step(a_dev)
    torch.cuda.synchronize()
    s_dev, o_dev = sim.get_state(), sim.obs.cpu().numpy().copy()
    sim.set_state(s0)
    a_host = a_dev.cpu().pin_memory()
    o_host = torch.zeros(sim.n_slots, 13).pin_memory()
    r_host = torch.zeros(sim.n_slots).pin_memory()
    B.mg_step_host(sim.handle, a_host, 1, o_host, r_host)
    assert np.array_equal(sim.get_state(), s_dev)
    assert np.array_equal(o_host.numpy(), o_dev)
    sim.close()


@pytest.mark.parametrize("per_env", [True, False])
def test_host_buffer_step_chunked_multi_step_equals_device_step(per_env):
    """Sizes that cut the launches into several copy/step chunks, 3 steps per
    call; at this size the step runs one launch per class (class tables as the
    kernel parameter)."""
    classes = vehicles.five_classes()
    counts = [300001, 3, 240001, 5, 9]   # class 0 spans two 2048-tile chunks
    sim = make_sim(classes, counts, K=1, reset=dict(vehicles.HOVER_DR if per_env else vehicles.HOVER),
                   per_env=per_env)
    assert sim.launches_per_step() == 5
    sim.reset(seed=3)
    s0 = sim.get_state()
    a_dev = (torch.rand(3, sim.action_floats, device="cuda") * 2 - 1).contiguous()
    B.mg_step(sim.handle, a_dev, 3, sim.obs, sim.reward)
    torch.cuda.synchronize()
    s_dev, o_dev, r_dev = sim.get_state(), sim.obs.cpu().numpy().copy(), sim.reward.cpu().numpy().copy()
    sim.set_state(s0)
    a_host = a_dev.cpu().pin_memory()
    o_host = torch.full((sim.n_slots, 13), 7.0).pin_memory()
    r_host = torch.full((sim.n_slots,), 7.0).pin_memory()
    B.mg_step_host(sim.handle, a_host, 3, o_host, r_host)
    assert np.array_equal(sim.get_state(), s_dev)
    assert np.array_equal(o_host.numpy(), o_dev)
    assert np.array_equal(r_host.numpy(), r_dev)
    sim.status()
    sim.close()


def test_graph_replay_and_autotune_keep_results():
    classes = vehicles.five_classes()
    counts = [100, 50, 60, 70, 80]
    sim = make_sim(classes, counts, K=4, reset=dict(vehicles.DR_TRAIN))
    sim.reset(seed=9)
    s0 = sim.get_state()
    T = 8
    a_dev = sim.pack_actions(workloads.actions(4, T, sim.n_envs))
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    sim.rollout(a_dev, T, obs, rew)
    torch.cuda.synchronize()
    s_ref, o_ref = sim.get_state(), obs.clone()
    shape = B.mg_autotune(sim.handle, T)
    assert shape["lanes_per_env"] in (1, 2) and shape["envs_per_block"] == 128 // shape["lanes_per_env"]
    assert shape["blocks_per_sm"] >= 0 and shape["us_per_step"] > 0
    assert shape == dict(B.mg_get_launch_shape(sim.handle), us_per_step=shape["us_per_step"])
    assert np.array_equal(sim.get_state(), s_ref)   # autotune restores the state
    B.mg_set_launch_shape(sim.handle, 1, shape["blocks_per_sm"])   # the one-lane kernels of s_ref
    sim.set_state(s0)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = B.mg_graph_capture(sim.handle, a_dev, T, obs, rew, stream=st)
        obs.zero_()
        B.mg_graph_launch(g, stream=st)
    st.synchronize()
    assert np.array_equal(sim.get_state(), s_ref)
    assert torch.equal(obs, o_ref)
    B.mg_graph_destroy(g)
    sim.close()


@pytest.mark.parametrize("per_env", [True, False])
@pytest.mark.parametrize("counts", [[70001, 3, 60001, 5, 9],      # groups side by side
                                    [300001, 3, 240001, 5, 9]])   # one launch per class
def test_fixed_grid_keeps_results(per_env, counts):
    """A fixed persistent grid (1 block per SM, above the occupancy limit, the
    default) leaves every result bit-identical: each env is computed by one
    thread whatever block walks its tile; negative counts are refused."""
    classes = vehicles.five_classes()
    sim = make_sim(classes, counts, K=2, reset=dict(vehicles.HOVER_DR if per_env else vehicles.HOVER),
                   per_env=per_env)
    sim.reset(seed=4)
    s0 = sim.get_state()
    a_dev = sim.pack_actions(workloads.actions(6, 2, sim.n_envs))
    out = []
    for b in (0, 1, 64):
        B.mg_set_blocks_per_sm(sim.handle, b)
        sim.set_state(s0)
        sim.step(a_dev, n_steps=2)
        torch.cuda.synchronize()
        out.append((sim.get_state(), sim.obs.cpu().numpy().copy(), sim.reward.cpu().numpy().copy()))
    for st, ob, rw in out[1:]:
        assert np.array_equal(st, out[0][0]) and np.array_equal(ob, out[0][1]) and np.array_equal(rw, out[0][2])
    with pytest.raises(B.MGError) as e:
        B.mg_set_blocks_per_sm(sim.handle, -1)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    sim.status()
    sim.close()


@pytest.mark.parametrize("per_env", [True, False])
def test_graph_of_per_class_launches_equals_direct_rollout(per_env):
    """A size that takes the one-launch-per-class plan (class tables as the
    kernel parameter, every launch a programmatic dependent): a captured
    4-step rollout replays to the same states, observations and rewards as
    the direct rollout, bit for bit."""
    classes = vehicles.five_classes()
    counts = [300001, 3, 240001, 5, 9]
    sim = make_sim(classes, counts, K=2, reset=dict(vehicles.HOVER_DR if per_env else vehicles.HOVER),
                   per_env=per_env)
    assert sim.launches_per_step() == 5
    sim.reset(seed=12)
    s0 = sim.get_state()
    T = 4
    a_dev = sim.pack_actions(workloads.actions(13, T, sim.n_envs))
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    sim.rollout(a_dev, T, obs, rew)
    torch.cuda.synchronize()
    s_ref, o_ref, r_ref = sim.get_state(), obs.clone(), rew.clone()
    sim.set_state(s0)
    obs.zero_()
    rew.zero_()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = B.mg_graph_capture(sim.handle, a_dev, T, obs, rew, stream=st)
        B.mg_graph_launch(g, stream=st)
    st.synchronize()
    assert np.array_equal(sim.get_state(), s_ref)
    assert torch.equal(obs, o_ref) and torch.equal(rew, r_ref)
    B.mg_graph_destroy(g)
    sim.status()
    sim.close()


def test_flop_count_matches_hand_count():
    """The counted substep of the 8-thruster class: rotor 3/thr, thrust 2/thr,
    allocation 6 x (8 mul + 7 add) = 90; the remaining terms are fixed."""
    s8, o8 = B.mg_count_flops(8)
    s4, _ = B.mg_count_flops(4)
    assert s8 - s4 == 4 * (3 + 2) + 6 * 4 * 2


def test_interleaved_class_map_through_env_order():
    """A caller whose envs carry an arbitrary class map (interleaved here)
    builds the simulator from mg_env_order's class counts and moves each env's
    data to library env lib_env[i]; every env's result, read back through the
    same map, equals the oracle run on that env in the caller's order. Then
    mg_observe of the final state gives the rollout's last observation and
    its reward without the command term."""
    classes = vehicles.five_classes()
    rng = np.random.default_rng(50)
    env_class = rng.integers(0, 5, 700).astype(np.int32)
    env_class[:10] = [3, 0, 4, 0, 1, 2, 2, 4, 3, 1]
    counts, lib_env = B.mg_env_order(env_class, 5)
    sim = make_sim(classes, counts.tolist(), K=4)
    n, T = sim.n_envs, 3
    # The caller's data, in the caller's order (env i of class env_class[i]).
    grouped = workloads.random_params(51, classes, counts.tolist())
    p_user = {k: np.asarray(v)[lib_env] for k, v in grouped.items()}
    assert np.array_equal(p_user["cls"], env_class)
    nthr_user = np.array([classes[c]["n_thr"] for c in env_class])
    s_user = workloads.random_states(52, n, nthr_user)
    a_user = workloads.actions(53, T, n)
    # Into the library's order: library env lib_env[i] holds the caller's env i.
    order = np.argsort(lib_env)
    sim.set_params(B.dict_to_params({k: v[order] for k, v in p_user.items()}, n))
    sim.set_state(s_user[order])
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    sim.rollout(sim.pack_actions(a_user[:, order]), T, obs, rew)
    o_now = torch.zeros(sim.n_slots, 13, device="cuda")
    r_now = torch.zeros(sim.n_slots, device="cuda")
    B.mg_observe(sim.handle, o_now, r_now)
    torch.cuda.synchronize()
    got = sim.get_state()[lib_env]          # back in the caller's order
    slots = sim.slots_of_envs()[lib_env]
    envs = oracle.make_envs(oracle_env_arrays(p_user))
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s_user.astype(np.float64), a_user, 0.01, 4)
    err = rel_state_err(got, ref)
    assert err.max() <= 3 * ONE_STEP_TOL, err.max()
    np.testing.assert_allclose(obs.cpu().numpy()[:, slots], o_ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(rew.cpu().numpy()[:, slots], r_ref, rtol=1e-4, atol=1e-3)
    np.testing.assert_allclose(o_now.cpu().numpy(), obs[-1].cpu().numpy(), rtol=1e-6, atol=1e-6)
    c = np.clip(a_user[-1].astype(np.float64), -1, 1) * (np.arange(8)[None, :] < nthr_user[:, None])
    np.testing.assert_allclose(r_now.cpu().numpy()[slots], rew[-1].cpu().numpy()[slots] + 0.01 * (c * c).sum(1),
                               rtol=1e-6, atol=1e-5)
    sim.status()
    sim.close()
