"""GPU parity of the propeller dead zone and of the zero-order rotor (paper
Sec. III-D: quadratic thrust with a dead zone; first-order rotor lag whose
zero time constant is the zero-order model) against the FP64 oracle.

The thrust of a propeller is 0 while its rotor state after the lag is inside
the dead zone (|n| < delta), k n|n| otherwise. The step kernel decides this
in FP32 and the oracle in FP64, so the rotor paths used here keep every
substep's |n| at least 1e-5 away from delta (the FP32 and FP64 rotor states
differ by ~1e-8), except in the zero-order tests, where n equals the FP32
command exactly on both sides and the commands sit on the threshold and on
its neighbouring floats. Each dead zone is an FP32 number, so that both sides
compare against the same threshold.

Three launch paths take the dead zone from three table sources: one launch
per class with the class tables as the kernel parameter (>= 300k envs), one
side-by-side launch per thruster count with the tables staged in shared
memory (<= 65k envs), and per-env parameter runs. Classes without a dead zone
share the batch, so the per-class choice of the test-free thrust path is
exercised next to the tested one. Tolerance: one-step relative state error
<= 1e-5, as for every one-step parity test.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import oracle_env_arrays, rel_state_err

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = 1e-5
MARGIN = 1e-5
K = 4
DT = 0.01


def dz_classes(zero_order=False):
    """The five workload classes with dead zones on classes 0, 2 and 4 (2: a
    different one per thruster, one of them 0) and none on 1 and 3."""
    cl = vehicles.five_classes()
    cl[0] = dict(cl[0], deadzone=[0.3125] * 8)
    cl[2] = dict(cl[2], deadzone=[0.125, 0.25, 0.125, 0.25, 0.1875, 0.0])
    cl[4] = dict(cl[4], deadzone=[0.25] * 6)
    if zero_order:
        cl = [dict(c, T_rotor=[0.0] * c["n_thr"]) for c in cl]
    return cl


def alphas(c):
    h = DT / K
    return np.array([1.0 - math.exp(-h / T) if T > 0 else 1.0 for T in c["T_rotor"]])


def rotor_substeps(n0, cmd, alpha):
    """FP64 rotor states after each of the K substeps of one step (the rotor
    lag is decoupled from the rest of the dynamics)."""
    out, n = [], n0
    for _ in range(K):
        n = n + alpha * (cmd - n)
        out.append(n)
    return np.array(out)


def straddling_rotors(rng, classes, ec, n_envs):
    """Initial rotor states and commands whose rotor paths cross the dead
    zone's edges, redrawn until every substep keeps |n| at least MARGIN away
    from delta."""
    n0 = np.zeros((n_envs, 8), np.float32)
    cmd = np.zeros((n_envs, 8), np.float32)
    for e in range(n_envs):
        c = classes[ec[e]]
        al = alphas(c)
        for j in range(c["n_thr"]):
            dz = c["deadzone"][j]
            for _ in range(1000):
                if dz > 0 and rng.random() < 0.7:
                    # Near the edge: start just inside or outside, command across.
                    s = rng.choice([-1.0, 1.0])
                    a = np.float32(s * (dz + rng.uniform(-0.05, 0.05)))
                    b = np.float32(s * (dz + rng.uniform(-0.15, 0.15)))
                else:
                    a, b = np.float32(rng.uniform(-1, 1)), np.float32(rng.uniform(-1, 1))
                path = rotor_substeps(float(a), float(b), al[j])
                if dz == 0 or np.all(np.abs(np.abs(path) - dz) > MARGIN):
                    n0[e, j], cmd[e, j] = a, b
                    break
            else:
                raise RuntimeError("no admissible rotor path")
    return n0, cmd


def one_step_case(classes, counts, per_env, ids, seed, specialised=1):
    """Step the sampled envs once from straddling rotor states; return the GPU
    and oracle states, observations and rewards, and the rotor decisions.
    specialised=0: the library's kernels instead of the class-specialised ones."""
    reset = dict(vehicles.HOVER_DR if per_env else vehicles.HOVER)
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=per_env, reset=reset)
    if not specialised:
        B.mg_set_launch_shape(sim.handle, 1, 0, 0)
    sim.reset(seed=seed)
    ec_all = workloads.env_classes(counts)
    ec = ec_all[ids]
    rng = np.random.default_rng(seed + 1)
    n0, cmd = straddling_rotors(rng, classes, ec, len(ids))
    s_all = sim.get_state()
    s_all[ids, 13:21] = n0
    sim.set_state(s_all)
    a_env = np.zeros((1, sim.n_envs, 8), np.float32)
    a_env[0, ids] = cmd
    sim.step(sim.pack_actions(a_env))
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids]
    slots = sim.slots_of_envs()[ids]
    obs, rew = sim.obs.cpu().numpy()[slots], sim.reward.cpu().numpy()[slots]
    launches = sim.launches_per_step()
    sim.status()
    sim.close()
    envs, _ = oracle.reset(classes, ec, reset, seed, env_ids=ids)
    s0 = s_all[ids].astype(np.float64)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0.copy(), cmd[None], DT, K)   # updates in place
    return dict(gpu=gpu, ref=ref, obs=obs, o_ref=o_ref[0], rew=rew, r_ref=r_ref[0], n0=n0, cmd=cmd, ec=ec,
                envs=envs, s0=s0, launches=launches)


def sample_ids(counts, n, seed):
    E = sum(counts)
    rng = np.random.default_rng(seed)
    b = np.cumsum(counts)
    ids = rng.choice(E, min(n, E), replace=False)
    return np.unique(np.concatenate([ids, [0, E - 1], b[:-1], b[:-1] - 1]).clip(0, E - 1))


@pytest.mark.parametrize("per_env,counts,launches,spec", [
    (False, [300001, 3, 240001, 5, 9], 5, 1),   # one launch per class, class-specialised kernels (tables as literals)
    (False, [300001, 3, 240001, 5, 9], 5, 0),   # one launch per class, library kernels (tables as the kernel parameter)
    (False, [20001, 3, 15001, 5, 9], 3, 1),     # groups side by side, tables in shared memory
    (True, [300001, 3, 240001, 5, 9], 5, 1),    # per-env parameters, one launch per class
    (True, [301, 7, 141, 9, 65], 3, 1),         # per-env parameters, side by side
])
def test_dead_zone_one_step_matches_oracle(per_env, counts, launches, spec):
    classes = dz_classes()
    ids = sample_ids(counts, 768, 17)
    r = one_step_case(classes, counts, per_env, ids, seed=21 + int(per_env), specialised=spec)
    assert r["launches"] == launches
    err = rel_state_err(r["gpu"], r["ref"])
    assert err.max() <= ONE_STEP_TOL, (err.max(), int(ids[np.argmax(err)]))
    np.testing.assert_allclose(r["obs"], r["o_ref"], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(r["rew"], r["r_ref"], rtol=1e-5, atol=1e-4)
    # The cases cross the edge: per dead-zone thruster, rotor states ending
    # inside and outside, and envs whose step saw a thruster switch.
    dz = np.array([np.pad(classes[c]["deadzone"], (0, 8 - classes[c]["n_thr"])) for c in r["ec"]])
    nth = np.array([classes[c]["n_thr"] for c in r["ec"]])
    has = (dz > 0) & (np.arange(8)[None, :] < nth[:, None])
    inside = np.abs(r["gpu"][:, 13:21]) < dz
    assert np.sum(inside & has) > 50 and np.sum(~inside & has) > 50
    start_in = np.abs(r["n0"]) < dz
    assert np.sum((start_in != inside) & has) > 20
    # The dead zone matters for these envs: without it the oracle lands elsewhere.
    free = [dict(c, deadzone=[0.0] * c["n_thr"]) for c in classes]
    ref_free, _, _ = oracle.rollout(free, r["envs"], r["s0"].copy(), r["cmd"][None], DT, K)
    moved = np.abs(ref_free[:, 7:13] - r["ref"][:, 7:13]).max(1) > 1e-4
    assert np.sum(moved) > 20


@pytest.mark.parametrize("per_env,counts", [(False, [20001, 3, 15001, 5, 9]), (False, [300001, 3, 240001, 5, 9]),
                                            (True, [33, 7, 41, 9, 65])])
def test_zero_order_rotor_on_the_threshold_matches_oracle(per_env, counts):
    """T_rotor = 0 (alpha = 1): from rest the rotor state after every substep
    is the FP32 command itself, so commands exactly on the dead zone's edge
    and on its neighbouring floats are decided the same way on both sides:
    no thrust below delta, k delta^2 at delta."""
    classes = dz_classes(zero_order=True)
    reset = dict(vehicles.HOVER_DR if per_env else vehicles.HOVER)
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=per_env, reset=reset)
    sim.reset(seed=31)
    ids = sample_ids(counts, 512, 32)
    ec = workloads.env_classes(counts)[ids]
    rng = np.random.default_rng(33)
    cmd = np.zeros((len(ids), 8), np.float32)
    for e, c in enumerate(ec):
        for j in range(classes[c]["n_thr"]):
            dz = np.float32(classes[c]["deadzone"][j])
            s = np.float32(rng.choice([-1.0, 1.0]))
            pick = rng.integers(0, 5)
            if dz > 0 and pick == 0:
                cmd[e, j] = s * dz
            elif dz > 0 and pick == 1:
                cmd[e, j] = s * np.nextafter(dz, np.float32(0))
            elif dz > 0 and pick == 2:
                cmd[e, j] = s * np.nextafter(dz, np.float32(1))
            else:
                cmd[e, j] = np.float32(rng.uniform(-1.2, 1.2))   # clamped to [-1, 1]
    s_all = sim.get_state()
    s_all[ids, 13:21] = 0.0
    sim.set_state(s_all)
    a_env = np.zeros((1, sim.n_envs, 8), np.float32)
    a_env[0, ids] = cmd
    sim.step(sim.pack_actions(a_env))
    torch.cuda.synchronize()
    gpu = sim.get_state()[ids]
    sim.status()
    sim.close()
    nth = np.array([classes[c]["n_thr"] for c in ec])
    mask = np.arange(8)[None, :] < nth[:, None]
    assert np.array_equal(gpu[:, 13:21], np.where(mask, np.clip(cmd, -1, 1), 0))   # n = c exactly
    envs, _ = oracle.reset(classes, ec, reset, 31, env_ids=ids)
    ref, _, _ = oracle.rollout(classes, envs, s_all[ids].astype(np.float64), cmd[None], DT, K)
    err = rel_state_err(gpu, ref)
    assert err.max() <= ONE_STEP_TOL, (err.max(), int(ids[np.argmax(err)]))
    dz = np.array([np.pad(classes[c]["deadzone"], (0, 8 - classes[c]["n_thr"])) for c in ec]).astype(np.float32)
    assert np.sum(mask & (dz > 0) & (np.abs(cmd) == dz)) > 20


def test_dead_zone_adjoint_matches_oracle_tangents():
    """Gradients through the dead zone (zero thrust derivative inside it)
    against the oracle's forward-mode tangents, with rotor paths crossing the
    edges over a 16-step recorded rollout."""
    from tests.test_gpu_adjoint import gpu_gradients
    classes = dz_classes()
    counts = [6, 3, 6, 3, 6]
    T, ckpt = 16, 5
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                record_steps=T, ckpt_every=ckpt)
    p = workloads.random_params(41, classes, counts)
    sim.set_params(B.dict_to_params(p, sim.n_envs))
    ec = workloads.env_classes(counts)
    nthr = np.array([classes[c]["n_thr"] for c in ec])
    s0 = workloads.random_states(42, sim.n_envs, nthr, pos_scale=2.0, vel_scale=0.3, rate_scale=0.4)
    rng = np.random.default_rng(43)
    a = np.zeros((T, sim.n_envs, 8), np.float32)
    # Rotor paths over the whole horizon stay MARGIN away from every edge.
    for e in range(sim.n_envs):
        c = classes[ec[e]]
        al = alphas(c)
        for j in range(c["n_thr"]):
            dz = c["deadzone"][j]
            n = float(s0[e, 13 + j])
            for t in range(T):
                for _ in range(1000):
                    if dz > 0 and rng.random() < 0.6:
                        v = np.float32(rng.choice([-1, 1]) * (dz + rng.uniform(-0.1, 0.1)))
                    else:
                        v = np.float32(rng.uniform(-0.99, 0.99))
                    path = rotor_substeps(n, float(v), al[j])
                    if dz == 0 or np.all(np.abs(np.abs(path) - dz) > MARGIN):
                        a[t, e, j] = v
                        n = path[-1]
                        break
                else:
                    raise RuntimeError("no admissible command")
    sim.set_state(s0)
    E = sim.n_envs
    g_obs = rng.normal(size=(T, E, 13)) * 0.1
    g_rew = -np.ones((T, E))
    g = gpu_gradients(sim, a, T, g_obs, g_rew, np.zeros((E, 21)))
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
            j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, DT, K, **d)
            want.append(np.einsum("te,te->e", g_rew, j["d_reward"]) + np.einsum("tek,tek->e", g_obs, j["d_obs"]))
            key = {"act": "d_actions", "A": "d_Ma", "dq": "d_dq"}[name]
            got.append(np.einsum("tek,tek->e", g[name], d[key]) if name == "act"
                       else np.einsum("ek,ek->e", g[name], d[key]))
        gv, rv = np.stack(got, 1), np.stack(want, 1)
        err = np.linalg.norm(gv - rv, axis=1) / np.maximum(np.linalg.norm(rv, axis=1), 1e-6)
        assert err.max() <= 1e-3, (name, err.max())
    sim.close()
