"""GPU adjoint (mg_step_backward) against the oracle's forward-mode tangents
and against central finite differences, for gradients with respect to the
actions, the per-env added-mass and damping coefficients and the initial
state (discretise-then-differentiate).

Tolerances: FP32 adjoint vs oracle tangents <= 1e-3 relative (per env, over a
set of random directions); GPU FP64 central differences vs oracle central
differences <= 1e-8 relative plus the differences' own roundoff
(64 eps_mach sum_t |r_t| / 2h); GPU FP64 differences vs oracle tangents
<= 1e-6 relative plus the same roundoff (h = 1e-6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import autograd as AG
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import oracle_env_arrays

pytestmark = pytest.mark.gpu


def setup(counts, T, K, ckpt, seed=1):
    classes = vehicles.five_classes()[:len(counts)]
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                record_steps=T, ckpt_every=ckpt)
    p = workloads.random_params(seed, classes, counts)
    sim.set_params(B.dict_to_params(p, sim.n_envs))
    nthr = np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])
    s0 = workloads.random_states(seed + 1, sim.n_envs, nthr, pos_scale=2.0, vel_scale=0.3, rate_scale=0.4)
    sim.set_state(s0)
    a = workloads.actions(seed + 2, T, sim.n_envs, lo=-0.99, hi=0.99)
    return classes, sim, p, s0, a, nthr


def gpu_gradients(sim, a, T, g_obs, g_rew, g_sT):
    slots = sim.slots_of_envs()
    a_dev = sim.pack_actions(a)
    obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
    rew = torch.zeros(T, sim.n_slots, device="cuda")
    B.mg_rollout(sim.handle, a_dev, T, obs, rew, True)
    go = torch.zeros(T, sim.n_slots, 13)
    gr = torch.zeros(T, sim.n_slots)
    gs = torch.zeros(sim.n_slots, 21)
    go[:, slots] = torch.from_numpy(g_obs).float()
    gr[:, slots] = torch.from_numpy(g_rew).float()
    gs[slots] = torch.from_numpy(g_sT).float()
    g_act = torch.zeros(T, sim.action_floats, device="cuda")
    gA = torch.zeros(sim.n_slots, 6, device="cuda")
    gD = torch.zeros(sim.n_slots, 12, device="cuda")
    g0 = torch.zeros(sim.n_slots, 21, device="cuda")
    B.mg_step_backward(sim.handle, a_dev, go.cuda(), gr.cuda(), gs.cuda(), g_act, gA, gD, g0)
    torch.cuda.synchronize()
    sim.status()
    return dict(act=sim.unpack_actions(g_act).astype(np.float64), A=gA.cpu().numpy()[slots].astype(np.float64),
                dl=gD.cpu().numpy()[slots, :6].astype(np.float64), dq=gD.cpu().numpy()[slots, 6:].astype(np.float64),
                s0=g0.cpu().numpy()[slots].astype(np.float64), obs=obs.cpu().numpy()[:, slots],
                rew=rew.cpu().numpy()[:, slots])


@pytest.mark.parametrize("counts,T,K,ckpt", [([3, 2, 2, 3, 2], 27, 4, 10), ([4, 4, 4, 4, 4], 200, 4, 20),
                                             ([5, 0, 3, 1, 2], 9, 1, 4), ([2, 3, 2, 2, 3], 100, 2, 45)])
def test_adjoint_matches_oracle_tangents(counts, T, K, ckpt):
    """Cotangents on every observation and reward and on the final state. In
    the last case checkpoints fall every 45 steps: each segment is reversed in
    units of 15 steps recomputed from its checkpoint, the last segment 10 steps
    long."""
    classes, sim, p, s0, a, nthr = setup(counts, T, K, ckpt)
    E = sim.n_envs
    rng = np.random.default_rng(3)
    g_obs = rng.normal(size=(T, E, 13)) * 0.1
    g_rew = -np.ones((T, E)) + 0.2 * rng.normal(size=(T, E))
    g_sT = rng.normal(size=(E, 21)) * 0.1
    g_sT[np.arange(21)[None, :] >= (13 + nthr)[:, None]] = 0.0
    g = gpu_gradients(sim, a, T, g_obs, g_rew, g_sT)
    envs = oracle.make_envs(oracle_env_arrays(p))
    thr_mask = (np.arange(8)[None, :] < nthr[:, None]).astype(np.float64)
    st_mask = (np.arange(21)[None, :] < (13 + nthr)[:, None]).astype(np.float64)
    groups = {"act": lambda: dict(d_actions=rng.normal(size=(T, E, 8)) * thr_mask[None]),
              "A": lambda: dict(d_Ma=rng.normal(size=(E, 6))),
              "dl": lambda: dict(d_dl=rng.normal(size=(E, 6))),
              "dq": lambda: dict(d_dq=rng.normal(size=(E, 6))),
              "s0": lambda: dict(d_state0=rng.normal(size=(E, 21)) * st_mask * 0.1)}
    for name, mk in groups.items():
        gpu_dirs, ref_dirs = [], []
        for _ in range(3):
            d = mk()
            j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, 0.01, K, **d)
            ref = (np.einsum("te,te->e", g_rew, j["d_reward"]) + np.einsum("tek,tek->e", g_obs, j["d_obs"])
                   + np.einsum("ek,ek->e", g_sT, j["d_state"]))
            if name == "act":
                got = np.einsum("tek,tek->e", g["act"], d["d_actions"])
            elif name == "s0":
                got = np.einsum("ek,ek->e", g["s0"], d["d_state0"])
            else:
                key = {"A": "d_Ma", "dl": "d_dl", "dq": "d_dq"}[name]
                got = np.einsum("ek,ek->e", g[name], d[key])
            gpu_dirs.append(got)
            ref_dirs.append(ref)
        gv, rv = np.stack(gpu_dirs, 1), np.stack(ref_dirs, 1)
        err = np.linalg.norm(gv - rv, axis=1) / np.maximum(np.linalg.norm(rv, axis=1), 1e-6)
        assert err.max() <= 1e-3, (name, err.max(), np.argmax(err))
    sim.close()


def test_fp64_gpu_differences_match_oracle():
    counts, T, K = [2, 2, 2, 2, 2], 40, 4
    classes, sim, p, s0, a, nthr = setup(counts, T, K, 20, seed=7)
    E, n_slots = sim.n_envs, sim.n_slots
    slots = sim.slots_of_envs()
    rng = np.random.default_rng(5)
    dA, ddl, ddq = (rng.normal(size=(E, 6)) for _ in range(3))
    a_dev = sim.pack_actions(a)

    def to_slots(x):
        out = np.zeros((n_slots, 6))
        out[slots] = x
        return torch.from_numpy(out).cuda()

    dA_d, ddl_d, ddq_d = to_slots(dA), to_slots(ddl), to_slots(ddq)
    eps = 1e-6
    r_p = torch.zeros(T, n_slots, dtype=torch.float64, device="cuda")
    r_m = torch.zeros_like(r_p)
    B.mg_rollout_fp64(sim.handle, a_dev, T, dA_d, ddl_d, ddq_d, eps, r_p)
    B.mg_rollout_fp64(sim.handle, a_dev, T, dA_d, ddl_d, ddq_d, -eps, r_m)
    r0 = torch.zeros_like(r_p)
    s_end = torch.zeros(n_slots, 21, dtype=torch.float64, device="cuda")
    B.mg_rollout_fp64(sim.handle, a_dev, T, None, None, None, 0.0, r0, s_end)
    torch.cuda.synchronize()
    fd_gpu = ((r_p - r_m).cpu().numpy()[:, slots] / (2 * eps)).sum(0)
    arr = oracle_env_arrays(p)
    envs = oracle.make_envs(arr)

    def oracle_L(sign):
        arr2 = dict(arr)
        arr2["Ma"] = arr["Ma"] + sign * eps * dA
        arr2["dl"] = arr["dl"] + sign * eps * ddl
        arr2["dq"] = arr["dq"] + sign * eps * ddq
        _, _, r = oracle.rollout(classes, oracle.make_envs(arr2), s0.astype(np.float64), a, 0.01, K)
        return r.sum(0)

    fd_ref = (oracle_L(1) - oracle_L(-1)) / (2 * eps)
    # FP64 GPU trajectory itself equals the oracle's to near machine precision.
    ref_s, _, ref_r = oracle.rollout(classes, envs, s0.astype(np.float64), a, 0.01, K)
    np.testing.assert_allclose(r0.cpu().numpy()[:, slots], ref_r, rtol=1e-11, atol=1e-11)
    # A central difference carries roundoff ~ eps_mach * sum_t |r_t| / h on each
    # side; the bound below is 64 times that plus 1e-8 relative.
    roundoff = 64 * np.finfo(np.float64).eps * np.abs(ref_r).sum(0) / (2 * eps)
    assert np.all(np.abs(fd_gpu - fd_ref) <= 1e-8 * np.abs(fd_ref) + roundoff)
    j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, 0.01, K, d_Ma=dA, d_dl=ddl, d_dq=ddq)
    jv = j["d_reward"].sum(0)
    assert np.all(np.abs(fd_gpu - jv) <= 1e-6 * np.abs(jv) + roundoff)
    # The FP32 adjoint against the FP64 differences on the GPU.
    g = gpu_gradients(sim, a, T, np.zeros((T, E, 13)), np.ones((T, E)), np.zeros((E, 21)))
    adj = np.einsum("ek,ek->e", g["A"], dA) + np.einsum("ek,ek->e", g["dl"], ddl) + np.einsum("ek,ek->e", g["dq"], ddq)
    assert (np.abs(adj - fd_gpu) / np.maximum(np.abs(fd_gpu), 1e-3)).max() <= 1e-3
    sim.close()


def test_checkpoint_interval_does_not_change_gradients():
    counts, T, K = [3, 3, 3, 3, 3], 30, 2
    res = []
    for ckpt in (1, 7, 30):
        classes, sim, p, s0, a, nthr = setup(counts, T, K, ckpt, seed=11)
        E = sim.n_envs
        g = gpu_gradients(sim, a, T, np.zeros((T, E, 13)), -np.ones((T, E)), np.zeros((E, 21)))
        res.append(g)
        sim.close()
    for k in ("act", "A", "dl", "dq", "s0"):
        for r in res[1:]:
            np.testing.assert_allclose(r[k], res[0][k], rtol=1e-5, atol=1e-6, err_msg=k)


def test_autograd_function_matches_direct_call():
    counts, T, K = [4, 4, 4, 4, 4], 12, 4
    classes, sim, p, s0, a, nthr = setup(counts, T, K, 5, seed=13)
    E, n_slots = sim.n_envs, sim.n_slots
    slots = sim.slots_of_envs()
    A = torch.zeros(n_slots, 6)
    dl = torch.zeros(n_slots, 6)
    dq = torch.zeros(n_slots, 6)
    A[slots] = torch.from_numpy(p["Ma"]).float()
    dl[slots] = torch.from_numpy(p["dl"]).float()
    dq[slots] = torch.from_numpy(p["dq"]).float()
    # Padding slots carry positive placeholders so that M stays invertible.
    pad = np.setdiff1d(np.arange(n_slots), slots)
    A[pad] = 1.0
    A, dl, dq = (x.cuda().requires_grad_(True) for x in (A, dl, dq))
    acts = sim.pack_actions(a).requires_grad_(True)
    obs, rew = AG.rollout(sim, acts, A, dl, dq)
    loss = -rew.sum()
    loss.backward()
    torch.cuda.synchronize()
    sim.set_state(s0)
    g = gpu_gradients(sim, a, T, np.zeros((T, E, 13)), -np.ones((T, E)), np.zeros((E, 21)))
    np.testing.assert_allclose(sim.unpack_actions(acts.grad), g["act"], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(A.grad.cpu().numpy()[slots], g["A"], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(dl.grad.cpu().numpy()[slots], g["dl"], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(dq.grad.cpu().numpy()[slots], g["dq"], rtol=1e-6, atol=1e-7)
    sim.close()


def test_backward_refuses_a_discarded_recording():
    """Every call that changes what produced a recording (parameters, state,
    task, a step, a reset, a graph replay) discards it: backward then returns
    MG_ERR_STATE instead of differentiating old checkpoints with new values."""
    counts, T, K = [2, 2, 2, 2, 2], 6, 2
    classes, sim, p, s0, a, nthr = setup(counts, T, K, 3, seed=17)
    a_dev = sim.pack_actions(a)
    n_slots = sim.n_slots
    A = torch.ones(n_slots, 6, device="cuda")
    params = sim.get_params()
    task = sim.get_task()

    def record():
        sim.set_state(s0)
        B.mg_rollout(sim.handle, a_dev, T, None, None, True)
        steps, rid = B.mg_recording(sim.handle)
        assert steps == T and rid != 0
        return rid

    changes = {
        "set_hydro": lambda: B.mg_set_hydro(sim.handle, A, None, None),
        "set_params": lambda: sim.set_params(params),
        "set_task": lambda: sim.set_task(task),
        "set_state": lambda: sim.set_state(s0),
        "step": lambda: sim.step(a_dev[:1]),
        "rollout": lambda: B.mg_rollout(sim.handle, a_dev, 2, None, None, False),
        "reset": lambda: sim.reset(seed=3),
    }
    ids = set()
    for name, change in changes.items():
        rid = record()
        assert rid not in ids
        ids.add(rid)
        B.mg_step_backward(sim.handle, a_dev)          # valid right after recording
        change()
        assert B.mg_recording(sim.handle) == (0, 0), name
        for fn in (B.mg_step_backward, B.mg_step_backward_noalloc):
            with pytest.raises(B.MGError) as e:
                fn(sim.handle, a_dev)
            assert e.value.code == B.MG_ERR_STATE, name
    # A replayed graph advances the same envs: it discards the recording too.
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = B.mg_graph_capture(sim.handle, a_dev, 2, None, None, stream=st)
    st.synchronize()
    record()
    with torch.cuda.stream(st):
        B.mg_graph_launch(g, stream=st)
    st.synchronize()
    with pytest.raises(B.MGError) as e:
        B.mg_step_backward(sim.handle, a_dev)
    assert e.value.code == B.MG_ERR_STATE
    B.mg_graph_destroy(g)
    torch.cuda.synchronize()
    sim.close()


def test_autograd_backward_after_another_forward_raises():
    """The simulator holds one recording: the first graph's backward after a
    second forward on the same simulator raises instead of returning the
    second rollout's gradients (the shapes would match)."""
    counts, T, K = [2, 2, 2, 2, 2], 5, 2
    classes, sim, p, s0, a, nthr = setup(counts, T, K, 5, seed=19)
    n_slots = sim.n_slots
    slots = sim.slots_of_envs()
    A = torch.ones(n_slots, 6)
    A[slots] = torch.from_numpy(p["Ma"]).float()
    dl = torch.zeros(n_slots, 6)
    dl[slots] = torch.from_numpy(p["dl"]).float()
    dq = torch.zeros(n_slots, 6)
    dq[slots] = torch.from_numpy(p["dq"]).float()
    A, dl, dq = (x.cuda().requires_grad_(True) for x in (A, dl, dq))
    acts = sim.pack_actions(a).requires_grad_(True)
    _, rew1 = AG.rollout(sim, acts, A, dl, dq)
    sim.set_state(s0)
    _, rew2 = AG.rollout(sim, acts, A, dl, dq)
    with pytest.raises(RuntimeError, match="no longer holds"):
        (-rew1.sum()).backward()
    (-rew2.sum()).backward()          # the current recording still differentiates
    torch.cuda.synchronize()
    assert torch.isfinite(acts.grad).all() and torch.isfinite(dl.grad).all()
    sim.close()
