"""GPU adjoint of RK4 runs (the classical fourth-order integrator the
simulator offers beside semi-implicit Euler for the rigid body, Sec. III-A)
against the oracle's forward-mode tangents of the same RK4 rollout: the four
stages of each substep reversed from the substep's start state, for the
multirotor classes, the rudder-propeller and tiltrotor classes and payload
runs, with domain randomisation and ocean current.

Tolerance as for the Euler adjoint: FP32 adjoint vs oracle tangents <= 1e-3
relative per env over random directions; the FP32 gradients of the summed
reward against central differences of the GPU's FP64 RK4 check path <= 1e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads
from tests.helpers import adjoint_vs_oracle_tangents, fp64_reward_differences
from tests.test_gpu_adjoint import gpu_gradients

pytestmark = pytest.mark.gpu

DT = 0.01
RK4 = 1


def rk4_sim(classes, counts, T, K, ckpt, seed, cfg, payload=False):
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=True, reset=cfg, payload=payload,
                record_steps=T, ckpt_every=ckpt, integrator=B.MG_INTEG_RK4)
    sim.reset(seed=seed)
    envs, _ = oracle.reset(classes, workloads.env_classes(counts), cfg, seed)
    nthr = np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])
    s0 = workloads.random_states(seed + 1, sim.n_envs, nthr, pos_scale=2.0, vel_scale=0.3, rate_scale=0.4)
    sim.set_state(s0)
    return sim, envs, s0, nthr


def case(kind):
    if kind == "multirotor":
        return vehicles.five_classes(), [3, 2, 2, 3, 2], dict(vehicles.HOVER_DR), False
    if kind == "actuated":
        return vehicles.actuated_classes(), [4, 5, 3], dict(vehicles.HOVER_DR), False
    return vehicles.five_classes(), [3, 2, 2, 3, 2], dict(vehicles.PAYLOAD_DR), True


@pytest.mark.parametrize("kind,K,ckpt", [("multirotor", 4, 8), ("multirotor", 1, 5), ("actuated", 4, 8),
                                         ("actuated", 2, 7), ("payload", 4, 8)])
def test_rk4_adjoint_matches_oracle_tangents(kind, K, ckpt):
    """T = 24; cotangents on every observation and reward."""
    classes, counts, cfg, payload = case(kind)
    T = 24
    sim, envs, s0, nthr = rk4_sim(classes, counts, T, K, ckpt, 111, cfg, payload)
    E = sim.n_envs
    rng = np.random.default_rng(112)
    a = workloads.actions(113, T, E, lo=-0.99, hi=0.99)
    go = rng.normal(size=(T, E, 13)) * 0.1
    gr = -1.0 + 0.2 * rng.normal(size=(T, E))
    g = gpu_gradients(sim, a, T, go, gr, np.zeros((E, 21)))
    sim.close()
    adjoint_vs_oracle_tangents(classes, envs, s0, a, DT, K, g, go, gr, nthr, np.arange(E), rng, integ=RK4)


def test_rk4_adjoint_sampled_at_4096_envs():
    """4096 envs over the five classes, T = 60, K = 4, a checkpoint every 20
    steps (the launch shape of a full-size backward): 72 sampled envs, every
    class boundary included."""
    classes = vehicles.five_classes()
    counts = workloads.class_counts(4096, 5)
    cfg = dict(vehicles.HOVER_DR)
    T, K = 60, 4
    sim, envs, s0, nthr = rk4_sim(classes, counts, T, K, 20, 121, cfg)
    E = sim.n_envs
    rng = np.random.default_rng(122)
    a = workloads.actions(123, T, E, lo=-0.99, hi=0.99)
    go = (rng.normal(size=(T, E, 13)) * 0.1).astype(np.float32)
    gr = (-1.0 + 0.2 * rng.normal(size=(T, E))).astype(np.float32)
    g = gpu_gradients(sim, a, T, go, gr, np.zeros((E, 21)))
    sim.close()
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 56, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    sub, _ = oracle.reset(classes, workloads.env_classes(counts)[ids], cfg, 121, env_ids=ids)
    adjoint_vs_oracle_tangents(classes, sub, s0, a, DT, K, g, go.astype(np.float64), gr.astype(np.float64),
                               nthr, ids, rng, integ=RK4)


@pytest.mark.parametrize("kind", ["multirotor", "actuated"])
def test_rk4_fp32_adjoint_against_fp64_differences(kind):
    """The FP32 adjoint's added-mass and damping gradients of the summed
    reward against central differences of the GPU's FP64 RK4 check path
    (h = 1e-6), and those differences against the oracle's RK4 tangents."""
    classes, counts, cfg, payload = case(kind)
    T, K = 30, 4
    sim, envs, s0, nthr = rk4_sim(classes, counts, T, K, 10, 131, cfg, payload)
    E = sim.n_envs
    rng = np.random.default_rng(132)
    a = workloads.actions(133, T, E, lo=-0.99, hi=0.99)
    dA, ddl, ddq = (rng.normal(size=(E, 6)) for _ in range(3))
    fd = fp64_reward_differences(sim, sim.pack_actions(a), T, dA, ddl, ddq)
    j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, DT, K, d_Ma=dA, d_dl=ddl, d_dq=ddq, integ=RK4)
    jv = j["d_reward"].sum(0)
    _, _, ref_r = oracle.rollout(classes, envs, s0.astype(np.float64), a, DT, K, integ=RK4)
    roundoff = 64 * np.finfo(np.float64).eps * np.abs(ref_r).sum(0) / 2e-6
    assert np.all(np.abs(fd - jv) <= 1e-6 * np.abs(jv) + roundoff), np.abs(fd - jv).max()
    g = gpu_gradients(sim, a, T, np.zeros((T, E, 13)), np.ones((T, E)), np.zeros((E, 21)))
    sim.close()
    adj = np.einsum("ek,ek->e", g["A"], dA) + np.einsum("ek,ek->e", g["dl"], ddl) + np.einsum("ek,ek->e", g["dq"], ddq)
    assert (np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-3)).max() <= 1e-3
