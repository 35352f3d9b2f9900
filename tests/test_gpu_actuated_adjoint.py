"""GPU adjoint of the model library's other propulsion types (Sec. III-D:
rudder-propeller vehicles with fins, tiltrotor vehicles with servo-tilted
propellers) beside a multirotor class, with domain randomisation and ocean
current, against the oracle's forward-mode tangents: gradients with respect
to the actions, the added-mass and damping coefficients and the initial
state, through the fin lift and drag and the tilt wrench.

Tolerance as for the propeller classes: FP32 adjoint vs oracle tangents
<= 1e-3 relative per env over random directions.
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


def actuated_sim(counts, T, K, ckpt, seed):
    classes = vehicles.actuated_classes()
    cfg = dict(vehicles.HOVER_DR)
    sim = B.Sim(classes, counts, dt=DT, K=K, per_env_params=True, reset=cfg, record_steps=T, ckpt_every=ckpt)
    sim.reset(seed=seed)
    envs, _ = oracle.reset(classes, workloads.env_classes(counts), cfg, seed)
    nthr = np.array([classes[c]["n_thr"] for c in workloads.env_classes(counts)])
    s0 = workloads.random_states(seed + 1, sim.n_envs, nthr, pos_scale=2.0, vel_scale=0.3, rate_scale=0.4)
    sim.set_state(s0)
    return classes, sim, envs, s0, nthr


@pytest.mark.parametrize("K,ckpt", [(4, 8), (1, 5)])
def test_actuated_adjoint_matches_oracle_tangents(K, ckpt):
    """Multirotor, rudder-propeller and tiltrotor envs, T = 24; cotangents on
    every observation and reward."""
    counts = [4, 5, 3]
    T = 24
    classes, sim, envs, s0, nthr = actuated_sim(counts, T, K, ckpt, seed=81)
    E = sim.n_envs
    rng = np.random.default_rng(82)
    a = workloads.actions(83, T, E, lo=-0.99, hi=0.99)
    go = rng.normal(size=(T, E, 13)) * 0.1
    gr = -1.0 + 0.2 * rng.normal(size=(T, E))
    g = gpu_gradients(sim, a, T, go, gr, np.zeros((E, 21)))
    sim.close()
    adjoint_vs_oracle_tangents(classes, envs, s0, a, DT, K, g, go, gr, nthr, np.arange(E), rng)


def test_actuated_adjoint_sampled_at_3072_envs():
    """3072 envs of the three types, T = 60, K = 4, a checkpoint every 20
    steps: 64 sampled envs, every class boundary included."""
    counts = workloads.class_counts(3072, 3)
    T, K = 60, 4
    classes, sim, envs, s0, nthr = actuated_sim(counts, T, K, 20, seed=91)
    E = sim.n_envs
    rng = np.random.default_rng(92)
    a = workloads.actions(93, T, E, lo=-0.99, hi=0.99)
    go = (rng.normal(size=(T, E, 13)) * 0.1).astype(np.float32)
    gr = (-1.0 + 0.2 * rng.normal(size=(T, E))).astype(np.float32)
    g = gpu_gradients(sim, a, T, go, gr, np.zeros((E, 21)))
    sim.close()
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 56, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    sub, _ = oracle.reset(classes, workloads.env_classes(counts)[ids], dict(vehicles.HOVER_DR), 91, env_ids=ids)
    adjoint_vs_oracle_tangents(classes, sub, s0, a, DT, K, g, go.astype(np.float64), gr.astype(np.float64),
                               nthr, ids, rng)


def test_fp32_adjoint_against_fp64_differences():
    """The FP32 adjoint's added-mass and damping gradients of the summed
    reward against central differences of the GPU's FP64 check path
    (h = 1e-6), and those differences against the oracle's tangents."""
    counts = [3, 3, 3]
    T, K = 30, 4
    classes, sim, envs, s0, nthr = actuated_sim(counts, T, K, 10, seed=101)
    E = sim.n_envs
    rng = np.random.default_rng(102)
    a = workloads.actions(103, T, E, lo=-0.99, hi=0.99)
    dA, ddl, ddq = (rng.normal(size=(E, 6)) for _ in range(3))
    fd = fp64_reward_differences(sim, sim.pack_actions(a), T, dA, ddl, ddq)
    j = oracle.rollout_jvp(classes, envs, s0.astype(np.float64), a, DT, K, d_Ma=dA, d_dl=ddl, d_dq=ddq)
    jv = j["d_reward"].sum(0)
    _, _, ref_r = oracle.rollout(classes, envs, s0.astype(np.float64), a, DT, K)
    roundoff = 64 * np.finfo(np.float64).eps * np.abs(ref_r).sum(0) / 2e-6
    assert np.all(np.abs(fd - jv) <= 1e-6 * np.abs(jv) + roundoff), np.abs(fd - jv).max()
    g = gpu_gradients(sim, a, T, np.zeros((T, E, 13)), np.ones((T, E)), np.zeros((E, 21)))
    sim.close()
    adj = np.einsum("ek,ek->e", g["A"], dA) + np.einsum("ek,ek->e", g["dl"], ddl) + np.einsum("ek,ek->e", g["dq"], ddq)
    assert (np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-3)).max() <= 1e-3
