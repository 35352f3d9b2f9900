"""GPU parity of the class-specialised step kernels (the one-lane step kernel
compiled at run time with a class's constants as literals) against the FP64
oracle and against the kernels built with the library.

Tolerance: one-step relative state error <= 1e-5 against the oracle; the
specialised and library-built kernels agree to rounding (2e-6 after one
step, 2e-5 after a 20-step rollout).
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


@pytest.mark.parametrize("K", [4, 1, 8])
def test_specialised_kernels_run_and_match_oracle_and_library_kernels(K):
    """At K = 4 (the workload), 1 and 8 substeps per step."""
    classes = vehicles.five_classes()
    classes[1] = dict(classes[1], deadzone=[0.25] * 4)        # a class with a dead zone among them
    counts = workloads.class_counts(1 << 20, 5)
    cfg = dict(vehicles.HOVER)
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=False, reset=cfg)
    shape = B.mg_get_launch_shape(sim.handle)
    assert shape["specialised"] == 1 and shape["specialised_launches"] == 5, shape
    sim.reset(seed=81)
    s0 = sim.get_state()
    E = sim.n_envs
    rng = np.random.default_rng(82)
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 1500, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    a_s = workloads.actions(83, 1, len(ids))
    a_env = np.zeros((1, E, 8), np.float32)
    a_env[:, ids] = a_s
    a_dev = sim.pack_actions(a_env)
    out = {}
    for spec in (1, 0):
        B.mg_set_launch_shape(sim.handle, 1, 0, spec)
        assert B.mg_get_launch_shape(sim.handle)["specialised_launches"] == (5 if spec else 0)
        sim.set_state(s0)
        sim.step(a_dev)
        torch.cuda.synchronize()
        out[spec] = (sim.get_state(), sim.obs.cpu().numpy().copy(), sim.reward.cpu().numpy().copy())
    slots = sim.slots_of_envs()[ids]
    envs, _ = oracle.reset(classes, workloads.env_classes(counts)[ids], cfg, 81, env_ids=ids)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0[ids].astype(np.float64), a_s, 0.01, K)
    err = rel_state_err(out[1][0][ids], ref)
    assert err.max() <= 1e-5, (err.max(), int(ids[np.argmax(err)]))
    np.testing.assert_allclose(out[1][1][slots], o_ref[0], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(out[1][2][slots], r_ref[0], rtol=1e-5, atol=1e-4)
    assert rel_state_err(out[1][0], out[0][0].astype(np.float64)).max() <= 2e-6
    # A 20-step rollout (the multi-step instantiations) of both kinds.
    T = 20
    a_all = torch.rand(T, sim.action_floats, device="cuda") * 2 - 1
    fin = {}
    for spec in (1, 0):
        B.mg_set_launch_shape(sim.handle, 1, 0, spec)
        sim.set_state(s0)
        sim.rollout(a_all, T)
        torch.cuda.synchronize()
        fin[spec] = sim.get_state()
    assert rel_state_err(fin[1], fin[0].astype(np.float64)).max() <= 2e-5
    sim.status()
    sim.close()


def test_per_env_specialised_kernels_match_oracle_and_library_kernels():
    """Per-env parameters (DR and current) at a size that runs one launch per
    class: the class-specialised kernels (actuator tables as literals, the
    physics from the parameter planes) against the oracle on sampled envs
    (every class boundary included) and against the library-built kernels
    (rounding), after one step and after a 20-step rollout."""
    classes = vehicles.five_classes()
    counts = [300001, 3, 240001, 5, 9]
    cfg = dict(vehicles.HOVER_DR)
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=cfg)
    assert sim.launches_per_step() == 5
    assert B.mg_get_launch_shape(sim.handle)["specialised_launches"] == 5
    sim.reset(seed=91)
    s0 = sim.get_state()
    E = sim.n_envs
    rng = np.random.default_rng(92)
    bounds = np.cumsum(counts)
    ids = np.unique(np.concatenate([rng.choice(E, 1500, replace=False), [0, E - 1], bounds[:-1], bounds[:-1] - 1]))
    a_s = workloads.actions(93, 1, len(ids))
    a_env = np.zeros((1, E, 8), np.float32)
    a_env[:, ids] = a_s
    a_dev = sim.pack_actions(a_env)
    out = {}
    for spec in (1, 0):
        B.mg_set_launch_shape(sim.handle, 1, 0, spec)
        sim.set_state(s0)
        sim.step(a_dev)
        torch.cuda.synchronize()
        out[spec] = (sim.get_state(), sim.obs.cpu().numpy().copy(), sim.reward.cpu().numpy().copy())
    slots = sim.slots_of_envs()[ids]
    envs, _ = oracle.reset(classes, workloads.env_classes(counts)[ids], cfg, 91, env_ids=ids)
    ref, o_ref, r_ref = oracle.rollout(classes, envs, s0[ids].astype(np.float64), a_s, 0.01, 4)
    err = rel_state_err(out[1][0][ids], ref)
    assert err.max() <= 1e-5, (err.max(), int(ids[np.argmax(err)]))
    np.testing.assert_allclose(out[1][1][slots], o_ref[0], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(out[1][2][slots], r_ref[0], rtol=1e-5, atol=1e-4)
    assert rel_state_err(out[1][0], out[0][0].astype(np.float64)).max() <= 2e-6
    T = 20
    a_all = torch.rand(T, sim.action_floats, device="cuda") * 2 - 1
    fin = {}
    for spec in (1, 0):
        B.mg_set_launch_shape(sim.handle, 1, 0, spec)
        sim.set_state(s0)
        sim.rollout(a_all, T)
        torch.cuda.synchronize()
        fin[spec] = sim.get_state()
    assert rel_state_err(fin[1], fin[0].astype(np.float64)).max() <= 2e-5
    sim.status()
    sim.close()
