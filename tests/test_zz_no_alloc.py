"""The allocation-free adjoint entry point (mg_step_backward_noalloc).

It serves callers that cannot allocate device memory while they run the
backward pass (a framework that owns the device through its own pool, a
process whose memory budget is already committed, a loop that must not take
cudaMalloc's implicit synchronisation). Its scratch is a fixed array compiled
into the library, so it must give the same gradients as mg_step_backward, on
consecutive calls that reuse that array, and refuse sizes beyond the array.

This file is collected last and passes both alone and after the other tests
(the first call in a process does the per-device set-up).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles, workloads

pytestmark = pytest.mark.gpu


def grads(fn, sim, acts, g_obs, g_rew, T):
    g_act = torch.zeros(T, sim.action_floats, device="cuda")
    gA = torch.zeros(sim.n_slots, 6, device="cuda")
    gD = torch.zeros(sim.n_slots, 12, device="cuda")
    g0 = torch.zeros(sim.n_slots, 21, device="cuda")
    fn(sim.handle, acts, g_obs, g_rew, None, g_act, gA, gD, g0)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (g_act, gA, gD, g0)]


def test_noalloc_backward_matches_backward_on_two_calls():
    classes = vehicles.five_classes()
    counts = [6, 5, 4, 7, 3]
    T, K, ckpt = 30, 4, 10
    sim = B.Sim(classes, counts, dt=0.01, K=K, per_env_params=True, reset=dict(vehicles.HOVER_DR),
                record_steps=T, ckpt_every=ckpt)
    rng = np.random.default_rng(0)
    for call in range(2):
        sim.reset(seed=100 + call)
        acts = sim.pack_actions(workloads.actions(200 + call, T, sim.n_envs, lo=-0.99, hi=0.99))
        obs = torch.zeros(T, sim.n_slots, 13, device="cuda")
        rew = torch.zeros(T, sim.n_slots, device="cuda")
        B.mg_rollout(sim.handle, acts, T, obs, rew, True)
        g_obs = torch.from_numpy(rng.normal(size=(T, sim.n_slots, 13)).astype(np.float32)).cuda()
        g_rew = torch.from_numpy(rng.normal(size=(T, sim.n_slots)).astype(np.float32)).cuda()
        ref = grads(B.mg_step_backward, sim, acts, g_obs, g_rew, T)
        got = grads(B.mg_step_backward_noalloc, sim, acts, g_obs, g_rew, T)
        for r, g in zip(ref, got):
            np.testing.assert_allclose(g, r, rtol=1e-6, atol=1e-7)
        assert any(np.abs(r).max() > 0 for r in ref)
    sim.status()
    sim.close()


def test_noalloc_backward_refuses_scratch_beyond_its_array():
    classes = vehicles.five_classes()
    counts = workloads.class_counts(65536, 5)
    sim = B.Sim(classes, counts, dt=0.01, K=4, per_env_params=True, reset=dict(vehicles.HOVER), record_steps=2,
                ckpt_every=20)
    acts = sim.new_actions(2)
    B.mg_rollout(sim.handle, acts, 2, None, None, True)
    with pytest.raises(B.MGError) as e:
        B.mg_step_backward_noalloc(sim.handle, acts, None, None, None, None, None, None, None)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
    sim.close()
