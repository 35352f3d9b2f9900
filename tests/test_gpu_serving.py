"""Serving loop (continuous batching): admission by device memory, shared
launches across requests, and per-request results that are identical alone
and in the mix and match the oracle.

A request's random draws (reset and actions) are keyed by its own seed and
its envs' indices within the request, so its trajectory does not depend on
which other requests share its launches.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle
from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import vehicles
from tests.helpers import rel_state_err

pytestmark = pytest.mark.gpu

CFG = dict(vehicles.HOVER_DR)


def run_alone(classes, req, budget=256 << 20, cfg=CFG, integ=B.MG_INTEG_EULER):
    srv = B.mg_server_create(classes, 0.01, budget_bytes=budget, max_requests=64, reset=cfg, integrator=integ)
    rid = B.mg_server_submit(srv, *req)
    B.mg_server_wait_idle(srv, 120)
    out = B.mg_server_poll(srv, rid)
    B.mg_server_destroy(srv)
    return out


def oracle_request(classes, req, cfg=CFG, integ=0):
    cls, n, horizon, K, seed = req
    envs, s = oracle.reset(classes, np.full(n, cls, np.int32), cfg, seed)
    a = np.zeros((horizon, n, 8), np.float32)
    nt = classes[cls]["n_thr"]
    for t in range(horizon):
        for e in range(n):
            for i in range(nt):
                a[t, e, i] = oracle.action(seed, e, t, i)
    s, _, r = oracle.rollout(classes, envs, s, a, 0.01, K, integ=integ)
    return s, r.sum(0)


@pytest.mark.parametrize("cfg", [CFG, dict(vehicles.HOVER)], ids=["per_env_dr", "class_constants"])
def test_request_alone_equals_in_mix_and_matches_oracle(cfg):
    """Per-env DR and current (ticks read per-env parameter planes), or
    neither (ticks read the class tables; the probe's class has a dead zone)."""
    classes = vehicles.five_classes()
    if not cfg["dr_enabled"]:
        classes[2] = dict(classes[2], deadzone=[0.25] * 6)
    probe = (2, 37, 40, 3, 1234567)
    alone = run_alone(classes, probe, cfg=cfg)
    assert alone["status"] == B.MG_REQ_DONE and alone["steps_done"] == 40
    srv = B.mg_server_create(classes, 0.01, budget_bytes=256 << 20, max_requests=64, reset=cfg)
    rng = np.random.default_rng(0)
    # 60 others: each thruster-count group of a tick holds more segments than
    # the kernel keeps in shared memory, so tiles find theirs through the
    # tick's tile map.
    others = [(int(rng.integers(0, 5)), int(rng.integers(1, 3000)), int(rng.integers(5, 60)),
               int(rng.integers(1, 9)), int(rng.integers(1 << 40))) for _ in range(60)]
    ids = [B.mg_server_submit(srv, *r) for r in others[:30]]
    time.sleep(0.02)                      # the probe arrives while others run
    pid = B.mg_server_submit(srv, *probe)
    for r in others[30:]:
        ids.append(B.mg_server_submit(srv, *r))
        time.sleep(0.002)
    B.mg_server_wait_idle(srv, 300)
    mixed = B.mg_server_poll(srv, pid)
    st = B.mg_server_stats_get(srv)
    B.mg_server_destroy(srv)
    assert mixed["status"] == B.MG_REQ_DONE
    assert np.array_equal(mixed["final_state"], alone["final_state"])
    assert np.array_equal(mixed["returns"], alone["returns"])
    # Shared launches actually happened: fewer ticks than total request steps.
    assert st["ticks"] < sum(r[2] for r in others) + probe[2]
    s_ref, ret_ref = oracle_request(classes, probe, cfg=cfg)
    err = rel_state_err(alone["final_state"].astype(np.float64), s_ref)
    assert err.max() <= 1e-3, err.max()
    np.testing.assert_allclose(alone["returns"], ret_ref, rtol=1e-4, atol=1e-3)


@pytest.mark.parametrize("cfg,integ", [(CFG, B.MG_INTEG_EULER), (dict(vehicles.HOVER), B.MG_INTEG_EULER),
                                       (CFG, B.MG_INTEG_RK4), (dict(vehicles.HOVER), B.MG_INTEG_RK4)],
                         ids=["per_env_dr", "class_constants", "per_env_dr_rk4", "class_constants_rk4"])
def test_generic_classes_alone_equal_in_mix_and_match_oracle(cfg, integ):
    """The model library's other propulsion types served beside propeller
    classes: a rudder-propeller (fins), a tiltrotor (servo-tilted
    propellers) and a multirotor request, each identical alone and in a mix
    of all five classes, and equal to the oracle; with the semi-implicit
    Euler or the RK4 substep for every request."""
    classes = vehicles.actuated_classes() + [vehicles.five_classes()[1], vehicles.five_classes()[4]]
    probes = [(1, 29, 30, 4, 424242), (2, 33, 25, 2, 737373), (4, 41, 20, 3, 919191)]
    alone = [run_alone(classes, p, cfg=cfg, integ=integ) for p in probes]
    for a in alone:
        assert a["status"] == B.MG_REQ_DONE
    srv = B.mg_server_create(classes, 0.01, budget_bytes=256 << 20, max_requests=64, reset=cfg, integrator=integ)
    rng = np.random.default_rng(3)
    others = [(int(rng.integers(0, 5)), int(rng.integers(1, 2000)), int(rng.integers(5, 40)),
               int(rng.integers(1, 9)), int(rng.integers(1 << 40))) for _ in range(40)]
    ids = [B.mg_server_submit(srv, *r) for r in others[:20]]
    time.sleep(0.02)
    pids = [B.mg_server_submit(srv, *p) for p in probes]
    for r in others[20:]:
        ids.append(B.mg_server_submit(srv, *r))
        time.sleep(0.002)
    B.mg_server_wait_idle(srv, 300)
    mixed = [B.mg_server_poll(srv, pid) for pid in pids]
    B.mg_server_destroy(srv)
    for p, a, m in zip(probes, alone, mixed):
        assert m["status"] == B.MG_REQ_DONE
        assert np.array_equal(m["final_state"], a["final_state"])
        assert np.array_equal(m["returns"], a["returns"])
        s_ref, ret_ref = oracle_request(classes, p, cfg=cfg, integ=integ)
        err = rel_state_err(a["final_state"].astype(np.float64), s_ref)
        assert err.max() <= 1e-3, (p, err.max())
        np.testing.assert_allclose(a["returns"], ret_ref, rtol=1e-4, atol=1e-3)


def test_admission_waits_for_memory_and_refuses_impossible_requests():
    classes = vehicles.five_classes()
    # Budget for roughly 2 x 4096 envs: requests queue until space frees up.
    per_slot = 16 * 10 + 4 + 21 * 4
    srv = B.mg_server_create(classes, 0.01, budget_bytes=per_slot * 8200, max_requests=16, reset=CFG)
    with pytest.raises(B.MGError) as e:
        B.mg_server_submit(srv, 0, 100000, 10, 1, 1)
    assert e.value.code == B.MG_ERR_ADMISSION_REFUSED
    ids = [B.mg_server_submit(srv, k % 5, 4000, 20, 2, k) for k in range(8)]
    B.mg_server_wait_idle(srv, 300)
    res = [B.mg_server_poll(srv, i) for i in ids]
    assert all(r["status"] == B.MG_REQ_DONE for r in res)
    # The arena holds two of these requests at a time (slots: 8200 / 4000):
    # the server's own account of the bytes held by admitted requests never
    # exceeded the budget, and requests ran two at a time, not more.
    st = B.mg_server_stats_get(srv)
    assert st["budget_bytes"] == per_slot * 8200
    assert 0 < st["peak_resident_bytes"] <= st["budget_bytes"]
    assert st["peak_requests"] == 2
    need = [4000 * (16 * 10 + 4) + 4 * 4000 * (13 + classes[k % 5]["n_thr"]) for k in range(8)]
    assert st["peak_resident_bytes"] >= min(a + b for a, b in zip(need, need[1:]))
    for i in ids:
        B.mg_server_release(srv, i)
    assert B.mg_server_poll(srv, ids[0])["status"] == B.MG_REQ_UNKNOWN
    with pytest.raises(B.MGError):
        B.mg_server_submit(srv, 7, 10, 10, 1, 1)   # no such class
    B.mg_server_destroy(srv)


def test_serving_stats_report_latency_quantiles():
    classes = vehicles.five_classes()
    srv = B.mg_server_create(classes, 0.01, budget_bytes=128 << 20, max_requests=64, reset=CFG)
    rng = np.random.default_rng(4)
    for k in range(30):
        B.mg_server_submit(srv, int(rng.integers(0, 5)), int(rng.integers(1, 2000)), int(rng.integers(1, 50)),
                           int(rng.integers(1, 9)), k)
    B.mg_server_wait_idle(srv, 300)
    st = B.mg_server_stats_get(srv)
    B.mg_server_destroy(srv)
    assert st["requests_done"] == 30
    assert 0 < st["step_latency_p50"] <= st["step_latency_p99"]
    assert 0 < st["tick_p50"] <= st["tick_p99"]
    assert st["env_steps"] > 0 and st["busy_seconds"] > 0
