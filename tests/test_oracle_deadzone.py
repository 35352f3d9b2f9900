"""CPU pins of the oracle's propeller dead zone (paper Sec. III-D: the thrust
of a propeller is a quadratic function of its speed with a dead zone).

Reading: f = k n|n| when |n| >= delta, and f = 0 when |n| < delta, with n the
rotor state after its first-order lag; the force acts along the thruster axis
d at its position r (wrench [f d ; r x f d]). Each test fixes what the model
fixes independently of the oracle's code: zero wrench strictly inside, the
jump k delta^2 at the threshold, each thruster's own threshold, a neutral
vehicle held inside the dead zone staying at rest bit for bit, the closed-form
steady surge speed outside it, and a zero tangent inside it.
"""
import math

import numpy as np

import oracle
from paper_2503_09203_b300 import vehicles
from tests.test_oracle_pins import env_from_class, rest_state, steps

K_F = 30.0


def surge_pair(deadzone, T_rotor=0.05):
    """Two thrusters along body x at (0, +-0.1, 0): pure surge force, and a
    yaw moment -0.1 f (+0.1 f) from each."""
    c = dict(vehicles.heavy8())
    c.update(n_thr=2, thr_pos=[(0.0, 0.1, 0.0), (0.0, -0.1, 0.0)], thr_dir=[(1.0, 0.0, 0.0)] * 2,
             k_f=[K_F, K_F], T_rotor=[T_rotor, T_rotor], deadzone=list(deadzone))
    return c


def wrench_of_first(c, n0):
    return oracle.actuator_wrench(c, [n0, 0.0])


def test_wrench_is_exactly_zero_strictly_inside_the_dead_zone():
    c = surge_pair([0.3, 0.1])
    for n0 in (0.0, 0.1, -0.1, 0.2999, -0.2999, np.nextafter(0.3, 0.0), -np.nextafter(0.3, 0.0)):
        tau = wrench_of_first(c, n0)
        assert np.array_equal(tau, np.zeros(6)), (n0, tau)


def test_wrench_at_and_above_the_threshold_is_quadratic_along_the_axis():
    c = surge_pair([0.3, 0.1])
    for n0 in (0.3, -0.3, np.nextafter(0.3, 1.0), 0.5, -0.75, 1.0):
        f = K_F * n0 * abs(n0)
        # Force f along x at r = (0, 0.1, 0): moment r x (f, 0, 0) = (0, 0, -0.1 f).
        np.testing.assert_allclose(wrench_of_first(c, n0), [f, 0, 0, 0, 0, -0.1 * f], rtol=1e-15, atol=0)
    # The jump at the threshold is k delta^2 (nothing below, full thrust at it).
    below, at = wrench_of_first(c, np.nextafter(0.3, 0.0))[0], wrench_of_first(c, 0.3)[0]
    assert below == 0.0 and abs(at - K_F * 0.09) <= 1e-15 * K_F


def test_each_thruster_uses_its_own_threshold():
    c = surge_pair([0.3, 0.1])
    tau = oracle.actuator_wrench(c, [0.2, 0.2])      # thruster 0 inside, thruster 1 outside
    f1 = K_F * 0.04
    # Only thruster 1 at r = (0, -0.1, 0) pushes: moment (0, 0, +0.1 f1).
    np.testing.assert_allclose(tau, [f1, 0, 0, 0, 0, 0.1 * f1], rtol=1e-15, atol=0)
    tau = oracle.actuator_wrench(c, [-0.05, 0.35])    # thruster 0 inside its 0.3, thruster 1 beyond its 0.1
    f1 = K_F * 0.35 * 0.35
    np.testing.assert_allclose(tau, [f1, 0, 0, 0, 0, 0.1 * f1], rtol=1e-15, atol=0)


def test_neutral_vehicle_commanded_inside_the_dead_zone_stays_at_rest():
    """Neutral heavy8 (CoB straight above the CoG) with every propeller's dead
    zone at 0.3125: commands with |c| < 0.3125 spin the rotors up along
    c (1 - (1 - alpha)^k) but never reach the threshold, so pose and velocity
    stay bit-identical for 200 steps."""
    c = dict(vehicles.heavy8(), deadzone=[0.3125] * 8)
    e = env_from_class(c)
    rng = np.random.default_rng(5)
    cmd = rng.uniform(-0.31, 0.31, 8).astype(np.float32)
    s0 = rest_state(p=(0.5, -1.0, 2.0))
    K, dt = 4, 0.01
    tr = steps(c, e, s0, 200, dt, K=K, action=cmd)
    assert np.array_equal(tr[:, :13], np.repeat(s0[None, :13], len(tr), 0))
    alpha = 1.0 - math.exp(-(dt / K) / c["T_rotor"][0])
    k = 200 * K
    np.testing.assert_allclose(tr[-1, 13:21], cmd.astype(np.float64) * (1 - (1 - alpha) ** k), rtol=1e-12)


def test_steady_surge_outside_and_no_motion_inside():
    """Symmetric surge thrust from commands beyond the dead zone reaches the
    closed-form speed u* = (-d_l + sqrt(d_l^2 + 4 d_q T)) / (2 d_q) with
    T = 2 k c|c|; commands inside it produce no motion at all."""
    c = surge_pair([0.25, 0.25])
    e = env_from_class(c)
    dl, dq = c["dl"][0], c["dq"][0]
    for cmd in (0.6, -0.4, 0.26):
        cmd = float(np.float32(cmd))   # commands are FP32 inputs
        Tn = 2 * K_F * cmd * abs(cmd)
        u_star = math.copysign((-dl + math.sqrt(dl * dl + 4 * dq * abs(Tn))) / (2 * dq), Tn)
        tr = steps(c, e, rest_state(), 3000, 0.01, action=[cmd, cmd])
        assert abs(tr[-1, 7] - u_star) <= 1e-9 * abs(u_star), (cmd, tr[-1, 7], u_star)
    tr = steps(c, e, rest_state(), 500, 0.01, action=[0.24, -0.2])
    assert np.all(tr[:, 0:13] == rest_state()[None, 0:13])


def test_tangent_is_zero_inside_and_matches_differences_outside():
    """Forward-mode tangent of a surge rollout with respect to the commands:
    exactly zero while the rotors stay inside the dead zone; equal to central
    differences of the oracle's own rollout when they are outside."""
    c = surge_pair([0.3, 0.3])
    e = env_from_class(c)
    envs = oracle.make_envs({k: np.asarray(v)[None] if k != "cls" else np.array([0], np.int32) for k, v in e.items()})
    T, K = 30, 2
    for cmd, inside in ((0.2, True), (0.7, False)):
        a = np.zeros((T, 1, 8), np.float32)
        a[:, 0, :2] = cmd
        d = np.zeros((T, 1, 8))
        d[:, 0, :2] = 1.0
        j = oracle.rollout_jvp([c], envs, rest_state().reshape(1, 21), a, 0.01, K, d_actions=d)
        if inside:
            # Only the command term of the reward (-0.01 |c|^2) still depends on c.
            assert np.all(j["d_state"][0, :13] == 0.0)
            np.testing.assert_allclose(j["d_reward"][:, 0], -0.02 * 2 * float(np.float32(cmd)), rtol=1e-12)
        else:
            h = 1e-4
            ap, am = a.copy(), a.copy()
            ap[:, 0, :2] = np.float32(cmd + h)
            am[:, 0, :2] = np.float32(cmd - h)
            c32 = float(np.float32(cmd))
            hp = float(np.float32(cmd + h)) - c32
            hm = c32 - float(np.float32(cmd - h))
            s_p = rest_state().reshape(1, 21).copy()
            s_m = rest_state().reshape(1, 21).copy()
            s_p, _, _ = oracle.rollout([c], envs, s_p, ap, 0.01, K)
            s_m, _, _ = oracle.rollout([c], envs, s_m, am, 0.01, K)
            fd = (s_p[0, 7] - s_m[0, 7]) / (hp + hm)
            assert abs(j["d_state"][0, 7] - fd) <= 1e-6 * abs(fd), (j["d_state"][0, 7], fd)
