"""CPU pins of the oracle's actuator kinds and of its RK4 variant (Sec. III-D:
rudder-propeller and tiltrotor types, fins with lift and drag that depend on
the angle of attack, servos with the shared first-order model).

Every expected value comes from a closed form for a special case, a library
rotation routine, or an invariant (lift does no work), not from the oracle's
own formulas.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_09203_b300 import vehicles

G = 9.81


def env_of(c, **over):
    e = dict(cls=0, mass=c["mass"], Ig=np.array(c["Ig"]), rg=np.array(c["rg"]), rb=np.array(c["rb"]),
             W=c["mass"] * G, B=c["buoy_ratio"] * c["mass"] * G, Ma=np.array(c["Ma"]),
             dl=np.array(c["dl"]), dq=np.array(c["dq"]), Vc=np.zeros(3), target=np.zeros(3))
    e.update(over)
    return e


def roll(c, e, s0, cmds, dt, K, integ=0):
    envs = oracle.make_envs({k: np.asarray(v)[None] if k != "cls" else np.array([v], np.int32)
                             for k, v in e.items()})
    s = np.array(s0, float).reshape(1, 21).copy()
    a = np.zeros((len(cmds), 1, 8), np.float32)
    for t, cm in enumerate(cmds):
        a[t, 0, :len(cm)] = cm
    s, _, _ = oracle.rollout([c], envs, s, a, dt, K, obs=False, integ=integ)
    return s[0]


def rest(nu=(0.0,) * 6, q=(1.0, 0.0, 0.0, 0.0), n=(0.0,) * 8):
    return np.array([0.0, 0.0, 0.0] + list(q) + list(nu) + list(n))


def one_fin(pos, axis, chord, cl=3.0, cd0=0.05, cda=1.2, area=0.02, rng_=0.4):
    c = dict(vehicles.lauv())
    c.update(n_thr=1, thr_pos=[pos], thr_dir=[(0.0, 0.0, 0.0)], k_f=[0.0], T_rotor=[0.05], deadzone=[0.0],
             act_kind=[vehicles.KIND_FIN], act_link=[0], act_axis=[axis], act_chord=[chord],
             act_range=[rng_], fin_area=[area], fin_cl=[cl], fin_cd0=[cd0], fin_cda=[cda])
    return c


# ---------------------------------------------------------------------------
# Fins.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("th", [-0.35, -0.1, 0.0, 0.05, 0.3])
@pytest.mark.parametrize("fin", [1, 2, 3, 4])
def test_fin_in_pure_surge_closed_form(th, fin):
    """Fin deflected by th in a pure surge flow u x: the angle of attack is
    -th, so F = 1/2 rho S u^2 [C_La sin th cos th (a x x) - (C_D0 + C_Da sin^2 th) x]
    and the moment is r x F; the other fins (undeflected) add drag only."""
    c = vehicles.lauv()
    u = 1.7
    n = np.zeros(5)
    n[fin] = th / c["act_range"][fin]
    tau = oracle.actuator_wrench(c, n, [u, 0, 0, 0, 0, 0])
    q = 0.5 * c["rho"] * u * u
    x = np.array([1.0, 0.0, 0.0])
    F_tot, M_tot = np.zeros(3), np.zeros(3)
    for i in range(1, 5):
        d = th if i == fin else 0.0
        S, a = c["fin_area"][i], np.array(c["act_axis"][i])
        F = q * S * (c["fin_cl"][i] * math.sin(d) * math.cos(d) * np.cross(a, x)
                     - (c["fin_cd0"][i] + c["fin_cda"][i] * math.sin(d) ** 2) * x)
        F_tot += F
        M_tot += np.cross(c["thr_pos"][i], F)
    np.testing.assert_allclose(tau, np.concatenate([F_tot, M_tot]), rtol=1e-13, atol=1e-12)


def test_fin_lift_does_no_work_and_drag_dissipates():
    """The wrench's power on the relative motion is F . (v_r + w x r): zero for a
    lift-only fin (lift is normal to the flow), negative with drag."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        axis = Rotation.random(random_state=rng).apply([0.0, 0.0, 1.0])
        chord = np.cross(axis, rng.normal(size=3))
        chord /= np.linalg.norm(chord)
        pos = rng.uniform(-1, 1, 3)
        nur = rng.uniform(-2, 2, 6)
        n = [rng.uniform(-1, 1)]
        lift_only = one_fin(pos, axis, chord, cd0=0.0, cda=0.0)
        tau = oracle.actuator_wrench(lift_only, n, nur)
        assert abs(tau @ nur) <= 1e-12 * (np.abs(tau).max() * np.abs(nur).max() + 1e-30)
        assert np.abs(tau).max() > 0.0 or abs(n[0]) < 1e-12
        full = one_fin(pos, axis, chord)
        assert oracle.actuator_wrench(full, n, nur) @ nur < 0.0


def test_fin_ignores_flow_along_its_span():
    rng = np.random.default_rng(8)
    for _ in range(50):
        axis = Rotation.random(random_state=rng).apply([0.0, 1.0, 0.0])
        chord = np.cross(axis, rng.normal(size=3))
        chord /= np.linalg.norm(chord)
        pos = rng.uniform(-1, 1, 3)
        c = one_fin(pos, axis, chord)
        nur = rng.uniform(-2, 2, 6)
        extra = np.concatenate([axis * rng.uniform(-3, 3), np.zeros(3)])
        n = [rng.uniform(-1, 1)]
        np.testing.assert_allclose(oracle.actuator_wrench(c, n, nur + extra), oracle.actuator_wrench(c, n, nur),
                                   rtol=1e-12, atol=1e-12)


def test_lauv_steady_surge_with_fin_drag():
    """Full propeller, fins at zero: pure surge with the fins' zero-angle drag
    4 * 1/2 rho S C_D0 u^2 added to the hull's quadratic damping."""
    c = vehicles.lauv()
    e = env_of(c)
    T = c["k_f"][0]
    dl = c["dl"][0]
    dq = c["dq"][0] + sum(0.5 * c["rho"] * c["fin_area"][i] * c["fin_cd0"][i] for i in range(1, 5))
    u_star = (-dl + math.sqrt(dl * dl + 4 * dq * T)) / (2 * dq)
    s = roll(c, e, rest(), [[1.0, 0.0, 0.0, 0.0, 0.0]] * 3000, 0.01, 2)
    assert s[7] == pytest.approx(u_star, rel=1e-9)
    np.testing.assert_allclose(s[8:13], 0.0, atol=1e-12)
    np.testing.assert_allclose(s[3:7], [1.0, 0.0, 0.0, 0.0], atol=1e-12)


def test_rudder_turns_the_lauv_and_elevator_pitches_it():
    """Signs: a positive top/bottom rudder deflection pushes the stern along
    z x x = +y (yaw rate < 0); a positive elevator deflection pushes the stern
    along y x x = -z, up (pitch rate < 0, nose down)."""
    c = vehicles.lauv()
    e = env_of(c)
    s = roll(c, e, rest(), [[1.0, 1.0, 1.0, 0.0, 0.0]] * 200, 0.01, 2)
    assert s[12] < -0.05 and abs(s[11]) < 0.5 * abs(s[12])
    s = roll(c, e, rest(), [[1.0, 0.0, 0.0, 1.0, 1.0]] * 200, 0.01, 2)
    assert s[11] < -0.05 and abs(s[12]) < 0.5 * abs(s[11])


# ---------------------------------------------------------------------------
# Tiltrotor.
# ---------------------------------------------------------------------------
def test_tilted_propellers_match_library_rotation():
    c = vehicles.tilt_hauv()
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = rng.uniform(-1, 1, 8)
        tau = oracle.actuator_wrench(c, n)
        F_tot, M_tot = np.zeros(3), np.zeros(3)
        for i in range(4):
            j = c["act_link"][i]
            th = n[j] * c["act_range"][j]
            d = Rotation.from_rotvec(np.array(c["act_axis"][i]) * th).apply(c["thr_dir"][i])
            F = c["k_f"][i] * n[i] * abs(n[i]) * d
            F_tot += F
            M_tot += np.cross(c["thr_pos"][i], F)
        np.testing.assert_allclose(tau, np.concatenate([F_tot, M_tot]), rtol=1e-12, atol=1e-12)


def test_servo_first_order_response():
    """Servo channels share the first-order model: n_k = c (1 - (1 - alpha)^k)."""
    c = vehicles.tilt_hauv()
    e = env_of(c)
    h = 0.01
    s = rest()
    alpha = 1.0 - math.exp(-h / c["T_rotor"][5])
    for k in range(1, 30):
        s = roll(c, e, s, [[0, 0, 0, 0, 0, 0.6, 0, 0]], h, 1)
        c6 = float(np.float32(0.6))   # commands are FP32
        assert s[13 + 5] == pytest.approx(c6 * (1 - (1 - alpha) ** k), rel=1e-13)


@pytest.mark.parametrize("integ", [0, 1])
@pytest.mark.parametrize("cls", ["lauv", "tilt"])
def test_rest_stays_rest_bit_exact(cls, integ):
    c = vehicles.lauv() if cls == "lauv" else vehicles.tilt_hauv()
    e = env_of(c, rb=np.array([0.0, 0.0, -0.02]))
    s = roll(c, e, rest(), [[0.0] * 8] * 50, 0.01, 4, integ=integ)
    assert np.array_equal(s, rest())


# ---------------------------------------------------------------------------
# RK4 variant.
# ---------------------------------------------------------------------------
def test_rk4_linear_decay_is_the_degree_four_taylor_factor():
    c = vehicles.heavy8()
    e = env_of(c, dq=np.zeros(6), rb=np.zeros(3))
    h, u0, n = 0.01, 0.8, 40
    z = h * c["dl"][0] / (c["mass"] + c["Ma"][0])
    f = 1 - z + z * z / 2 - z ** 3 / 6 + z ** 4 / 24
    s = roll(c, e, rest(nu=(u0, 0, 0, 0, 0, 0)), [[0.0] * 8] * n, h, 1, integ=1)
    assert s[7] == pytest.approx(u0 * f ** n, rel=1e-13)
    assert s[0] > 0 and np.abs(s[8:13]).max() == 0.0


def test_rk4_pure_yaw_closed_form():
    """Constant yaw rate w (no yaw damping, principal axes): each RK4 step
    multiplies q by (1 - x^2/2 + x^4/24, 0, 0, x - x^3/6), x = h w / 2."""
    c = vehicles.heavy8()
    dl = np.array(c["dl"]); dl[5] = 0.0
    dq = np.array(c["dq"]); dq[5] = 0.0
    e = env_of(c, dl=dl, dq=dq, rb=np.zeros(3))
    w, h, n = 0.9, 0.02, 25
    s = roll(c, e, rest(nu=(0, 0, 0, 0, 0, w)), [[0.0] * 8] * n, h, 1, integ=1)
    x = h * w / 2
    step = 2 * math.atan2(x - x ** 3 / 6, 1 - x * x / 2 + x ** 4 / 24)
    yaw = 2 * math.atan2(s[6], s[3])
    assert yaw == pytest.approx(n * step, rel=1e-12)
    assert s[12] == w and np.abs(s[0:3]).max() == 0.0


def _drift_error(h, integ, T=0.6):
    c = vehicles.heavy8()
    e = env_of(c, dl=np.zeros(6), dq=np.zeros(6), rb=np.zeros(3))
    s0 = rest(nu=(0.4, -0.3, 0.2, 0.9, -0.7, 1.1))
    n = int(round(T / h))
    return roll(c, e, s0, [[0.0] * 8] * n, h, 1, integ=integ)


def test_rk4_converges_at_fourth_order():
    ref = _drift_error(0.6 / 1024, 1)
    e1 = np.linalg.norm(_drift_error(0.6 / 32, 1) - ref)
    e2 = np.linalg.norm(_drift_error(0.6 / 64, 1) - ref)
    assert 12.0 < e1 / e2 < 20.0
    # Euler on the same problem is first order.
    ref_e = _drift_error(0.6 / 8192, 0)
    f1 = np.linalg.norm(_drift_error(0.6 / 256, 0) - ref_e)
    f2 = np.linalg.norm(_drift_error(0.6 / 512, 0) - ref_e)
    assert 1.6 < f1 / f2 < 2.4
