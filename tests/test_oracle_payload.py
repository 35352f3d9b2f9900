"""CPU pins of the oracle's payload model (Sec. III-B mission payloads, Table 2
payload mass): a point mass rigidly attached to the vehicle moves the CoG off
the body origin and couples translation and rotation through M_RB, C_RB and
the restoring moment (Fossen 2011, Eq. 6.37 and 6.43).

Each pin follows from mechanics the oracle's code does not share: the kinetic
energy of the vehicle plus a point mass, the moment of the two weights, the
resting attitude of a pendulum, Kirchhoff's impulses of a free body.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_09203_b300 import vehicles, workloads

G = 9.81
PAYLOAD = vehicles.PAYLOAD


def draws(seed, env, mass):
    """The payload the reset draws for one env (stream 1, draws 23-26)."""
    u = [oracle.uniform(seed, 1, env, j) for j in (23, 24, 25, 26)]
    mp = mass * (PAYLOAD["payload_lo"] + (PAYLOAD["payload_hi"] - PAYLOAD["payload_lo"]) * u[0])
    rp = np.array([-0.1 + 0.2 * u[1], -0.1 + 0.2 * u[2], 0.05 + 0.1 * u[3]])
    return mp, rp


def env_dict(arr, i):
    keys = ("mass", "Ig", "rg", "rb", "W", "B", "Ma", "dl", "dq", "Vc", "target", "Ig_off")
    d = {k: np.array(arr[k][i]) for k in keys}
    d["cls"] = int(arr["cls"][i])
    return d


@pytest.fixture(scope="module")
def payload_envs():
    classes = vehicles.five_classes()
    counts = [3, 3, 3, 3, 3]
    envs, s0 = oracle.reset(classes, workloads.env_classes(counts), PAYLOAD, 17)
    return classes, counts, oracle.envs_to_arrays(envs)


def test_composite_kinetic_energy(payload_envs):
    """1/2 nu^T M_RB nu = vehicle's 1/2 m |v|^2 + 1/2 w^T Ig w plus the point
    mass's 1/2 m_p |v + w x r_p|^2 (added mass zeroed)."""
    classes, counts, arr = payload_envs
    rng = np.random.default_rng(0)
    cls_of = workloads.env_classes(counts)
    for i in range(len(cls_of)):
        c = classes[cls_of[i]]
        mp, rp = draws(17, i, c["mass"])
        assert mp > 0
        e = env_dict(arr, i)
        e["Ma"] = np.zeros(6)
        M = oracle.mass_matrix(e)
        np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
        for _ in range(5):
            nu = rng.uniform(-1, 1, 6)
            v, w = nu[:3], nu[3:]
            ke = 0.5 * c["mass"] * v @ v + 0.5 * np.sum(np.array(c["Ig"]) * w * w)
            vp = v + np.cross(w, rp)
            ke += 0.5 * mp * vp @ vp
            assert 0.5 * nu @ M @ nu == pytest.approx(ke, rel=1e-12)


def test_mass_weight_and_cog(payload_envs):
    classes, counts, arr = payload_envs
    cls_of = workloads.env_classes(counts)
    for i in range(len(cls_of)):
        c = classes[cls_of[i]]
        mp, rp = draws(17, i, c["mass"])
        assert arr["mass"][i] == pytest.approx(c["mass"] + mp, rel=1e-14)
        assert arr["W"][i] == pytest.approx((c["mass"] + mp) * G, rel=1e-14)
        np.testing.assert_allclose(arr["rg"][i] * (c["mass"] + mp), mp * rp, rtol=1e-12, atol=1e-15)


def test_restoring_moment_of_two_weights(payload_envs):
    """The weights m g at the origin and m_p g at r_p and the buoyancy B at r_b:
    g(eta) = -[sum of forces; sum of moments] in the body frame."""
    classes, counts, arr = payload_envs
    rng = np.random.default_rng(1)
    cls_of = workloads.env_classes(counts)
    for i in range(len(cls_of)):
        c = classes[cls_of[i]]
        mp, rp = draws(17, i, c["mass"])
        e = env_dict(arr, i)
        for _ in range(4):
            q = Rotation.random(random_state=rng).as_quat()[[3, 0, 1, 2]]
            R = oracle.rotation(q)
            down = R.T @ np.array([0.0, 0.0, 1.0])
            F = (c["mass"] * G + mp * G - e["B"]) * down
            Mo = np.cross(rp, mp * G * down) + np.cross(e["rb"], -e["B"] * down)
            g = oracle.restoring(e, q)
            np.testing.assert_allclose(g, -np.concatenate([F, Mo]), atol=1e-10 * (c["mass"] * G))


def test_neutral_vehicle_settles_like_a_pendulum(payload_envs):
    """With buoyancy equal to the total weight, the body comes to rest with
    the net moment arm W' r_g - B r_b pointing straight down."""
    classes, counts, arr = payload_envs
    for i in (0, 4):   # a 11.5 kg and a 10 kg vehicle
        c = classes[workloads.env_classes(counts)[i]]
        e = env_dict(arr, i)
        e["B"] = e["W"]
        e["cls"] = 0   # the rollout below gets this env's class alone
        envs = oracle.make_envs({k: np.asarray(v)[None] if k != "cls" else np.array([v], np.int32)
                                 for k, v in e.items()})
        s = np.zeros((1, 21))
        s[0, 3] = 1.0
        T = 4000
        a = np.zeros((T, 1, 8), np.float32)
        s, _, _ = oracle.rollout([c], envs, s, a, 0.01, 2, obs=False)
        R = oracle.rotation(s[0, 3:7])
        down = R.T @ np.array([0.0, 0.0, 1.0])
        arm = e["W"] * e["rg"] - e["B"] * e["rb"]
        np.testing.assert_allclose(down, arm / np.linalg.norm(arm), atol=1e-6)
        np.testing.assert_allclose(s[0, 7:13], 0.0, atol=1e-7)


def _free_drift(e, c, h, T=1.0):
    """Free body in an ideal fluid (no damping, no restoring, no current)."""
    nu0 = np.array([0.4, -0.3, 0.2, 0.6, -0.5, 0.7])
    envs = oracle.make_envs({k: np.asarray(v)[None] if k != "cls" else np.array([v], np.int32)
                             for k, v in e.items()})
    s = np.zeros((1, 21))
    s[0, 3] = 1.0
    s[0, 7:13] = nu0
    M = oracle.mass_matrix(e)

    def impulses(st):
        R = oracle.rotation(st[3:7])
        hm = M @ st[7:13]
        P = R @ hm[:3]
        return P, R @ hm[3:] + np.cross(st[0:3], P), 0.5 * st[7:13] @ hm

    first = impulses(s[0])
    n = int(round(T / h))
    s, _, _ = oracle.rollout([c], envs, s, np.zeros((n, 1, 8), np.float32), h, 1, obs=False)
    last = impulses(s[0])
    dP = np.linalg.norm(last[0] - first[0]) / np.linalg.norm(first[0])
    dL = np.linalg.norm(last[1] - first[1]) / np.linalg.norm(first[1])
    dE = (last[2] - first[2]) / first[2]
    return dP, dL, dE


def test_free_body_with_payload_keeps_kirchhoff_impulses_to_first_order(payload_envs):
    """Linear and angular impulse of M nu in the inertial frame and the kinetic
    energy are invariants of the continuous law with an off-origin CoG and a
    full inertia tensor; the explicit substep drifts at first order in h."""
    classes, counts, arr = payload_envs
    c = classes[0]
    e = env_dict(arr, 1)
    assert e["cls"] == 0
    e.update(dl=np.zeros(6), dq=np.zeros(6), rb=np.array(e["rg"]), B=e["W"])
    assert np.abs(e["Ig_off"]).max() > 1e-4 and np.abs(e["rg"]).max() > 1e-3
    d1 = _free_drift(e, c, 2e-3)
    d2 = _free_drift(e, c, 1e-3)
    for a, b in zip(d1, d2):
        assert abs(a) < 0.05 and 1.6 < a / b < 2.4


def test_attach_payload_matches_reset_and_zero_payload_is_identity(payload_envs):
    classes, counts, arr = payload_envs
    cls_of = workloads.env_classes(counts)
    envs, _ = oracle.reset(classes, cls_of, vehicles.HOVER, 17)
    pay = np.array([[*np.atleast_1d(draws(17, i, classes[cls_of[i]]["mass"])[0]),
                     *draws(17, i, classes[cls_of[i]]["mass"])[1]] for i in range(len(cls_of))])
    oracle.attach_payload(envs, pay)
    got = oracle.envs_to_arrays(envs)
    for k in ("mass", "Ig", "rg", "W", "Ig_off"):
        np.testing.assert_allclose(got[k], arr[k], rtol=1e-13, atol=1e-15, err_msg=k)
    envs0, _ = oracle.reset(classes, cls_of, vehicles.HOVER, 17)
    before = oracle.envs_to_arrays(envs0)
    oracle.attach_payload(envs0, np.zeros((len(cls_of), 4)))
    after = oracle.envs_to_arrays(envs0)
    for k in ("mass", "Ig", "rg", "W", "Ig_off"):
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)
