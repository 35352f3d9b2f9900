"""FP64 CPU oracle of the MarineGym UUV step (arXiv 2503.09203, Sec. III).

TEST INFRASTRUCTURE ONLY. Imported by the test-suite, by the smoke check and by
the benchmark's CPU-baseline leg; the product package never imports it and it
imports nothing from the product package. Inputs arrive as plain numpy arrays
and dictionaries of numbers (the vehicle-class tables), which this module packs
into its own C records.

The arithmetic lives in ``mg_oracle.cpp`` (FP64, OpenMP over environments);
this wrapper only marshals arrays through ctypes and builds the shared object
with g++ when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmgoracle.so")

STATE_DIM = 21
OBS_DIM = 13
MAX_THR = 8


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, OpenMP, strict IEEE: no fast-math)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class or_class(C.Structure):
    _fields_ = [("n_thr", C.c_int32), ("pad0", C.c_int32), ("mass", C.c_double),
                ("Ig", C.c_double * 3), ("rg", C.c_double * 3), ("rb", C.c_double * 3),
                ("buoy_ratio", C.c_double), ("Ma", C.c_double * 6), ("dl", C.c_double * 6),
                ("dq", C.c_double * 6), ("thr_pos", (C.c_double * 3) * 8),
                ("thr_dir", (C.c_double * 3) * 8), ("k_f", C.c_double * 8),
                ("T_rotor", C.c_double * 8), ("deadzone", C.c_double * 8),
                ("act_kind", C.c_int32 * 8), ("act_link", C.c_int32 * 8),
                ("act_axis", (C.c_double * 3) * 8), ("act_chord", (C.c_double * 3) * 8),
                ("act_range", C.c_double * 8), ("fin_area", C.c_double * 8), ("fin_cl", C.c_double * 8),
                ("fin_cd0", C.c_double * 8), ("fin_cda", C.c_double * 8), ("rho", C.c_double)]

# Actuator kinds (Sec. III-D): propeller, servo, fin, propeller tilted by a servo.
KIND_PROP, KIND_SERVO, KIND_FIN, KIND_TILT = 0, 1, 2, 3


class or_env(C.Structure):
    _fields_ = [("cls", C.c_int32), ("pad0", C.c_int32), ("mass", C.c_double),
                ("Ig", C.c_double * 3), ("rg", C.c_double * 3), ("rb", C.c_double * 3),
                ("W", C.c_double), ("B", C.c_double), ("Ma", C.c_double * 6),
                ("dl", C.c_double * 6), ("dq", C.c_double * 6), ("Vc", C.c_double * 3),
                ("target", C.c_double * 3), ("traj_a", C.c_double * 3), ("traj_w", C.c_double * 3),
                ("traj_phi", C.c_double * 3), ("traj_v", C.c_double * 3), ("k0", C.c_double),
                ("Ig_off", C.c_double * 3)]


class or_reset_cfg(C.Structure):
    _fields_ = [("dr_enabled", C.c_int32), ("current_enabled", C.c_int32),
                ("current_3d", C.c_int32), ("init_mode", C.c_int32),
                ("mass_lo", C.c_double), ("mass_hi", C.c_double),
                ("added_lo", C.c_double), ("added_hi", C.c_double),
                ("damp_lo", C.c_double), ("damp_hi", C.c_double),
                ("cob_lo", C.c_double), ("cob_hi", C.c_double),
                ("cur_lo", C.c_double), ("cur_hi", C.c_double),
                ("target_half", C.c_double), ("pos_radius", C.c_double),
                ("max_angle", C.c_double), ("track", C.c_int32), ("track_kind", C.c_int32),
                ("payload", C.c_int32), ("pad1", C.c_int32), ("payload_lo", C.c_double),
                ("payload_hi", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        _lib.or_rollout.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int, C.c_int,
                                    fp, dp, dp, dp, C.c_int, C.c_int, C.c_int]
        _lib.or_rollout_jvp.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int, C.c_int,
                                        fp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, C.c_int, C.c_int]
        _lib.or_reset.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.c_int64, C.c_void_p,
                                  C.c_uint64, C.POINTER(C.c_int64), C.c_void_p, dp]
        _lib.or_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.or_uniform.restype = C.c_double
        _lib.or_action.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int]
        _lib.or_action.restype = C.c_float
        _lib.or_attach_payload.argtypes = [C.c_void_p, C.c_double, dp]
        _lib.or_attach_payload.restype = None
        for name in ("or_rotation", "or_coriolis", "or_mass", "or_restoring", "or_actuator_wrench",
                     "or_acceleration", "or_philox4x64"):
            getattr(_lib, name).restype = C.c_int
        assert _lib.or_sizeof_class() == C.sizeof(or_class)
        assert _lib.or_sizeof_env() == C.sizeof(or_env)
        assert _lib.or_sizeof_reset_cfg() == C.sizeof(or_reset_cfg)
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


# ---------------------------------------------------------------------------
# Packing of input data (dicts of numbers) into the oracle's own records.
# ---------------------------------------------------------------------------

def pack_class(d: dict) -> or_class:
    c = or_class()
    n = int(d["n_thr"])
    c.n_thr = n
    c.mass = float(d["mass"])
    for i in range(3):
        c.Ig[i] = float(d["Ig"][i]); c.rg[i] = float(d["rg"][i]); c.rb[i] = float(d["rb"][i])
    c.buoy_ratio = float(d["buoy_ratio"])
    for i in range(6):
        c.Ma[i] = float(d["Ma"][i]); c.dl[i] = float(d["dl"][i]); c.dq[i] = float(d["dq"][i])
    for i in range(n):
        for k in range(3):
            c.thr_pos[i][k] = float(d["thr_pos"][i][k]); c.thr_dir[i][k] = float(d["thr_dir"][i][k])
        c.k_f[i] = float(d["k_f"][i]); c.T_rotor[i] = float(d["T_rotor"][i])
        c.deadzone[i] = float(d["deadzone"][i])
        c.act_kind[i] = int(d.get("act_kind", [KIND_PROP] * n)[i])
        c.act_link[i] = int(d.get("act_link", [0] * n)[i])
        for k in range(3):
            c.act_axis[i][k] = float(d.get("act_axis", [(0.0, 0.0, 0.0)] * n)[i][k])
            c.act_chord[i][k] = float(d.get("act_chord", [(0.0, 0.0, 0.0)] * n)[i][k])
        for name in ("act_range", "fin_area", "fin_cl", "fin_cd0", "fin_cda"):
            getattr(c, name)[i] = float(d.get(name, [0.0] * n)[i])
    c.rho = float(d.get("rho", 0.0))
    return c


def pack_classes(classes):
    arr = (or_class * len(classes))()
    for i, d in enumerate(classes):
        arr[i] = pack_class(d)
    return arr


def pack_reset_cfg(d: dict) -> or_reset_cfg:
    r = or_reset_cfg()
    for name, _ in or_reset_cfg._fields_:
        if name in d:
            setattr(r, name, type(getattr(r, name))(d[name]))
    return r


def envs_to_arrays(envs) -> dict:
    """Per-env parameter records -> dict of numpy arrays (for inspection)."""
    n = len(envs)
    out = {k: np.zeros((n,) + s) for k, s in
           (("mass", ()), ("Ig", (3,)), ("rg", (3,)), ("rb", (3,)), ("W", ()), ("B", ()),
            ("Ma", (6,)), ("dl", (6,)), ("dq", (6,)), ("Vc", (3,)), ("target", (3,)),
            ("traj_a", (3,)), ("traj_w", (3,)), ("traj_phi", (3,)), ("traj_v", (3,)), ("k0", ()),
            ("Ig_off", (3,)))}
    out["cls"] = np.zeros(n, dtype=np.int32)
    for i in range(n):
        e = envs[i]
        out["cls"][i] = e.cls
        for k in out:
            if k == "cls":
                continue
            v = getattr(e, k)
            out[k][i] = v if np.ndim(out[k][i]) == 0 else np.array(list(v))
    return out


def make_envs(arrays: dict):
    """dict of numpy arrays (keys as in :func:`envs_to_arrays`) -> env records."""
    n = len(arrays["cls"])
    envs = (or_env * n)()
    for i in range(n):
        e = envs[i]
        e.cls = int(arrays["cls"][i])
        for k in ("mass", "W", "B"):
            setattr(e, k, float(arrays[k][i]))
        if "k0" in arrays:
            e.k0 = float(arrays["k0"][i])
        for k, m in (("Ig", 3), ("rg", 3), ("rb", 3), ("Ma", 6), ("dl", 6), ("dq", 6), ("Vc", 3),
                     ("target", 3), ("traj_a", 3), ("traj_w", 3), ("traj_phi", 3), ("traj_v", 3),
                     ("Ig_off", 3)):
            if k not in arrays:
                continue
            dst = getattr(e, k)
            for j in range(m):
                dst[j] = float(arrays[k][i][j])
    return envs


# ---------------------------------------------------------------------------
# Entry points.
# ---------------------------------------------------------------------------

def reset(classes, env_class, cfg: dict, seed: int, env_ids=None):
    """Sample per-env parameters and initial states. Returns (envs, state[E,21]).

    env_ids: the env index that keys each record's random draws (default
    0..E-1), so that any subset of a large batch can be reproduced."""
    L = lib()
    env_class = np.ascontiguousarray(env_class, dtype=np.int32)
    ids = None if env_ids is None else np.ascontiguousarray(env_ids, dtype=np.int64)
    n = len(env_class)
    envs = (or_env * n)()
    state = np.zeros((n, STATE_DIM))
    cls = pack_classes(classes)
    rc = L.or_reset(C.cast(cls, C.c_void_p), len(classes),
                    env_class.ctypes.data_as(C.POINTER(C.c_int32)), n,
                    C.cast(C.pointer(pack_reset_cfg(cfg)), C.c_void_p), int(seed) & (2**64 - 1),
                    None if ids is None else ids.ctypes.data_as(C.POINTER(C.c_int64)),
                    C.cast(envs, C.c_void_p), _dp(state))
    if rc != 0:
        raise ValueError(f"or_reset failed: {rc}")
    return envs, state


def attach_payload(envs, payload):
    """Attach payloads in place: payload [E, 4] = (m_p, r_p) per env record."""
    L = lib()
    p = np.asarray(payload, dtype=np.float64).reshape(-1, 4)
    assert len(p) == len(envs)
    for i in range(len(envs)):
        rp = np.ascontiguousarray(p[i, 1:4])
        L.or_attach_payload(C.cast(C.byref(envs, i * C.sizeof(or_env)), C.c_void_p), float(p[i, 0]), _dp(rp))
    return envs


def rollout(classes, envs, state, actions, dt, K, obs=True, form=0, threads=0, integ=0):
    """Run actions[T,E,8] (float32) from state[E,21] (FP64, updated in place).

    Returns (state, obs[T,E,13] or None, reward[T,E] or None)."""
    L = lib()
    actions = np.ascontiguousarray(actions, dtype=np.float32)
    T, E = actions.shape[0], actions.shape[1]
    assert actions.shape[2] == MAX_THR and state.shape == (E, STATE_DIM) and state.dtype == np.float64
    assert state.flags.c_contiguous
    o = np.zeros((T, E, OBS_DIM)) if obs else None
    r = np.zeros((T, E)) if obs else None
    cls = pack_classes(classes)
    rc = L.or_rollout(C.cast(cls, C.c_void_p), C.cast(envs, C.c_void_p), E, float(dt), int(K), T,
                      _fp(actions), _dp(state), _dp(o), _dp(r), int(form), int(threads), int(integ))
    if rc != 0:
        raise ValueError(f"or_rollout failed: {rc}")
    return state, o, r


def rollout_jvp(classes, envs, state, actions, dt, K, d_actions=None, d_state0=None, d_Ma=None,
                d_dl=None, d_dq=None, threads=0, integ=0):
    """Directional derivative of a rollout (integ: 0 semi-implicit Euler, 1
    RK4). Returns dict of values and tangents."""
    L = lib()
    actions = np.ascontiguousarray(actions, dtype=np.float32)
    T, E = actions.shape[0], actions.shape[1]
    state = np.ascontiguousarray(state, dtype=np.float64).copy()
    conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    d_actions, d_state0, d_Ma, d_dl, d_dq = map(conv, (d_actions, d_state0, d_Ma, d_dl, d_dq))
    d_state = np.zeros((E, STATE_DIM))
    o = np.zeros((T, E, OBS_DIM)); do = np.zeros_like(o)
    r = np.zeros((T, E)); dr = np.zeros_like(r)
    cls = pack_classes(classes)
    rc = L.or_rollout_jvp(C.cast(cls, C.c_void_p), C.cast(envs, C.c_void_p), E, float(dt), int(K), T,
                          _fp(actions), _dp(d_actions), _dp(state), _dp(d_state0), _dp(d_Ma), _dp(d_dl),
                          _dp(d_dq), _dp(d_state), _dp(o), _dp(do), _dp(r), _dp(dr), int(threads), int(integ))
    if rc != 0:
        raise ValueError(f"or_rollout_jvp failed: {rc}")
    return dict(state=state, d_state=d_state, obs=o, d_obs=do, reward=r, d_reward=dr)


def uniform(seed, stream, env, j) -> float:
    return lib().or_uniform(seed, stream, env, j)


def action(seed, env, step, thr) -> float:
    return lib().or_action(seed, env, step, thr)


def philox4x64(ctr, key):
    L = lib()
    c = (C.c_uint64 * 4)(*ctr)
    k = (C.c_uint64 * 2)(*key)
    o = (C.c_uint64 * 4)()
    L.or_philox4x64(c, k, o)
    return [int(v) for v in o]


def rotation(q):
    R = np.zeros(9)
    lib().or_rotation(_dp(np.ascontiguousarray(q, dtype=np.float64)), _dp(R))
    return R.reshape(3, 3)


def _one_env(env_arrays: dict):
    arr = {k: np.asarray(v)[None] for k, v in env_arrays.items()}
    arr["cls"] = np.array([int(env_arrays.get("cls", 0))], dtype=np.int32)
    return make_envs(arr)


def coriolis(env_arrays: dict, nu):
    envs = _one_env(env_arrays)
    Crb = np.zeros(36); Ca = np.zeros(36)
    lib().or_coriolis(C.cast(envs, C.c_void_p), _dp(np.ascontiguousarray(nu, dtype=np.float64)),
                      _dp(Crb), _dp(Ca))
    return Crb.reshape(6, 6), Ca.reshape(6, 6)


def mass_matrix(env_arrays: dict):
    envs = _one_env(env_arrays)
    M = np.zeros(36)
    lib().or_mass(C.cast(envs, C.c_void_p), _dp(M))
    return M.reshape(6, 6)


def restoring(env_arrays: dict, q):
    envs = _one_env(env_arrays)
    g = np.zeros(6)
    lib().or_restoring(C.cast(envs, C.c_void_p), _dp(np.ascontiguousarray(q, dtype=np.float64)), _dp(g))
    return g


def actuator_wrench(cls: dict, n, nur=None):
    """Wrench of actuator states n; nur = body velocity relative to the water (fins)."""
    c = pack_class(cls)
    nn = np.zeros(8)
    nn[:len(n)] = n
    tau = np.zeros(6)
    v = None if nur is None else np.ascontiguousarray(nur, dtype=np.float64)
    lib().or_actuator_wrench(C.byref(c), _dp(nn), _dp(v), _dp(tau))
    return tau


def acceleration(env_arrays: dict, s, tau, form=0):
    envs = _one_env(env_arrays)
    out = np.zeros(6)
    lib().or_acceleration(C.cast(envs, C.c_void_p), _dp(np.ascontiguousarray(s, dtype=np.float64)),
                          _dp(np.ascontiguousarray(tau, dtype=np.float64)), int(form), _dp(out))
    return out
