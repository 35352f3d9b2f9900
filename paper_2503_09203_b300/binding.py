"""Thin ctypes binding of libmarinegym (include/marinegym.h).

Functions keep the C names (``mg_create``, ``mg_step`` ...) and only marshal
arguments: torch tensors become raw device pointers, streams become their
CUDA handles, and non-zero return codes raise :class:`MGError` with the
library's message. Every step of the path runs in the library's kernels;
there is no Python or CPU fallback, and loading fails loudly when the library
has not been built.

:class:`Sim` is a convenience owner of one simulator handle and the torch
buffers that match its layout (per-class action views, observation and reward
buffers).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MG_LIB_PATH") or os.path.join(_HERE, "libmarinegym.so")

MG_OK = 0
MG_ERR_INVALID_ARG = -1
MG_ERR_OOM = -2
MG_ERR_CUDA = -3
MG_ERR_NONFINITE = -4
MG_ERR_TIMEOUT = -5
MG_ERR_ADMISSION_REFUSED = -6
MG_ERR_STATE = -7
MG_MAX_THR = 8
MG_ACT_PROP, MG_ACT_SERVO, MG_ACT_FIN, MG_ACT_TILT = 0, 1, 2, 3   # actuator kinds
MG_INTEG_EULER, MG_INTEG_RK4 = 0, 1
MG_MAX_CLASSES = 16
MG_STATE_DIM = 21
MG_OBS_DIM = 13
MG_ENV_PARAM_DIM = 34
MG_REQ_PENDING, MG_REQ_RUNNING, MG_REQ_DONE, MG_REQ_UNKNOWN = 0, 1, 2, -1


class MGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class mg_class_desc(C.Structure):
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


class mg_reset_cfg(C.Structure):
    _fields_ = [("dr_enabled", C.c_int32), ("current_enabled", C.c_int32),
                ("current_3d", C.c_int32), ("init_mode", C.c_int32),
                ("mass_lo", C.c_double), ("mass_hi", C.c_double),
                ("added_lo", C.c_double), ("added_hi", C.c_double),
                ("damp_lo", C.c_double), ("damp_hi", C.c_double),
                ("cob_lo", C.c_double), ("cob_hi", C.c_double),
                ("cur_lo", C.c_double), ("cur_hi", C.c_double),
                ("target_half", C.c_double), ("pos_radius", C.c_double),
                ("max_angle", C.c_double), ("track_kind", C.c_int32), ("pad0", C.c_int32),
                ("payload_lo", C.c_double), ("payload_hi", C.c_double)]


class mg_config(C.Structure):
    _fields_ = [("n_classes", C.c_int32), ("class_counts", C.POINTER(C.c_int32)),
                ("dt", C.c_double), ("K", C.c_int32), ("per_env_params", C.c_int32),
                ("reset", mg_reset_cfg), ("record_steps", C.c_int32), ("ckpt_every", C.c_int32),
                ("mem_budget", C.c_size_t), ("task", C.c_int32), ("payload", C.c_int32),
                ("integrator", C.c_int32), ("pad1", C.c_int32)]


class mg_class_layout(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("n_thr", C.c_int32), ("env_offset", C.c_int32),
                ("slot_offset", C.c_int32), ("state_offset", C.c_int64), ("state_stride", C.c_int32),
                ("pad0", C.c_int32), ("action_offset", C.c_int64)]


class mg_layout(C.Structure):
    _fields_ = [("n_classes", C.c_int32), ("n_envs", C.c_int32), ("n_slots", C.c_int32),
                ("launches_per_step", C.c_int32), ("action_floats", C.c_int64), ("state_floats", C.c_int64),
                ("cls", mg_class_layout * MG_MAX_CLASSES)]


class mg_launch_shape(C.Structure):
    _fields_ = [("lanes_per_env", C.c_int32), ("envs_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("specialised", C.c_int32), ("us_per_step", C.c_double), ("specialised_launches", C.c_int32),
                ("pad0", C.c_int32)]


class mg_server_config(C.Structure):
    _fields_ = [("dt", C.c_double), ("budget_bytes", C.c_size_t), ("max_requests", C.c_int32),
                ("max_queue", C.c_int32), ("reset", mg_reset_cfg), ("integrator", C.c_int32),
                ("pad0", C.c_int32)]


class mg_request(C.Structure):
    _fields_ = [("cls", C.c_int32), ("n_envs", C.c_int32), ("horizon", C.c_int32), ("K", C.c_int32),
                ("seed", C.c_uint64)]


class mg_request_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_envs", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("steps_done", C.c_int64),
                ("final_state", C.POINTER(C.c_float)), ("returns", C.POINTER(C.c_float))]


class mg_server_stats(C.Structure):
    _fields_ = [("requests_done", C.c_int64), ("env_steps", C.c_int64), ("ticks", C.c_int64),
                ("busy_seconds", C.c_double), ("step_latency_p50", C.c_double),
                ("step_latency_p99", C.c_double), ("queue_delay_p50", C.c_double),
                ("queue_delay_p99", C.c_double), ("tick_p50", C.c_double), ("tick_p99", C.c_double),
                ("budget_bytes", C.c_size_t), ("peak_resident_bytes", C.c_size_t), ("peak_requests", C.c_int32),
                ("pad0", C.c_int32)]


_VP, _I32, _I64, _U64, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
_SIGS = {
    "mg_create": [C.POINTER(mg_config), C.POINTER(mg_class_desc), C.POINTER(_VP)],
    "mg_destroy": [_VP],
    "mg_get_layout": [_VP, C.POINTER(mg_layout)],
    "mg_reset": [_VP, _VP, _I32, _U64, _VP],
    "mg_step": [_VP, _VP, _I32, _VP, _VP, _VP],
    "mg_rollout": [_VP, _VP, _I32, _VP, _VP, _I32, _VP],
    "mg_observe": [_VP, _VP, _VP, _VP],
    "mg_recording": [_VP, C.POINTER(_I32), C.POINTER(_U64)],
    "mg_env_order": [_VP, _I32, _I32, _VP, _VP],
    "mg_step_host": [_VP, _VP, _I32, _VP, _VP, _VP],
    "mg_step_backward": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "mg_step_backward_noalloc": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "mg_set_hydro": [_VP, _VP, _VP, _VP, _VP],
    "mg_rollout_fp64": [_VP, _VP, _I32, _VP, _VP, _VP, _D, _VP, _VP, _VP],
    "mg_get_state": [_VP, _VP, C.c_size_t],
    "mg_set_state": [_VP, _VP, C.c_size_t],
    "mg_get_params": [_VP, _VP, C.c_size_t],
    "mg_get_task": [_VP, _VP, C.c_size_t],
    "mg_set_task": [_VP, _VP, C.c_size_t],
    "mg_get_payload": [_VP, _VP, C.c_size_t],
    "mg_set_payload": [_VP, _VP, C.c_size_t],
    "mg_set_params": [_VP, _VP, C.c_size_t],
    "mg_status": [_VP, _VP],
    "mg_test_wait_timeout": [_VP, _U64, _VP],
    "mg_autotune": [_VP, _I32, _VP, C.POINTER(mg_launch_shape)],
    "mg_get_launch_shape": [_VP, C.POINTER(mg_launch_shape)],
    "mg_set_launch_shape": [_VP, C.POINTER(mg_launch_shape)],
    "mg_set_blocks_per_sm": [_VP, _I32],
    "mg_graph_capture": [_VP, _VP, _I32, _VP, _VP, _VP, C.POINTER(_VP)],
    "mg_graph_launch": [_VP, _VP],
    "mg_graph_destroy": [_VP],
    "mg_count_flops": [_I32, _I32, C.POINTER(_D), C.POINTER(_D), C.POINTER(_D)],
    "mg_server_create": [C.POINTER(mg_server_config), C.POINTER(mg_class_desc), _I32, C.POINTER(_VP)],
    "mg_server_submit": [_VP, C.POINTER(mg_request), C.POINTER(_I64)],
    "mg_server_poll": [_VP, _I64, C.POINTER(mg_request_result)],
    "mg_server_release": [_VP, _I64],
    "mg_server_wait_idle": [_VP, _D],
    "mg_server_stats_get": [_VP, C.POINTER(mg_server_stats)],
    "mg_server_destroy": [_VP],
}

_lib = None


def lib() -> C.CDLL:
    """Load libmarinegym.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmarinegym.so is not built ({LIB_PATH}); run "
                               "`python -m paper_2503_09203_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, argt in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = argt
            f.restype = C.c_int
        for name in ("mg_last_error", "mg_strerror", "mg_server_last_error"):
            getattr(L, name).restype = C.c_char_p
        L.mg_last_error.argtypes = [_VP]
        L.mg_strerror.argtypes = [C.c_int]
        L.mg_server_last_error.argtypes = [_VP]
        _lib = L
    return _lib


def _check(rc: int, handle=None, server=False):
    if rc != MG_OK:
        L = lib()
        msg = (L.mg_server_last_error(handle) if server else L.mg_last_error(handle)) or b""
        raise MGError(rc, msg.decode() or L.mg_strerror(rc).decode())
    return rc


def _ptr(t) -> Optional[int]:
    """Device (or host) pointer of a tensor / array, or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# Packing of the vehicle tables into the library's records.
# ---------------------------------------------------------------------------

def pack_class(d: dict) -> mg_class_desc:
    c = mg_class_desc()
    n = int(d["n_thr"])
    c.n_thr = n
    c.mass = float(d["mass"])
    for i in range(3):
        c.Ig[i] = float(d["Ig"][i]); c.rg[i] = float(d["rg"][i]); c.rb[i] = float(d["rb"][i])
    c.buoy_ratio = float(d["buoy_ratio"])
    for i in range(6):
        c.Ma[i] = float(d["Ma"][i]); c.dl[i] = float(d["dl"][i]); c.dq[i] = float(d["dq"][i])
    # n_thr is passed through unchecked (the library validates it); at most 8
    # thrusters are copied.
    for i in range(min(n, MG_MAX_THR, len(d["thr_pos"]))):
        for k in range(3):
            c.thr_pos[i][k] = float(d["thr_pos"][i][k]); c.thr_dir[i][k] = float(d["thr_dir"][i][k])
        c.k_f[i] = float(d["k_f"][i]); c.T_rotor[i] = float(d["T_rotor"][i]); c.deadzone[i] = float(d["deadzone"][i])
        # Actuator kinds (absent: every channel a fixed propeller).
        c.act_kind[i] = int(d.get("act_kind", [MG_ACT_PROP] * n)[i])
        c.act_link[i] = int(d.get("act_link", [0] * n)[i])
        for k in range(3):
            c.act_axis[i][k] = float(d.get("act_axis", [(0.0, 0.0, 0.0)] * n)[i][k])
            c.act_chord[i][k] = float(d.get("act_chord", [(0.0, 0.0, 0.0)] * n)[i][k])
        for name in ("act_range", "fin_area", "fin_cl", "fin_cd0", "fin_cda"):
            getattr(c, name)[i] = float(d.get(name, [0.0] * n)[i])
    c.rho = float(d.get("rho", 0.0))
    return c


def pack_reset(d: dict) -> mg_reset_cfg:
    r = mg_reset_cfg()
    for name, _ in mg_reset_cfg._fields_:
        if name in d:
            setattr(r, name, type(getattr(r, name))(d[name]))
    return r


# ---------------------------------------------------------------------------
# C entry points with the same names.
# ---------------------------------------------------------------------------

TASK_HOVER, TASK_TRACK = 0, 1


def mg_create(classes: Sequence[dict], counts: Sequence[int], dt: float, K: int, per_env_params: bool = True,
              reset: Optional[dict] = None, record_steps: int = 0, ckpt_every: int = 0, mem_budget: int = 0,
              task: int = TASK_HOVER, payload: bool = False, integrator: int = MG_INTEG_EULER):
    L = lib()
    arr = (mg_class_desc * len(classes))(*[pack_class(c) for c in classes])
    cnt = (C.c_int32 * len(counts))(*[int(x) for x in counts])
    cfg = mg_config(n_classes=len(classes), class_counts=cnt, dt=float(dt), K=int(K),
                    per_env_params=int(bool(per_env_params)), reset=pack_reset(reset or {}),
                    record_steps=int(record_steps), ckpt_every=int(ckpt_every), mem_budget=int(mem_budget),
                    task=int(task), payload=int(bool(payload)), integrator=int(integrator))
    h = _VP()
    _check(L.mg_create(C.byref(cfg), arr, C.byref(h)), None)
    return h.value


def mg_destroy(sim):
    return _check(lib().mg_destroy(sim), sim)


def mg_get_layout(sim) -> mg_layout:
    lay = mg_layout()
    _check(lib().mg_get_layout(sim, C.byref(lay)), sim)
    return lay


def mg_reset(sim, env_ids=None, n: int = 0, seed: int = 0, stream=None):
    return _check(lib().mg_reset(sim, _ptr(env_ids), int(n), int(seed) & (2 ** 64 - 1), _stream(stream)), sim)


def mg_step(sim, actions, n_steps: int = 1, obs=None, reward=None, stream=None):
    return _check(lib().mg_step(sim, _ptr(actions), int(n_steps), _ptr(obs), _ptr(reward), _stream(stream)), sim)


def mg_rollout(sim, actions, n_steps: int, obs=None, reward=None, record: bool = False, stream=None):
    return _check(lib().mg_rollout(sim, _ptr(actions), int(n_steps), _ptr(obs), _ptr(reward), int(bool(record)),
                                   _stream(stream)), sim)


def mg_observe(sim, obs=None, reward=None, stream=None):
    return _check(lib().mg_observe(sim, _ptr(obs), _ptr(reward), _stream(stream)), sim)


def mg_recording(sim):
    """(steps, id) of the simulator's current recording ((0, 0): none)."""
    n, i = _I32(), _U64()
    _check(lib().mg_recording(sim, C.byref(n), C.byref(i)), sim)
    return n.value, i.value


def mg_env_order(env_class, n_classes: int):
    """Library order of an env -> class map: (class_counts [n_classes],
    lib_env [n_envs]) with lib_env[i] the library env index of env i."""
    ec = np.ascontiguousarray(env_class, dtype=np.int32)
    counts = np.zeros(int(n_classes), np.int32)
    lib_env = np.zeros(len(ec), np.int32)
    _check(lib().mg_env_order(ec.ctypes.data, len(ec), int(n_classes), counts.ctypes.data, lib_env.ctypes.data))
    return counts, lib_env


def mg_step_host(sim, actions_host, n_steps: int = 1, obs_host=None, reward_host=None, stream=None):
    return _check(lib().mg_step_host(sim, _ptr(actions_host), int(n_steps), _ptr(obs_host), _ptr(reward_host),
                                     _stream(stream)), sim)


def mg_step_backward(sim, actions, g_obs=None, g_rew=None, g_state_T=None, g_actions=None, g_added_mass=None,
                     g_damping=None, g_state0=None, stream=None):
    return _check(lib().mg_step_backward(sim, _ptr(actions), _ptr(g_obs), _ptr(g_rew), _ptr(g_state_T),
                                         _ptr(g_actions), _ptr(g_added_mass), _ptr(g_damping), _ptr(g_state0),
                                         _stream(stream)), sim)


def mg_step_backward_noalloc(sim, actions, g_obs=None, g_rew=None, g_state_T=None, g_actions=None,
                             g_added_mass=None, g_damping=None, g_state0=None, stream=None):
    """mg_step_backward without any device allocation: for callers that cannot
    allocate device memory during the backward pass (see the header)."""
    return _check(lib().mg_step_backward_noalloc(sim, _ptr(actions), _ptr(g_obs), _ptr(g_rew), _ptr(g_state_T),
                                                 _ptr(g_actions), _ptr(g_added_mass), _ptr(g_damping),
                                                 _ptr(g_state0), _stream(stream)), sim)


def mg_set_hydro(sim, A=None, dl=None, dq=None, stream=None):
    return _check(lib().mg_set_hydro(sim, _ptr(A), _ptr(dl), _ptr(dq), _stream(stream)), sim)


def mg_rollout_fp64(sim, actions, n_steps, dA=None, ddl=None, ddq=None, eps=0.0, reward=None, state=None,
                    stream=None):
    return _check(lib().mg_rollout_fp64(sim, _ptr(actions), int(n_steps), _ptr(dA), _ptr(ddl), _ptr(ddq),
                                        float(eps), _ptr(reward), _ptr(state), _stream(stream)), sim)


def mg_get_state(sim, n_envs: int) -> np.ndarray:
    out = np.zeros((n_envs, MG_STATE_DIM), np.float32)
    _check(lib().mg_get_state(sim, out.ctypes.data, out.nbytes), sim)
    return out


def mg_set_state(sim, state: np.ndarray):
    s = np.ascontiguousarray(state, dtype=np.float32)
    return _check(lib().mg_set_state(sim, s.ctypes.data, s.nbytes), sim)


def mg_get_params(sim, n_envs: int) -> np.ndarray:
    out = np.zeros((n_envs, MG_ENV_PARAM_DIM), np.float64)
    _check(lib().mg_get_params(sim, out.ctypes.data, out.nbytes), sim)
    return out


def mg_set_params(sim, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float64)
    return _check(lib().mg_set_params(sim, p.ctypes.data, p.nbytes), sim)


TASK_DIM = 16   # c[3], a[3], w[3], phi[3], v[3], step counter


def mg_get_task(sim, n_envs: int) -> np.ndarray:
    out = np.zeros((n_envs, TASK_DIM), np.float64)
    _check(lib().mg_get_task(sim, out.ctypes.data, out.nbytes), sim)
    return out


def mg_set_task(sim, task: np.ndarray):
    t = np.ascontiguousarray(task, dtype=np.float64)
    return _check(lib().mg_set_task(sim, t.ctypes.data, t.nbytes), sim)


PAYLOAD_DIM = 4   # m_p, r_p (x, y, z)


def mg_get_payload(sim, n_envs: int) -> np.ndarray:
    out = np.zeros((n_envs, PAYLOAD_DIM), np.float64)
    _check(lib().mg_get_payload(sim, out.ctypes.data, out.nbytes), sim)
    return out


def mg_set_payload(sim, payload: np.ndarray):
    p = np.ascontiguousarray(payload, dtype=np.float64)
    return _check(lib().mg_set_payload(sim, p.ctypes.data, p.nbytes), sim)


def mg_status(sim, stream=None):
    return _check(lib().mg_status(sim, _stream(stream)), sim)


def mg_test_wait_timeout(sim, limit_ns: int, stream=None):
    return _check(lib().mg_test_wait_timeout(sim, int(limit_ns), _stream(stream)), sim)


def _shape_dict(sh: "mg_launch_shape") -> dict:
    return {name: getattr(sh, name) for name, _ in mg_launch_shape._fields_ if name != "pad0"}


def mg_autotune(sim, n_steps: int = 0, stream=None) -> dict:
    """Time the launch-shape candidates on a rollout of n_steps steps (0: 20)
    and keep the fastest; returns the chosen shape."""
    sh = mg_launch_shape()
    _check(lib().mg_autotune(sim, int(n_steps), _stream(stream), C.byref(sh)), sim)
    return _shape_dict(sh)


def mg_get_launch_shape(sim) -> dict:
    sh = mg_launch_shape()
    _check(lib().mg_get_launch_shape(sim, C.byref(sh)), sim)
    return _shape_dict(sh)


def mg_set_launch_shape(sim, lanes_per_env: int = 1, blocks_per_sm: int = 0, specialised: int = 1):
    sh = mg_launch_shape(lanes_per_env=int(lanes_per_env), blocks_per_sm=int(blocks_per_sm),
                         specialised=int(specialised))
    return _check(lib().mg_set_launch_shape(sim, C.byref(sh)), sim)


def mg_set_blocks_per_sm(sim, blocks_per_sm: int):
    return _check(lib().mg_set_blocks_per_sm(sim, int(blocks_per_sm)), sim)


def mg_graph_capture(sim, actions, n_steps, obs=None, reward=None, stream=None):
    g = _VP()
    _check(lib().mg_graph_capture(sim, _ptr(actions), int(n_steps), _ptr(obs), _ptr(reward), _stream(stream),
                                  C.byref(g)), sim)
    return g.value


def mg_graph_launch(graph, stream=None):
    return _check(lib().mg_graph_launch(graph, _stream(stream)))


def mg_graph_destroy(graph):
    return _check(lib().mg_graph_destroy(graph))


def mg_count_flops(n_thr: int, adjoint: bool = False, with_current: bool = True):
    """(substep, observe) FP32 op counts, plus the substep adjoint's if asked.
    with_current=False: the class-constant variant (no current terms)."""
    s, o, a = C.c_double(), C.c_double(), C.c_double()
    _check(lib().mg_count_flops(int(n_thr), int(bool(with_current)), C.byref(s), C.byref(o), C.byref(a)))
    return (s.value, o.value, a.value) if adjoint else (s.value, o.value)


# Canonical per-env parameter record (MG_ENV_PARAM_DIM doubles).
PARAM_FIELDS = (("mass", 0, 1), ("Ig", 1, 3), ("rb", 4, 3), ("W", 7, 1), ("B", 8, 1), ("Ma", 9, 6),
                ("dl", 15, 6), ("dq", 21, 6), ("Vc", 27, 3), ("target", 30, 3))


def params_to_dict(p: np.ndarray) -> dict:
    return {k: (p[:, o] if n == 1 else p[:, o:o + n]) for k, o, n in PARAM_FIELDS}


def dict_to_params(d: dict, n_envs: int) -> np.ndarray:
    p = np.zeros((n_envs, MG_ENV_PARAM_DIM))
    for k, o, n in PARAM_FIELDS:
        v = np.asarray(d[k], dtype=np.float64)
        if n == 1:
            p[:, o] = v.reshape(n_envs)
        else:
            p[:, o:o + n] = v.reshape(n_envs, n)
    return p


# ---------------------------------------------------------------------------
# Convenience owner of one simulator and its torch buffers.
# ---------------------------------------------------------------------------

class Sim:
    """One simulator on the current CUDA device.

    ``actions`` is a flat device buffer laid out per class (see
    :meth:`class_actions`); ``obs`` [n_slots, 13] and ``reward`` [n_slots]
    receive the hover observation and reward.
    """

    def __init__(self, classes, counts, dt=0.01, K=1, per_env_params=True, reset=None, record_steps=0,
                 ckpt_every=0, mem_budget=0, task=TASK_HOVER, payload=False, integrator=MG_INTEG_EULER,
                 device="cuda"):
        import torch
        self.classes = list(classes)
        self.counts = [int(c) for c in counts]
        self.dt, self.K = float(dt), int(K)
        self.handle = mg_create(self.classes, self.counts, dt, K, per_env_params, reset, record_steps,
                                ckpt_every, mem_budget, task, payload, integrator)
        self.layout = mg_get_layout(self.handle)
        self.n_envs = self.layout.n_envs
        self.n_slots = self.layout.n_slots
        self.action_floats = self.layout.action_floats
        self.device = torch.device(device)
        self.obs = torch.zeros(self.n_slots, MG_OBS_DIM, device=self.device)
        self.reward = torch.zeros(self.n_slots, device=self.device)

    # -- layout helpers ------------------------------------------------------
    def launches_per_step(self) -> int:
        """Kernel launches one step call makes (current launch plan)."""
        return int(mg_get_layout(self.handle).launches_per_step)

    def cls(self, c):
        return self.layout.cls[c]

    def slots_of_envs(self) -> np.ndarray:
        """Slot index of every env (env order)."""
        out = np.zeros(self.n_envs, np.int64)
        for c in range(self.layout.n_classes):
            L = self.layout.cls[c]
            out[L.env_offset:L.env_offset + L.n_envs] = L.slot_offset + np.arange(L.n_envs)
        return out

    def new_actions(self, n_steps=1):
        import torch
        return torch.zeros(n_steps, self.action_floats, device=self.device)

    def class_actions(self, actions, c, step=0):
        """[n_envs_c, n_thr_c] view of class c's actions inside a flat buffer."""
        L = self.layout.cls[c]
        flat = actions.view(-1, self.action_floats)[step]
        return flat[L.action_offset:L.action_offset + L.n_envs * L.n_thr].view(L.n_envs, L.n_thr)

    def pack_actions(self, a_env8):
        """[T, n_envs, 8] (numpy or torch, env order, padded to 8) -> flat device buffer."""
        import torch
        a = torch.as_tensor(np.asarray(a_env8, dtype=np.float32))
        T = a.shape[0]
        out = torch.zeros(T, self.action_floats)
        for c in range(self.layout.n_classes):
            L = self.layout.cls[c]
            if L.n_envs == 0:
                continue
            blk = a[:, L.env_offset:L.env_offset + L.n_envs, :L.n_thr].reshape(T, -1)
            out[:, L.action_offset:L.action_offset + L.n_envs * L.n_thr] = blk
        return out.to(self.device)

    def unpack_actions(self, flat):
        """Flat [T, action_floats] -> [T, n_envs, 8] numpy (env order)."""
        f = flat.detach().cpu().numpy().reshape(-1, self.action_floats)
        T = f.shape[0]
        out = np.zeros((T, self.n_envs, MG_MAX_THR), f.dtype)
        for c in range(self.layout.n_classes):
            L = self.layout.cls[c]
            if L.n_envs == 0:
                continue
            blk = f[:, L.action_offset:L.action_offset + L.n_envs * L.n_thr].reshape(T, L.n_envs, L.n_thr)
            out[:, L.env_offset:L.env_offset + L.n_envs, :L.n_thr] = blk
        return out

    # -- calls -----------------------------------------------------------------
    def reset(self, seed=0, env_ids=None, stream=None):
        n = 0 if env_ids is None else int(env_ids.numel())
        mg_reset(self.handle, env_ids, n, seed, stream)

    def step(self, actions, n_steps=1, obs=True, stream=None):
        mg_step(self.handle, actions, n_steps, self.obs if obs else None, self.reward if obs else None, stream)

    def rollout(self, actions, n_steps, obs=None, reward=None, record=False, stream=None):
        mg_rollout(self.handle, actions, n_steps, obs, reward, record, stream)

    def observe(self, stream=None):
        mg_observe(self.handle, self.obs, self.reward, stream)
        return self.obs

    def get_state(self):
        return mg_get_state(self.handle, self.n_envs)

    def set_state(self, s):
        mg_set_state(self.handle, s)

    def get_params(self):
        return mg_get_params(self.handle, self.n_envs)

    def set_params(self, p):
        mg_set_params(self.handle, p)

    def get_task(self):
        return mg_get_task(self.handle, self.n_envs)

    def set_task(self, t):
        mg_set_task(self.handle, t)

    def get_payload(self):
        return mg_get_payload(self.handle, self.n_envs)

    def set_payload(self, p):
        mg_set_payload(self.handle, p)

    def status(self, stream=None):
        return mg_status(self.handle, stream)

    def close(self):
        if self.handle:
            mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Serving loop.
# ---------------------------------------------------------------------------

def mg_server_create(classes, dt: float, budget_bytes: int = 0, max_requests: int = 1024, max_queue: int = 100000,
                     reset: Optional[dict] = None, integrator: int = MG_INTEG_EULER):
    L = lib()
    arr = (mg_class_desc * len(classes))(*[pack_class(c) for c in classes])
    cfg = mg_server_config(dt=float(dt), budget_bytes=int(budget_bytes), max_requests=int(max_requests),
                           max_queue=int(max_queue), reset=pack_reset(reset or {}), integrator=int(integrator))
    h = _VP()
    rc = L.mg_server_create(C.byref(cfg), arr, len(classes), C.byref(h))
    if rc != MG_OK:
        raise MGError(rc, L.mg_strerror(rc).decode())
    return h.value


def mg_server_submit(srv, cls: int, n_envs: int, horizon: int, K: int, seed: int) -> int:
    req = mg_request(cls=int(cls), n_envs=int(n_envs), horizon=int(horizon), K=int(K), seed=int(seed) & (2 ** 64 - 1))
    rid = _I64()
    _check(lib().mg_server_submit(srv, C.byref(req), C.byref(rid)), srv, server=True)
    return rid.value


def mg_server_poll(srv, rid: int) -> dict:
    r = mg_request_result()
    _check(lib().mg_server_poll(srv, int(rid), C.byref(r)), srv, server=True)
    out = dict(status=r.status, n_envs=r.n_envs, t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done,
               steps_done=r.steps_done)
    if r.status == MG_REQ_DONE:
        n = r.n_envs
        out["final_state"] = np.ctypeslib.as_array(r.final_state, shape=(n * MG_STATE_DIM,)).reshape(n, MG_STATE_DIM).copy()
        out["returns"] = np.ctypeslib.as_array(r.returns, shape=(n,)).copy()
    return out


def mg_server_release(srv, rid: int):
    return _check(lib().mg_server_release(srv, int(rid)), srv, server=True)


def mg_server_wait_idle(srv, timeout_s: float = 60.0):
    return _check(lib().mg_server_wait_idle(srv, float(timeout_s)), srv, server=True)


def mg_server_stats_get(srv) -> dict:
    st = mg_server_stats()
    _check(lib().mg_server_stats_get(srv, C.byref(st)), srv, server=True)
    return {name: getattr(st, name) for name, _ in mg_server_stats._fields_}


def mg_server_destroy(srv):
    return _check(lib().mg_server_destroy(srv), srv, server=True)
