"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/marinegym.h declares, its record layouts match the binding's, and the
host-only paths (argument validation, FLOP count) behave. No compute calls."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2503_09203_b300 import binding as B
from paper_2503_09203_b300 import build as mgbuild
from paper_2503_09203_b300 import vehicles

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "marinegym.h")


@pytest.fixture(scope="module")
def lib():
    mgbuild.build()
    return B.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(mg_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 30
    out = subprocess.check_output(["nm", "-D", "--defined-only", B.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT\s+(mg_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_binding_covers_header(lib):
    names = set(declared_functions())
    bound = set(B._SIGS) | {"mg_last_error", "mg_strerror", "mg_server_last_error"}
    assert names == bound


def test_record_layouts_match_header(tmp_path):
    structs = ["mg_class_desc", "mg_reset_cfg", "mg_config", "mg_class_layout", "mg_layout",
               "mg_server_config", "mg_request", "mg_request_result", "mg_server_stats", "mg_launch_shape"]
    prog = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){"]
    for s in structs:
        prog.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(B, s)._fields_:
            prog.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    prog.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", str(c), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    for line in out:
        if not line:
            continue
        key, val = line.split()
        if "." in key:
            s, f = key.split(".")
            assert getattr(getattr(B, s), f).offset == int(val), key
        else:
            assert C.sizeof(getattr(B, key)) == int(val), key


def test_flop_count_is_host_only_and_sane(lib):
    s8, o8 = B.mg_count_flops(8)
    s4, o4 = B.mg_count_flops(4)
    assert 300 <= s8 <= 500 and s4 < s8 and 60 <= o8 <= 120
    with pytest.raises(B.MGError) as e:
        B.mg_count_flops(9)
    assert e.value.code == B.MG_ERR_INVALID_ARG


@pytest.mark.parametrize("nt", range(1, 9))
def test_flop_count_equals_hand_count(lib, nt):
    """mg_count_flops against a count by hand of the substep and observation
    as the kernels write them (add, sub, mul = 1, a fused multiply-add 2,
    reciprocal square root 1; compare, abs, negate 0):
    rotor lag 3 and thrust k n|n| 2 per thruster, allocation 6 (2 NT - 1);
    R(q) from doubled components 27; body right-hand side 100 (I w 3, a1 / m v
    + a1 / A_a w + I w 15, three cross products 27, damping 18, W - B 1, B r_b 3,
    (B r_b) x e 9, linear rows 12, angular rows 12); velocity update
    (h minv_j) rhs_j 18; position 21; attitude 41 (h/2 1, quaternion rate 20,
    q + h/2 qdot 8, norm and reciprocal square root 8, scaling 4). The ocean
    current adds R^T V_c and v - v_c (18), w x v_c (9) and A_l o (w x v_c) in
    the linear rows (6). Observation: R(q) 27, p - p* 3, R^T d 15, sign 4,
    |d|^2 5, |nu|^2 11, |c|^2 2 NT - 1, reward 4."""
    sub_plain = 5 * nt + 6 * (2 * nt - 1) + 27 + 100 + 18 + 21 + 41
    s0, o0 = B.mg_count_flops(nt, with_current=False)
    s1, o1 = B.mg_count_flops(nt, with_current=True)
    assert s0 == sub_plain == 17 * nt + 201
    assert s1 == sub_plain + 18 + 9 + 6
    assert o0 == o1 == 27 + 3 + 15 + 4 + 5 + 11 + (2 * nt - 1) + 4


@pytest.mark.parametrize("bad", ["dt", "K", "n_thr", "rg", "counts", "per_env", "payload_per_env",
                                 "ckpt_every", "payload_range"])
def test_create_rejects_bad_arguments_before_touching_the_device(lib, bad):
    classes = [vehicles.heavy8()]
    counts, dt, K, per_env, reset = [8], 0.01, 1, True, dict(vehicles.NO_DR)
    record, payload, ckpt = 0, False, 0
    if bad == "dt":
        dt = -1.0
    elif bad == "K":
        K = 0
    elif bad == "n_thr":
        classes = [dict(vehicles.heavy8(), n_thr=9)]
    elif bad == "rg":
        classes = [dict(vehicles.heavy8(), rg=(0.0, 0.0, 0.01))]
    elif bad == "counts":
        counts = [-1]
    elif bad == "per_env":
        per_env, reset = False, dict(vehicles.DR_TRAIN)
    elif bad == "payload_per_env":
        per_env, payload = False, True
    elif bad == "ckpt_every":
        record, ckpt = 10, -1
    elif bad == "payload_range":
        payload, reset = True, dict(vehicles.PAYLOAD, payload_lo=0.3, payload_hi=0.1)
    with pytest.raises(B.MGError) as e:
        B.mg_create(classes, counts, dt, K, per_env, reset, record_steps=record, ckpt_every=ckpt, payload=payload)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    if bad.startswith("payload"):
        assert "payload" in str(e.value)


def test_error_strings(lib):
    for code in (B.MG_OK, B.MG_ERR_INVALID_ARG, B.MG_ERR_OOM, B.MG_ERR_NONFINITE, B.MG_ERR_STATE):
        assert lib.mg_strerror(code)


@pytest.mark.parametrize("bad", ["integrator", "fin_chord", "tilt_link", "kind", "fin_rho"])
def test_create_rejects_bad_actuators_before_touching_the_device(lib, bad):
    classes = [vehicles.lauv(), vehicles.tilt_hauv()]
    counts, record, integ = [4, 4], 0, B.MG_INTEG_EULER
    if bad == "integrator":
        integ = 7
    elif bad == "fin_chord":
        classes[0]["act_chord"] = [(0.0, 0.0, 0.0)] + [(0.0, 0.6, 0.8)] * 4   # not normal to the y/z span axes
    elif bad == "tilt_link":
        classes[1]["act_link"] = [0, 5, 6, 7, 0, 0, 0, 0]                    # a propeller, not a servo
    elif bad == "kind":
        classes[1]["act_kind"] = [3, 3, 3, 3, 1, 1, 1, 9]
    elif bad == "fin_rho":
        classes[0]["rho"] = 0.0
    with pytest.raises(B.MGError) as e:
        B.mg_create(classes, counts, 0.01, 1, True, dict(vehicles.HOVER), record_steps=record, integrator=integ)
    assert e.value.code == B.MG_ERR_INVALID_ARG


def test_server_refuses_bad_classes_before_touching_the_device(lib):
    """Generic classes are served; a class whose CoG is off the origin (only a
    payload moves it) is refused before any device work."""
    with pytest.raises(B.MGError) as e:
        B.mg_server_create([vehicles.lauv(), dict(vehicles.heavy8(), rg=(0.0, 0.0, 0.01))], dt=0.01,
                           max_requests=4, max_queue=4)
    assert e.value.code == B.MG_ERR_INVALID_ARG
    with pytest.raises(B.MGError) as e:
        B.mg_server_create([vehicles.lauv(), vehicles.heavy8()], dt=0.01, max_requests=4, max_queue=4, integrator=3)
    assert e.value.code == B.MG_ERR_INVALID_ARG



def test_env_order_is_a_stable_sort_by_class(lib):
    """mg_env_order: per-class counts, and lib_env[i] places env i in the
    library's class-grouped order (stable within a class); host only."""
    import numpy as np
    rng = np.random.default_rng(4)
    env_class = rng.integers(0, 5, size=1000).astype(np.int32)
    env_class[:7] = [4, 0, 4, 2, 2, 0, 1]
    counts, lib_env = B.mg_env_order(env_class, 5)
    assert counts.tolist() == np.bincount(env_class, minlength=5).tolist()
    assert sorted(lib_env.tolist()) == list(range(1000))           # a permutation
    order = np.argsort(env_class, kind="stable")                     # library env k holds user env order[k]
    assert np.array_equal(lib_env[order], np.arange(1000))
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    for c in range(5):                                               # class c owns [start_c, start_c + n_c)
        idx = lib_env[env_class == c]
        assert np.all(np.diff(idx) == 1) and (len(idx) == 0 or idx[0] == starts[c])
    with pytest.raises(B.MGError) as e:
        B.mg_env_order(np.array([0, 5, 1], np.int32), 5)
    assert e.value.code == B.MG_ERR_INVALID_ARG and "class 5" in str(e.value)
