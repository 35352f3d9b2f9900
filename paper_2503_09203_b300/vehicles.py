"""Synthetic vehicle-class tables (input data only; no step arithmetic).

The paper's model library (Sec. III-D) names five vehicles (BlueROV with 6
thrusters, BlueROV Heavy with 8, LAUV, iAUV and a tiltrotor HAUV) but prints no
mass, inertia, hydrodynamic or thruster values, so the classes here are
synthetic. Class 0 follows the plain-step workload: 11.5 kg, neutrally buoyant,
centre of buoyancy 0.02 m above the centre of gravity, 8 thrusters in a fixed
vectored layout, diagonal added mass 5-10 kg / 0.1-0.5 kg m^2, translational
linear damping 4-20 and quadratic damping 10-50. Rotational damping is 1/20 of
the translational range, which keeps the explicit substep stable. Classes 1-4
carry 4, 6, 8 and 6 thrusters and 10, 25, 60 and 200 kg; their lengths scale
with (m / 11.5)^(1/3).

Coefficients are positive magnitudes (added mass and damping are subtracted
in the equation of motion). The body frame is x forward, y starboard, z down;
the centre of buoyancy "above" the centre of gravity therefore has negative z.
Every dictionary holds plain numbers; each side of the parity check (CUDA path
and oracle) packs them into its own records and derives everything else
(allocation matrix, rotor factor, inverse inertia, weight) itself.
"""
from __future__ import annotations

import math

BASE_MASS = 11.5
_S2 = math.sqrt(0.5)


def _vectored4(ax: float, ay: float):
    """Four horizontal thrusters at (+-ax, +-ay, 0) angled 45 degrees."""
    pos = [(ax, ay, 0.0), (ax, -ay, 0.0), (-ax, ay, 0.0), (-ax, -ay, 0.0)]
    d = [(_S2, -_S2, 0.0), (_S2, _S2, 0.0), (_S2, _S2, 0.0), (_S2, -_S2, 0.0)]
    return pos, d


def heavy8() -> dict:
    """Class 0: the plain-step vehicle (8 thrusters, 11.5 kg)."""
    hp, hd = _vectored4(0.15, 0.10)
    vp = [(0.12, 0.22, 0.0), (0.12, -0.22, 0.0), (-0.12, 0.22, 0.0), (-0.12, -0.22, 0.0)]
    vd = [(0.0, 0.0, 1.0)] * 4
    return dict(
        name="heavy8", n_thr=8, mass=11.5, Ig=(0.20, 0.25, 0.25), rg=(0.0, 0.0, 0.0),
        rb=(0.0, 0.0, -0.02), buoy_ratio=1.0,
        Ma=(6.0, 7.0, 9.0, 0.12, 0.12, 0.30),
        dl=(8.0, 10.0, 12.0, 0.4, 0.4, 0.3),
        dq=(20.0, 25.0, 30.0, 1.0, 1.0, 0.8),
        thr_pos=hp + vp, thr_dir=hd + vd,
        k_f=[40.0] * 8, T_rotor=[0.05] * 8, deadzone=[0.0] * 8,
    )


def _layout(n_thr: int):
    if n_thr == 8:
        hp, hd = _vectored4(0.15, 0.10)
        vp = [(0.12, 0.22, 0.0), (0.12, -0.22, 0.0), (-0.12, 0.22, 0.0), (-0.12, -0.22, 0.0)]
        return hp + vp, hd + [(0.0, 0.0, 1.0)] * 4
    if n_thr == 6:
        hp, hd = _vectored4(0.15, 0.10)
        vp = [(0.0, 0.11, 0.0), (0.0, -0.11, 0.0)]
        return hp + vp, hd + [(0.0, 0.0, 1.0)] * 2
    if n_thr == 4:
        pos = [(-0.15, 0.12, 0.0), (-0.15, -0.12, 0.0), (0.15, 0.0, 0.0), (-0.15, 0.0, 0.0)]
        d = [(1.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0)]
        return pos, d
    raise ValueError(f"no thruster layout for {n_thr} thrusters")


def scaled(name: str, mass: float, n_thr: int) -> dict:
    """A class geometrically similar to class 0 at another mass."""
    b = heavy8()
    rho = mass / BASE_MASS
    s = rho ** (1.0 / 3.0)
    pos, d = _layout(n_thr)
    return dict(
        name=name, n_thr=n_thr, mass=mass,
        Ig=tuple(v * rho * s * s for v in b["Ig"]), rg=(0.0, 0.0, 0.0),
        rb=(0.0, 0.0, -0.02 * s), buoy_ratio=1.0,
        Ma=tuple(v * rho for v in b["Ma"][:3]) + tuple(v * rho * s * s for v in b["Ma"][3:]),
        dl=tuple(v * s * s for v in b["dl"][:3]) + tuple(v * s ** 4 for v in b["dl"][3:]),
        dq=tuple(v * s * s for v in b["dq"][:3]) + tuple(v * s ** 5 for v in b["dq"][3:]),
        thr_pos=[tuple(c * s for c in p) for p in pos], thr_dir=list(d),
        k_f=[40.0 * s * s] * n_thr, T_rotor=[0.05 * s] * n_thr, deadzone=[0.0] * n_thr,
    )


# Actuator kinds (Sec. III-D): propeller, servo, fin (control surface),
# propeller tilted by a servo.
KIND_PROP, KIND_SERVO, KIND_FIN, KIND_TILT = 0, 1, 2, 3
RHO_WATER = 1025.0


def lauv() -> dict:
    """Rudder-propeller class (Sec. III-D, LAUV/iAUV type): one stern propeller
    and a cruciform tail of four independently driven fins (channels: propeller,
    top and bottom rudders with span axis z, port and starboard elevators with
    span axis y; chord along x). 18 kg torpedo body; underactuated."""
    fins_pos = [(-0.8, 0.0, -0.1), (-0.8, 0.0, 0.1), (-0.8, -0.1, 0.0), (-0.8, 0.1, 0.0)]
    fins_axis = [(0.0, 0.0, 1.0), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0), (0.0, 1.0, 0.0)]
    return dict(
        name="lauv5", n_thr=5, mass=18.0, Ig=(0.08, 1.6, 1.6), rg=(0.0, 0.0, 0.0),
        rb=(0.0, 0.0, -0.01), buoy_ratio=1.0,
        Ma=(1.0, 16.0, 16.0, 0.02, 1.6, 1.6),
        dl=(2.0, 20.0, 20.0, 0.2, 4.0, 4.0),
        dq=(4.0, 60.0, 60.0, 0.1, 8.0, 8.0),
        thr_pos=[(-0.95, 0.0, 0.0)] + fins_pos,
        thr_dir=[(1.0, 0.0, 0.0)] + [(0.0, 0.0, 0.0)] * 4,
        k_f=[30.0] + [0.0] * 4, T_rotor=[0.1] + [0.05] * 4, deadzone=[0.0] * 5,
        act_kind=[KIND_PROP] + [KIND_FIN] * 4, act_link=[0] * 5,
        act_axis=[(0.0, 0.0, 0.0)] + fins_axis, act_chord=[(0.0, 0.0, 0.0)] + [(1.0, 0.0, 0.0)] * 4,
        act_range=[0.0] + [0.35] * 4, fin_area=[0.0] + [0.012] * 4, fin_cl=[0.0] + [3.0] * 4,
        fin_cd0=[0.0] + [0.05] * 4, fin_cda=[0.0] + [1.2] * 4, rho=RHO_WATER,
    )


def tilt_hauv() -> dict:
    """Tiltrotor class (Sec. III-D, hybrid aerial-underwater type): four rotors
    at the ends of diagonal arms, thrust along -z at zero tilt, each turned
    about its own arm by a servo (channels 0-3 rotors, 4-7 servos, +-90 deg)."""
    s2 = math.sqrt(0.5)
    pos = [(0.18, 0.18, 0.0), (0.18, -0.18, 0.0), (-0.18, 0.18, 0.0), (-0.18, -0.18, 0.0)]
    arms = [(s2, s2, 0.0), (s2, -s2, 0.0), (-s2, s2, 0.0), (-s2, -s2, 0.0)]
    return dict(
        name="tilt8", n_thr=8, mass=2.8, Ig=(0.035, 0.035, 0.06), rg=(0.0, 0.0, 0.0),
        rb=(0.0, 0.0, -0.01), buoy_ratio=1.0,
        Ma=(1.2, 1.2, 2.5, 0.01, 0.01, 0.015),
        dl=(2.5, 2.5, 5.0, 0.04, 0.04, 0.03),
        dq=(5.0, 5.0, 10.0, 0.08, 0.08, 0.06),
        thr_pos=pos + pos, thr_dir=[(0.0, 0.0, -1.0)] * 4 + [(0.0, 0.0, 0.0)] * 4,
        k_f=[15.0] * 4 + [0.0] * 4, T_rotor=[0.05] * 4 + [0.08] * 4, deadzone=[0.0] * 8,
        act_kind=[KIND_TILT] * 4 + [KIND_SERVO] * 4, act_link=[4, 5, 6, 7] + [0] * 4,
        act_axis=arms + [(0.0, 0.0, 0.0)] * 4, act_chord=[(0.0, 0.0, 0.0)] * 8,
        act_range=[0.0] * 4 + [0.5 * math.pi] * 4, fin_area=[0.0] * 8, fin_cl=[0.0] * 8,
        fin_cd0=[0.0] * 8, fin_cda=[0.0] * 8, rho=RHO_WATER,
    )


def actuated_classes() -> list:
    """The three propulsion types of the model library side by side:
    multirotor (class 0), rudder-propeller, tiltrotor."""
    return [heavy8(), lauv(), tilt_hauv()]


def five_classes() -> list:
    """The five classes of the heterogeneous workloads (4/6/8 thrusters, 10-200 kg)."""
    return [heavy8(), scaled("quad4", 10.0, 4), scaled("rov6", 25.0, 6),
            scaled("work8", 60.0, 8), scaled("big6", 200.0, 6)]


# Domain-randomisation ranges, shaped like the training column of Table 2:
# per-env factors U[0.8, 1.2] on mass (inertia scales with it), added mass,
# damping and the CoB offset; current speed U[0, 0.5] m/s.
DR_TRAIN = dict(dr_enabled=1, current_enabled=1, current_3d=0, init_mode=0,
                mass_lo=0.8, mass_hi=1.2, added_lo=0.8, added_hi=1.2,
                damp_lo=0.8, damp_hi=1.2, cob_lo=0.8, cob_hi=1.2,
                cur_lo=0.0, cur_hi=0.5, target_half=5.0, pos_radius=2.0,
                max_angle=math.radians(30.0))

NO_DR = dict(DR_TRAIN, dr_enabled=0, current_enabled=0)
HOVER = dict(NO_DR, init_mode=1)
HOVER_DR = dict(DR_TRAIN, init_mode=1)
# Trajectory tracking (Sec. IV-B): helix or Lissajous references; the oracle
# reads `track`, the library reads the simulator's task.
TRACK_HELIX = dict(HOVER, track=1, track_kind=0)
TRACK_LISSAJOUS = dict(HOVER, track=1, track_kind=1)
TRACK_HELIX_DR = dict(HOVER_DR, track=1, track_kind=0)
# Payload disturbance (Sec. III-B; Table 2 payload mass, train range [0, 0.3]
# of the vehicle mass); the oracle reads `payload`, the library its config.
PAYLOAD = dict(HOVER, payload=1, payload_lo=0.0, payload_hi=0.3)
PAYLOAD_DR = dict(HOVER_DR, payload=1, payload_lo=0.0, payload_hi=0.3)
