"""Pins of the orbit oracle (oracle/orbit.py) against closed forms of
Sec. 3.4's ODE: two-body energy and angular-momentum conservation, the
circular-orbit period 2 pi sqrt(a^3/mu), torque-free spin of a symmetric
body (q(t) = q0 (x) (cos(wt/2), sin(wt/2) axis)), the cannonball
acceleration, and complex-step vs central-difference gradients."""
import math

import numpy as np

from oracle import mlp as omlp
from oracle import orbit as O


def test_two_body_invariants_one_day():
    m = O.Model("none", j2=0.0)
    z0 = O.circular_state(26560e3, math.radians(55))
    z0[3:6] *= 1.05  # eccentric
    z, tr = O.rk4(m, z0, np.zeros(1), 60.0, 1440, keep=True)
    E = 0.5 * np.sum(tr[:, 3:6] ** 2, axis=1) - O.MU / np.linalg.norm(tr[:, :3], axis=1)
    Hm = np.linalg.norm(np.cross(tr[:, :3], tr[:, 3:6]), axis=1)
    assert np.max(np.abs(E / E[0] - 1)) < 1e-9
    assert np.max(np.abs(Hm / Hm[0] - 1)) < 1e-9


def test_circular_period():
    a = 26560e3
    T = 2 * math.pi * math.sqrt(a ** 3 / O.MU)
    m = O.Model("none", j2=0.0)
    z0 = O.circular_state(a, math.radians(55), 0.3, 0.7)
    z = O.rk4(m, z0, np.zeros(1), T / 720, 720)
    assert np.linalg.norm(z[:3] - z0[:3]) / a < 1e-7


def test_torque_free_symmetric_spin():
    m = O.Model("none", inertia=(300.0, 300.0, 300.0), j2=0.0)
    z0 = O.circular_state(7000e3, 0.1)
    w = 0.01
    z0[10:13] = [0.0, 0.0, w]
    t = 600.0
    z = O.rk4(m, z0, np.zeros(1), 1.0, 600)
    q = z[6:10]
    assert np.allclose(q, [math.cos(w * t / 2), 0, 0, math.sin(w * t / 2)], atol=1e-10)
    assert np.allclose(z[10:13], [0, 0, w], atol=1e-15)


def test_cannonball_acceleration():
    m = O.Model("cannonball", P=4.56e-6, mass=800.0, sun=(0.0, 0.6, 0.8))
    rng = np.random.default_rng(0)
    q = rng.normal(size=4); q /= np.linalg.norm(q)
    z = np.concatenate([[7e6, 1e5, -2e5], [0, 7.5e3, 0], q, [1e-3, -2e-3, 5e-4]])
    k = m.f(z, np.array([12.0]))
    a_srp = k[3:6] - O.gravity(z[:3])
    # recovered by subtracting ~8 m/s^2 gravity from the total: round-off ~1e-15 m/s^2
    assert np.allclose(a_srp, -4.56e-6 * 12.0 / 800.0 * np.array([0.0, 0.6, 0.8]), rtol=0, atol=1e-14)


def test_complex_step_matches_central_difference():
    p = omlp.init_params(seed=2, sizes=(19, 16, 16, 16, 16, 6))
    scale = np.concatenate([np.ones(3), 4 * np.ones(14), np.ones(2) / (math.pi / 2)])
    offset = np.concatenate([np.zeros(3), -np.ones(14), np.zeros(2)])
    m = O.Model("proxy", P=4.56e-6 * 1e3, mass=100.0, sun=(0.3, 0.5, 0.81), params=p, scale=scale,
                offset=offset, mean=np.zeros(6), std=np.full(6, 5.0))
    z0 = O.circular_state(7000e3, 0.9)
    z0[10:13] = [1e-3, 2e-3, -1e-3]
    th = np.random.default_rng(1).uniform(0, 0.5, size=16)
    wN = np.random.default_rng(2).normal(size=13)
    gt, gz = O.cs_grad(m, z0, th, 10.0, 60, wN)
    for j in (0, 7, 15):
        # central differences are O(h^2): Richardson-combine steps 3e-3 and 1e-3 (O(h^4))
        f3 = O.fd_grad(m, z0, th, 10.0, 60, wN, j, 3e-3)
        f1 = O.fd_grad(m, z0, th, 10.0, 60, wN, j, 1e-3)
        fd = (9.0 * f1 - f3) / 8.0
        assert abs(fd - gt[j]) <= 1e-5 * abs(fd) + 1e-7, (j, fd, gt[j])


# ---------------------------------------------------------------- eclipse and third bodies (Sec. 3.4)
GM_SUN = 1.32712440018e20
AU = 1.495978707e11


def test_cylinder_eclipse_switches_srp():
    """Cylinder shadow: behind the Earth (r.e < 0) and within Re of the
    Earth-sun line the SRP acceleration is zero; in front, or outside the
    cylinder, it is the cannonball value."""
    m = O.Model("cannonball", P=1e-5, mass=10.0, sun=(1.0, 0.0, 0.0), eclipse=True)
    th = np.array([2.0])
    q = np.array([1.0, 0.0, 0.0, 0.0])
    def srp_acc(r):
        z = np.concatenate([r, [0, 0, 0], q, [0, 0, 0]])
        g = O.gravity(np.asarray(r, float))
        return m.f(z, th)[3:6] - g
    full = -1e-5 * 2.0 / 10.0 * np.array([1.0, 0.0, 0.0])
    assert np.allclose(srp_acc([7e6, 0.0, 0.0]), full, rtol=1e-12)                  # sunlit side
    assert np.allclose(srp_acc([-7e6, 0.0, 0.0]), 0.0, atol=1e-20)                  # umbra (on the axis)
    assert np.allclose(srp_acc([-7e6, O.RE * 0.999, 0.0]), 0.0, atol=1e-20)         # inside the cylinder
    assert np.allclose(srp_acc([-7e6, O.RE * 1.001, 0.0]), full, rtol=1e-12)        # just outside
    assert np.allclose(srp_acc([1.0, 7e6, 0.0]), full, rtol=1e-12)                  # terminator, r.e > 0


def test_third_body_tidal_limit():
    """For |r| << |s| the point-mass difference tends to the tidal
    acceleration GM/|s|^3 (3 (e.r) e - r) (Montenbruck & Gill Eq. 3.37's
    leading term); at r = 0 it vanishes exactly."""
    e = np.array([0.6, 0.8, 0.0])
    m = O.Model("none", sun=e, gm_sun=GM_SUN, sun_dist=AU)
    assert np.allclose(m.third_body(np.zeros(3)), 0.0, atol=1e-25)
    r = np.array([7.0e6, -2.0e6, 3.0e6])
    tidal = GM_SUN / AU ** 3 * (3.0 * (e @ r) * e - r)
    assert np.allclose(m.third_body(r), tidal, rtol=1e-4)
    moon = np.array([3.844e8, 0.0, 0.0])
    mm = O.Model("none", gm_moon=4.9028e12, moon=moon)
    rm = np.array([0.0, 7e6, 0.0])
    d = moon - rm
    want = 4.9028e12 * (d / np.linalg.norm(d) ** 3 - moon / np.linalg.norm(moon) ** 3)
    assert np.allclose(mm.third_body(rm), want, rtol=1e-14)


def test_complex_step_with_eclipse_and_third_bodies():
    """The discrete-map gradient stays exact (complex step vs central
    difference) with the eclipse switch and both point masses on, on an
    orbit that enters the shadow (the switch is constant between steps)."""
    m = O.Model("cannonball", P=1e-3, mass=10.0, sun=(1.0, 0.0, 0.0), eclipse=True, gm_sun=GM_SUN, sun_dist=AU,
                gm_moon=4.9028e12, moon=(0.0, 3.844e8, 0.0))
    z0 = O.circular_state(7.0e6, 0.3, u=2.5)
    th = np.array([3.0])
    wN = np.zeros(13); wN[0] = 1.0; wN[4] = 100.0
    g_th, g_z = O.cs_grad(m, z0, th, 30.0, 40, wN)
    fd = O.fd_grad(m, z0, th, 30.0, 40, wN, 0, 1e-4)
    assert abs(g_th[0] - fd) <= 1e-6 * abs(fd) + 1e-12
    # it really crossed into the shadow: the final state differs from the no-eclipse run
    m2 = O.Model("cannonball", P=1e-3, mass=10.0, sun=(1.0, 0.0, 0.0), gm_sun=GM_SUN, sun_dist=AU,
                 gm_moon=4.9028e12, moon=(0.0, 3.844e8, 0.0))
    zs = O.rk4(m, z0, th, 30.0, 40)
    zn = O.rk4(m2, z0, th, 30.0, 40)
    assert np.linalg.norm(zs[:3] - zn[:3]) > 1e-3


def test_j2_nodal_regression():
    """The J2 term against its classical secular effect on a circular
    orbit: the node regresses at dOmega/dt = -3/2 n J2 (Re/a)^2 cos i
    (first-order theory; Vallado, "Fundamentals of Astrodynamics", secular
    J2 rates).  A 7000 km, 50 degree orbit over 15 revolutions: the node
    moved by about -4.7 degrees; the measured drift (node from the angular
    momentum vector, sampled at the same phase of each revolution) agrees
    to 2 % (0.2 % in fact), and the inclination stays constant (no
    secular J2 rate)."""
    a, inc = 7000e3, math.radians(50.0)
    n = math.sqrt(O.MU / a ** 3)
    T = 2 * math.pi / n
    steps_per_rev = 120
    m = O.Model("none")
    z0 = O.circular_state(a, inc, 0.4, 0.0)
    z, tr = O.rk4(m, z0, np.zeros(1), T / steps_per_rev, 15 * steps_per_rev, keep=True)
    h = np.cross(tr[:, :3], tr[:, 3:6])
    node = np.unwrap(np.arctan2(h[:, 0], -h[:, 1]))
    incl = np.arccos(h[:, 2] / np.linalg.norm(h, axis=1))
    revs = node[::steps_per_rev]                                  # same phase of each revolution
    t = np.arange(len(revs)) * T
    rate = np.polyfit(t, revs, 1)[0]
    want = -1.5 * n * O.J2 * (O.RE / a) ** 2 * math.cos(inc)
    assert abs(rate / want - 1.0) < 0.02, (rate, want)
    assert abs(np.polyfit(t, incl[::steps_per_rev], 1)[0]) * t[-1] < 1e-3 * inc
    # with J2 off the node stays put
    z2 = O.rk4(O.Model("none", j2=0.0), z0, np.zeros(1), T / steps_per_rev, 15 * steps_per_rev)
    h2 = np.cross(z2[:3], z2[3:6])
    assert abs(math.atan2(h2[0], -h2[1]) - 0.4) < 1e-9


def test_torque_free_tumbling_conserves_inertial_angular_momentum():
    """Torque-free asymmetric body (I = 500, 400, 300 kg m^2) tumbling about
    all three axes: the inertial angular momentum R(q) I w and the kinetic
    energy 1/2 w.I w are conserved (Euler's equations with the quaternion
    kinematics q' = 1/2 q (x) (0, w)).  Only the consistent conventions
    conserve the vector: a flipped gyroscopic term or a transposed R(q)
    conserves the energy and |I w| but not R(q) I w."""
    m = O.Model("none", j2=0.0)
    z0 = O.circular_state(7000e3, 0.3)
    q = np.array([0.8, -0.2, 0.5, 0.26]); q /= np.linalg.norm(q)
    z0[6:10] = q
    z0[10:13] = [0.01, 0.02, -0.015]
    _, tr = O.rk4(m, z0, np.zeros(1), 0.5, 4000, keep=True)
    I = np.array([500.0, 400.0, 300.0])
    L = np.array([O.rot(s[6:10]) @ (I * s[10:13]) for s in tr])
    E = 0.5 * np.sum(I * tr[:, 10:13] ** 2, axis=1)
    assert np.max(np.linalg.norm(L - L[0], axis=1)) < 1e-9 * np.linalg.norm(L[0])
    assert np.max(np.abs(E / E[0] - 1.0)) < 1e-9
    assert np.max(np.abs(np.linalg.norm(tr[:, 6:10], axis=1) - 1.0)) < 1e-9
    # the body rate really tumbles (w changes direction by a large angle)
    w = tr[:, 10:13]
    assert np.min(w @ w[0] / (np.linalg.norm(w, axis=1) * np.linalg.norm(w[0]))) < 0.5
