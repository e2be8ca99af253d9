"""FP64 oracle of the spacecraft ODE and its RK4 integration -- TEST
INFRASTRUCTURE.

State z (13) = (r, v, q, w): position and velocity (inertial, m, m/s), the
unit quaternion q = (q0, q1, q2, q3) rotating body vectors into the inertial
frame, and the body angular velocity w (rad/s) (Sec. 3.4, state vector).

ODE (Sec. 3.4, Eq. "ODE"):
  r' = v
  v' = T^T F(wbar, theta) / m + o(r)          T = R(q)^T (inertial -> body)
  q' = 1/2 q (x) (0, w)                        quaternion kinematics
  w' = I^-1 (tau(wbar, theta) - w x I w)      I diagonal
with wbar = T e_sun the body-frame sun direction and o(r) two-body + J2
gravity:  -mu r/|r|^3 - 3/2 J2 mu Re^2/|r|^5 (x(1-5z^2/r^2), y(1-5z^2/r^2),
z(3-5z^2/r^2)).
Force models:
  'none'       F = tau = 0
  'cannonball' F = -P theta[0] wbar, tau = 0   (area x (1 + 4 rho_d/9))
  'proxy'      (F, tau) = P (std * y + mean), y = MLP(scale * (wbar, theta)
               + offset)  (the proxy of Sec. 3.3, FP32 weights held in FP64)
Optional terms of the paper's orbit force model (Sec. 3.4, "additional
accelerations"; Montenbruck & Gill's formulas):
  eclipse     cylinder shadow: SRP force and torque are zero while
              r.e_sun < 0 and |r - (r.e_sun) e_sun| < Re;
  third body  point masses at fixed inertial positions s (the Sun at
              sun_dist along e_sun, an optional Moon position):
              a = GM [(s - r)/|s - r|^3 - s/|s|^3].
RK4 (Sec. 3.4.1): z+ = z + h/6 (k1 + 2 k2 + 2 k3 + k4).
Gradient of L(z_N) w.r.t. theta and z0: complex-step differentiation of the
discrete map (d/dp f = Im f(p + i h)/h with h = 1e-30), exact to round-off
for this analytic map; `fd_grad` gives central differences for the pin.
"""
from __future__ import annotations

import numpy as np

MU = 3.986004418e14
J2 = 1.08263e-3
RE = 6378137.0


def rot(q):
    """R(q): body -> inertial, for q = (q0, q1, q2, q3) (scalar first);
    written for complex arguments (no abs, no normalisation)."""
    q0, q1, q2, q3 = q
    return np.array([
        [q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3), 2 * (q1 * q3 + q0 * q2)],
        [2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, 2 * (q2 * q3 - q0 * q1)],
        [2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1), q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3]])


def gravity(r, mu=MU, j2=J2, re=RE):
    x, y, z = r
    r2 = x * x + y * y + z * z
    rn = np.sqrt(r2)
    a = -mu * r / (rn * r2)
    k = -1.5 * j2 * mu * re * re / (r2 * r2 * rn)
    f = 5.0 * z * z / r2
    return a + k * np.array([x * (1.0 - f), y * (1.0 - f), z * (3.0 - f)])


class Model:
    def __init__(self, kind="none", P=1361.0 / 299792458.0, mass=1000.0, inertia=(500.0, 400.0, 300.0),
                 sun=(1.0, 0.0, 0.0), params=None, scale=None, offset=None, mean=None, std=None, j2=J2,
                 eclipse=False, gm_sun=0.0, sun_dist=0.0, gm_moon=0.0, moon=(0.0, 0.0, 0.0)):
        self.kind, self.P, self.mass = kind, P, mass
        self.I = np.asarray(inertia, np.float64)
        self.sun = np.asarray(sun, np.float64)
        self.params = params
        self.scale = None if scale is None else np.asarray(scale, np.float64)
        self.offset = None if offset is None else np.asarray(offset, np.float64)
        self.mean = None if mean is None else np.asarray(mean, np.float64)
        self.std = None if std is None else np.asarray(std, np.float64)
        self.j2 = j2
        self.eclipse = eclipse
        self.gm_sun, self.sun_dist = gm_sun, sun_dist
        self.gm_moon, self.moon = gm_moon, np.asarray(moon, np.float64)

    def in_shadow(self, r):
        """Cylinder eclipse test on the real part of r."""
        rr = np.real(np.asarray(r))
        p = rr @ self.sun
        return p < 0.0 and (rr @ rr - p * p) < RE * RE

    def third_body(self, r):
        a = np.zeros(3, dtype=np.result_type(r, np.float64))
        for gm, s in ((self.gm_sun, self.sun_dist * self.sun), (self.gm_moon, self.moon)):
            if gm == 0.0:
                continue
            d = s - r
            dn = np.sqrt(d @ d)
            sn = np.sqrt(s @ s)
            a = a + gm * (d / (dn * dn * dn) - s / (sn * sn * sn))
        return a

    def srp(self, wbar, theta):
        if self.kind == "none":
            return np.zeros(3, dtype=wbar.dtype), np.zeros(3, dtype=wbar.dtype)
        if self.kind == "cannonball":
            return -self.P * theta[0] * wbar, np.zeros(3, dtype=wbar.dtype)
        x = self.scale * np.concatenate([wbar, theta]) + self.offset
        h = x
        L = len(self.params)
        for l, (W, b) in enumerate(self.params):
            zz = W @ h + b
            h = zz / (1.0 + np.exp(-zz)) if l < L - 1 else zz
        y = self.P * (self.std * h + self.mean)
        return y[:3], y[3:]

    def f(self, z, theta):
        r, v, q, w = z[:3], z[3:6], z[6:10], z[10:13]
        R = rot(q)
        wbar = R.T @ self.sun
        F, tau = self.srp(wbar, theta)
        if self.eclipse and self.in_shadow(r):
            F, tau = 0.0 * F, 0.0 * tau
        a = R @ F / self.mass + gravity(r, j2=self.j2) + self.third_body(r)
        q0, q1, q2, q3 = q
        wx, wy, wz = w
        qd = 0.5 * np.array([-q1 * wx - q2 * wy - q3 * wz,
                             q0 * wx + q2 * wz - q3 * wy,
                             q0 * wy + q3 * wx - q1 * wz,
                             q0 * wz + q1 * wy - q2 * wx])
        Iw = self.I * w
        wd = (tau - np.cross(w, Iw)) / self.I
        return np.concatenate([v, a, qd, wd])


def rk4(model, z0, theta, h, n, keep=False):
    z = np.array(z0, dtype=np.result_type(z0, theta, np.float64))
    traj = [z.copy()] if keep else None
    for _ in range(n):
        k1 = model.f(z, theta)
        k2 = model.f(z + 0.5 * h * k1, theta)
        k3 = model.f(z + 0.5 * h * k2, theta)
        k4 = model.f(z + h * k3, theta)
        z = z + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if keep:
            traj.append(z.copy())
    return (z, np.array(traj)) if keep else z


def cs_grad(model, z0, theta, h, n, wN):
    """d(wN . z_N)/d theta and /d z0 by complex step."""
    eps = 1e-30
    th = np.asarray(theta, np.float64)
    g_th = np.zeros(th.shape[0])
    for j in range(th.shape[0]):
        tc = th.astype(np.complex128)
        tc[j] += 1j * eps
        g_th[j] = np.imag(wN @ rk4(model, np.asarray(z0, np.complex128), tc, h, n)) / eps
    g_z = np.zeros(13)
    for j in range(13):
        zc = np.asarray(z0, np.complex128).copy()
        zc[j] += 1j * eps
        g_z[j] = np.imag(wN @ rk4(model, zc, th.astype(np.complex128), h, n)) / eps
    return g_th, g_z


def fd_grad(model, z0, theta, h, n, wN, j, step):
    th = np.asarray(theta, np.float64)
    tp = th.copy(); tp[j] += step
    tm = th.copy(); tm[j] -= step
    return (wN @ rk4(model, z0, tp, h, n) - wN @ rk4(model, z0, tm, h, n)) / (2 * step)


def circular_state(a, inc, raan=0.0, u=0.0):
    """Circular orbit of radius a, inclination inc, node raan, argument u;
    identity attitude, zero body rate."""
    n = np.sqrt(MU / a ** 3)
    cu, su = np.cos(u), np.sin(u)
    cO, sO = np.cos(raan), np.sin(raan)
    ci, si = np.cos(inc), np.sin(inc)
    r = a * np.array([cO * cu - sO * su * ci, sO * cu + cO * su * ci, su * si])
    v = a * n * np.array([-cO * su - sO * cu * ci, -sO * su + cO * cu * ci, cu * si])
    return np.concatenate([r, v, [1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
