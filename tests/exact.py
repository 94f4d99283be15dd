"""Closed-form solutions of ideal relativistic hydrodynamics used to pin the oracle.

Written from the physics, independently of the oracle's code:

* the 1-D Riemann problem for p = c^2 e with both states at rest
  (left-facing rarefaction + right-facing shock), from the Riemann invariant
  atanh(v) + c/(1+c^2) ln e and the Taub jump conditions
  s [T^00] = [T^01], s [T^01] = [T^11];
* the Bjorken boost-invariant flow v = z/t, e = e0 (tau0/tau)^(1+c^2);
* the Hubble-like 3-D expansion of Sec. 3.2.2, v = r/t,
  e = e0 (tau0/tau)^(3(1+c^2));
* a stationary 2-D vortex: circular flow v_phi(r) held by the radial
  pressure gradient, dp/dr = (e + p) gamma^2 v_phi^2 / r.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq


def _tmunu(e, v, c2):
    p = c2 * e
    g2 = 1.0 / (1.0 - v * v)
    w = (e + p) * g2
    return w - p, w * v, w * v * v + p   # T00, T01, T11


def _shock_velocity_behind(e_s, e_r, c2):
    """Fluid velocity behind a right-moving shock into rest state e_r (Taub)."""
    p_s, p_r = c2 * e_s, c2 * e_r

    def resid(v):
        t00, t01, t11 = _tmunu(e_s, v, c2)
        # eliminate the shock speed s = T01 / (T00 - e_r)
        return t01 * t01 - (t11 - p_r) * (t00 - e_r)

    vmax = 1.0 - 1e-15
    return brentq(resid, 1e-300, vmax, xtol=1e-16, rtol=1e-15, maxiter=500) if p_s > p_r else 0.0


class Riemann:
    """Exact solution for left state (e_l, v=0), right state (e_r, v=0), e_l > e_r."""

    def __init__(self, e_l=10.0, e_r=1.0, c2=1.0 / 3.0):
        self.e_l, self.e_r, self.c2 = e_l, e_r, c2
        self.c = math.sqrt(c2)
        k = self.c / (1.0 + c2)

        def match(e_s):
            v_rare = math.tanh(k * math.log(e_l / e_s))
            return v_rare - _shock_velocity_behind(e_s, e_r, c2)

        self.e_star = brentq(match, e_r * (1 + 1e-12), e_l * (1 - 1e-12), xtol=1e-15,
                             rtol=1e-15)
        self.v_star = math.tanh(k * math.log(e_l / self.e_star))
        t00, t01, _ = _tmunu(self.e_star, self.v_star, c2)
        self.shock_speed = t01 / (t00 - e_r)
        self.head = -self.c
        self.tail = (self.v_star - self.c) / (1.0 - self.v_star * self.c)

    def sample_n(self, x, t, n_l, n_r):
        """Rest-frame density n of a passive conserved charge (R = n gamma with
        flux R v, the EOS independent of n) in the same Riemann problem.
        Smooth flow conserves both s u^mu and n u^mu, so n/s is constant along
        flow lines, with s ~ e^(1/(1+c^2)) for p = c^2 e (ds/s = de/(e+p)):
        n = n_l (e/e_l)^(1/(1+c^2)) in the fan and up to the contact, which
        moves with v*.  Across the shock, n gamma (v - s) is continuous:
        n = n_r s / (gamma* (s - v*)) between the contact and the shock."""
        xi = np.asarray(x, dtype=np.float64) / t
        e, _ = self.sample(x, t)
        k = 1.0 / (1.0 + self.c2)
        n = n_l * (e / self.e_l) ** k
        s = self.shock_speed
        g = 1.0 / math.sqrt(1.0 - self.v_star ** 2)
        right_star = (xi >= self.v_star) & (xi < s)
        n[right_star] = n_r * s / (g * (s - self.v_star))
        n[xi >= s] = n_r
        return n

    def jump_residuals(self):
        t00, t01, t11 = _tmunu(self.e_star, self.v_star, self.c2)
        s = self.shock_speed
        return (s * (t00 - self.e_r) - t01, s * t01 - (t11 - self.c2 * self.e_r))

    def sample(self, x, t):
        xi = np.asarray(x, dtype=np.float64) / t
        e = np.empty_like(xi)
        v = np.empty_like(xi)
        c, c2 = self.c, self.c2
        left = xi < self.head
        fan = (xi >= self.head) & (xi < self.tail)
        star = (xi >= self.tail) & (xi < self.shock_speed)
        right = xi >= self.shock_speed
        e[left], v[left] = self.e_l, 0.0
        vf = (xi[fan] + c) / (1.0 + xi[fan] * c)
        v[fan] = vf
        e[fan] = self.e_l * ((1.0 - vf) / (1.0 + vf)) ** ((1.0 + c2) / (2.0 * c))
        e[star], v[star] = self.e_star, self.v_star
        e[right], v[right] = self.e_r, 0.0
        return e, v


def bjorken(z, t, e0=1.0, tau0=1.0, c2=1.0 / 3.0):
    z = np.asarray(z, dtype=np.float64)
    tau = np.sqrt(t * t - z * z)
    return e0 * (tau0 / tau) ** (1.0 + c2), z / t


def hubble(r, t, e0=1.0, tau0=4.0, c2=1.0 / 3.0):
    r = np.asarray(r, dtype=np.float64)
    tau = np.sqrt(t * t - r * r)
    return e0 * (tau0 / tau) ** (3.0 * (1.0 + c2)), r / t


def ellipsoidal(coords, t, C=2.0, b=1.0, T=(0.4, 0.6, 0.8)):
    """The ellipsoidal flow of Sec. 3.2 (pressureless, p = 0): with
    a_i = t/(t + T_i), v_i = a_i x_i / t = x_i/(t + T_i) (reading R17: the
    printed index order of v is taken as a typo, tau pairs a_i with x_i) and
    tau^2 = t^2 - sum_i a_i^2 x_i^2,
        e = C / prod_i(t + T_i) * exp(-b^2 t^2 / tau^2)  inside tau^2 > 0,
    vacuum (e = v = 0) outside.  Every element moves ballistically (t/tau is
    its Lorentz factor, constant along the motion) and the lab-frame density
    e gamma scales with the inverse volume prod_i(t + T_i) of the expansion,
    so E and M solve the p = 0 equations exactly.  coords: one array per
    active axis (1, 2 or 3 of them, broadcastable), with T[i] for axis i."""
    v = [np.asarray(x, dtype=np.float64) / (t + T[i]) for i, x in enumerate(coords)]
    v2 = sum(vi * vi for vi in v)
    inside = v2 < 1.0
    gamma2 = np.where(inside, 1.0 / np.where(inside, 1.0 - v2, 1.0), 0.0)
    norm = C / np.prod([t + T[i] for i in range(len(coords))])
    e = np.where(inside, norm * np.exp(-b * b * gamma2), 0.0)
    return e, [np.where(inside, vi, 0.0) for vi in v]


def vortex(x, y, vmax=0.5, w=0.1, e_far=1.0, c2=1.0 / 3.0):
    """Stationary vortex of an ideal fluid with p = c^2 e in the xy plane.

    Circular flow v_phi(r) = vmax (r/w) exp((1 - r^2/w^2)/2) (largest, vmax,
    at r = w).  For steady circular flow the energy equation holds trivially
    (the flux (e+p) gamma^2 v is divergence-free) and the radial momentum
    equation is the balance dp/dr = (e + p) gamma^2 v_phi^2 / r, i.e.
    d ln e / dr = (1 + c^2)/c^2 * v_phi^2 / ((1 - v_phi^2) r), integrated
    inwards from e = e_far at r = 20 w by adaptive quadrature.  The state is a
    solution at every time.  Returns (e, vx, vy) on the points (x, y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = np.sqrt(x * x + y * y)

    def vphi(s):
        return vmax * (s / w) * np.exp(0.5 * (1.0 - (s / w) ** 2))

    def dlne(s):
        v = vphi(s)
        return (1.0 + c2) / c2 * v * v / ((1.0 - v * v) * s)

    def lne(s):
        if s >= 20.0 * w:
            return math.log(e_far)
        val, _ = quad(dlne, max(s, 1e-300), 20.0 * w, epsabs=1e-15, epsrel=1e-13, limit=200)
        return math.log(e_far) - val

    e = np.exp(np.vectorize(lne)(r))
    vp = vphi(r)
    rs = np.where(r > 0, r, 1.0)
    return e, -vp * y / rs, vp * x / rs
