"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a value fixed by the paper or by
mathematics: the paper's printed limiter functions and their symmetry
(Sec. 2.5), Lorentz-boosted stress tensors (Eq. 3-4), the paper's own
fixed-point iteration for Eq. 23, the textbook FORCE flux, exact
solutions (Riemann problem, Bjorken flow, Hubble-like expansion of
Sec. 3.2.2), conservation, mirror and axis symmetry, closed forms of the
tabulated EOS, finite differences for the MLP gradient.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_06340_b300 import inputs as I
from tests import exact

RNG = np.random.default_rng(1510_06340)


# ---------------------------------------------------------------- limiters
def xi_paper(kind, r):
    """The limiter functions as printed in Sec. 2.5 (Eq. 18-21); MC from van Leer (1977)."""
    if kind == "minmod":
        return max(0.0, min(1.0, r))
    if kind == "superbee":
        return max(0.0, min(2 * r, 1.0), min(r, 2.0))
    if kind == "vanleer":
        return (r + abs(r)) / (1 + abs(r))
    if kind == "vanalbada":       # clipped to r > 0 (reading R5)
        return (r * r + r) / (r * r + 1) if r > 0 else 0.0
    if kind == "mc":
        return max(0.0, min(2 * r, 0.5 * (1 + r), 2.0))
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["minmod", "superbee", "vanleer", "vanalbada", "mc"])
def test_limited_slope_is_a_times_xi_of_r(kind):
    o = O.Oracle(4, limiter=kind)
    for _ in range(2000):
        a, b = RNG.normal(size=2) * 10.0 ** RNG.uniform(-3, 3, size=2)
        want = a * xi_paper(kind, b / a)
        got = o.limiter(a, b)
        assert abs(got - want) <= 1e-14 * max(abs(a), abs(b)), (kind, a, b, got, want)


@pytest.mark.parametrize("kind", ["minmod", "superbee", "vanleer", "vanalbada", "mc"])
def test_limiter_symmetry_and_tvd_region(kind):
    """xi(1/r) = xi(r)/r (Eq. 22) <=> phi(a, b) = phi(b, a); xi(1) = 1; TVD bounds."""
    o = O.Oracle(4, limiter=kind)
    for _ in range(2000):
        a, b = RNG.normal(size=2)
        s = o.limiter(a, b)
        assert abs(s - o.limiter(b, a)) <= 1e-15 * max(abs(a), abs(b))
        if a * b <= 0:
            assert s == 0.0
        else:
            assert s * a >= 0
            assert abs(s) <= 2 * min(abs(a), abs(b)) + 1e-15
        assert abs(o.limiter(a, a) - a) <= 1e-15 * abs(a)


def test_no_limiter_is_central_slope():
    """Eq. 14: Delta_i = (U_{i+1} - U_{i-1}) / 2."""
    o = O.Oracle(4, limiter="none")
    for _ in range(100):
        um, u0, up = RNG.normal(size=3)
        assert abs(o.limiter(u0 - um, up - u0) - 0.5 * (up - um)) < 1e-15


# --------------------------------------------------------- stress tensor
def boosted_tensor(e, v, c2=1.0 / 3.0):
    """T^{mu nu} = Lambda diag(e, p, p, p) Lambda^T for the boost taking rest to velocity v."""
    v = np.asarray(v, dtype=np.float64)
    v2 = v @ v
    g = 1.0 / math.sqrt(1.0 - v2)
    L = np.eye(4)
    L[0, 0] = g
    L[0, 1:] = L[1:, 0] = g * v
    if v2 > 0:
        L[1:, 1:] += (g - 1.0) * np.outer(v, v) / v2
    p = c2 * e
    return L @ np.diag([e, p, p, p]) @ L.T


def random_prim(vmax=0.99):
    e = 10.0 ** RNG.uniform(-2, 2)
    d = RNG.normal(size=3)
    d /= np.linalg.norm(d)
    return e, d * vmax * RNG.uniform() ** (1 / 3)


def test_prim2cons_is_boosted_rest_tensor():
    o = O.Oracle(4)
    for _ in range(500):
        e, v = random_prim()
        T = boosted_tensor(e, v)
        U = o.prim2cons(e, v)
        np.testing.assert_allclose(U, T[0], rtol=1e-13, atol=1e-13 * T[0, 0])


def test_cons2prim_roundtrip_to_high_velocity():
    o = O.Oracle(4)
    for vmax in (0.5, 0.9, 0.999, 0.999999):
        for _ in range(200):
            e, v = random_prim(vmax)
            U = boosted_tensor(e, v)[0]
            e2, v2, p2, st, _ = o.cons2prim(U)
            g2 = 1.0 / (1.0 - v @ v)
            assert st == 0
            assert np.abs(v2 - v).max() <= 2e-15 * g2 + 1e-15
            assert abs(e2 - e) <= 1e-14 * e * g2
            assert abs(p2 - e / 3.0) <= 1e-14 * e * g2


def test_cons2prim_matches_paper_fixed_point():
    """Sec. 2.6 solves Eq. 23 as a fixed point in v; the oracle's closed form is its limit."""
    o = O.Oracle(4)
    for _ in range(200):
        e, v = random_prim(0.95)
        U = boosted_tensor(e, v)[0]
        E, M = U[0], np.linalg.norm(U[1:])
        vv = 0.0
        for _ in range(2000):
            vv = M / (E + (E - M * vv) / 3.0)
        _, v2, _, _, _ = o.cons2prim(U)
        assert abs(np.linalg.norm(v2) - vv) <= 1e-14


def test_cons2prim_caps_and_vacuum():
    o = O.Oracle(4)
    e, v, p, st, _ = o.cons2prim([1.0, 2.0, 0.0, 0.0])     # |M| > E
    assert st == 1 and 0 < v[0] < 1 and p >= 0
    e, v, p, st, _ = o.cons2prim([-1.0, 0.1, 0.0, 0.0])    # E <= 0
    assert st == 2 and p == 0 and not v.any()


def test_cons2prim_is_scale_free_down_to_the_vacuum_threshold():
    """R18: the p = c2 e recovery is homogeneous (v of lambda U equals v of U,
    p scales with lambda) down to E = 2^-500, where E^2 is still normal; below
    it the state is vacuum.  Without the threshold E ~ 1e-323 gave |v| > 1."""
    for cs2 in (0.0, 1.0 / 3.0):
        o = O.Oracle(4, cs2=cs2)
        U = np.array([1.0, 0.5, 0.3, 0.2])
        e1, v1, p1, _, _ = o.cons2prim(U)
        for k in (-200, -450, -499):
            s = 2.0 ** k
            e2, v2, p2, st, _ = o.cons2prim(U * s)
            assert st == 0 and np.allclose(v2, v1, rtol=1e-14, atol=0)
            assert p2 == pytest.approx(p1 * s, rel=1e-13, abs=0)
        for E in (2.0 ** -501, 1e-300, 2.47e-323):
            e, v, p, st, _ = o.cons2prim(np.array([E, 0.4 * E, 0.0, 0.8 * E]))
            assert st == 2 and p == 0 and not v.any()


@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_is_row_of_boosted_tensor(d):
    """Eq. 3: F_d = (T^{d0}, T^{dx}, T^{dy}, T^{dz})."""
    o = O.Oracle(4)
    for _ in range(300):
        e, v = random_prim()
        T = boosted_tensor(e, v)
        F = o.flux(d, T[0])
        np.testing.assert_allclose(F, T[1 + d], rtol=1e-12, atol=1e-13 * T[0, 0])


# ------------------------------------------------------------ MUSTA-FORCE
def test_musta_force_is_consistent():
    for k in (1, 2, 3, 4):
        o = O.Oracle(4, stages=k)
        for _ in range(50):
            e, v = random_prim()
            U = boosted_tensor(e, v)[0]
            for d in range(3):
                F = o.musta_force(d, 0.37, U, U)
                np.testing.assert_allclose(F, o.flux(d, U), rtol=1e-15, atol=1e-15 * U[0])


def test_single_stage_is_textbook_force():
    """k = 1 is Toro's FORCE flux 1/4 [F_L + 2 F(U_0) + F_R - (dx/dt)(U_R - U_L)],
    U_0 = (U_L + U_R)/2 - (dt/2dx)(F_R - F_L)  (reading R1 of Eq. 10)."""
    o = O.Oracle(4, stages=1)
    lam = 0.31
    for _ in range(200):
        UL = boosted_tensor(*random_prim(0.8))[0]
        UR = boosted_tensor(*random_prim(0.8))[0]
        d = int(RNG.integers(3))
        FL, FR = o.flux(d, UL), o.flux(d, UR)
        U0 = 0.5 * (UL + UR) - 0.5 * lam * (FR - FL)
        want = 0.25 * (FL + 2.0 * o.flux(d, U0) + FR - (UR - UL) / lam)
        got = o.musta_force(d, lam, UL, UR)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * max(UL[0], UR[0]))


def test_musta_predictor_fixes_uniform_states():
    """For U_L = U_R the local Riemann update of Eq. 8 leaves both states unchanged."""
    o2 = O.Oracle(4, stages=2)
    U = boosted_tensor(*random_prim(0.6))[0]
    np.testing.assert_allclose(o2.musta_force(0, 0.4, U, U), o2.flux(0, U), rtol=1e-15)


# ------------------------------------------------------------ signal speed
def test_signal_speed_special_cases():
    o = O.Oracle(4)
    c = math.sqrt(1.0 / 3.0)
    U = boosted_tensor(1.0, [0, 0, 0])[0]
    for d in range(3):
        assert abs(o.signal_speed(U, d) - c) < 1e-15
    for _ in range(100):
        s = RNG.uniform(-0.99, 0.99)
        U = boosted_tensor(2.0, [s, 0, 0])[0]
        # along the flow: relativistic velocity addition
        assert abs(o.signal_speed(U, 0) - (abs(s) + c) / (1 + abs(s) * c)) < 1e-13
        # across the flow
        want = c * math.sqrt((1 - s * s) / (1 - s * s * c * c))
        assert abs(o.signal_speed(U, 1) - want) < 1e-13
    for _ in range(300):
        U = boosted_tensor(*random_prim(0.999))[0]
        for d in range(3):
            assert 0 < o.signal_speed(U, d) <= 1.0


# ------------------------------------------------------------- Riemann problem
def test_exact_riemann_solver_jump_conditions():
    R = exact.Riemann(10.0, 1.0)
    r1, r2 = R.jump_residuals()
    assert abs(r1) < 1e-12 and abs(r2) < 1e-12
    # independently derived star state for e_L = 10, e_R = 1, p = e/3
    assert abs(R.e_star - 3.139831558201) < 1e-11
    assert abs(R.v_star - 0.463381465430) < 1e-11
    assert abs(R.shock_speed - 0.752115385414) < 1e-11


def run_shock_tube(n, limiter="minmod", stages=2, rk_order=2, hancock=1):
    g, prim = I.shock_tube(n)
    o = O.Oracle(n, dx=g["dx"], x0=-1.0, bc="outflow", limiter=limiter, stages=stages,
                 rk_order=rk_order, hancock=hancock, cfl=0.4)
    U = o.prim2cons_field(*prim)
    nsteps, t = o.run(U, 100000, t_end=0.8)
    e, vx, _, _, _ = o.cons2prim_field(U)
    x = I.cell_centres(n, -1.0, g["dx"])
    ex, vex = exact.Riemann().sample(x, 0.8)
    l1e = np.abs(e.ravel() - ex).sum() / np.abs(ex).sum()
    l1v = np.abs(vx.ravel() - vex).sum() / np.abs(vex).sum()
    return l1e, l1v, nsteps, t, e.ravel(), vx.ravel()


def test_shock_tube_converges_to_exact_solution():
    errs = [run_shock_tube(n)[:2] for n in (250, 500, 1000)]
    for (e1, v1), (e2, v2) in zip(errs, errs[1:]):
        assert e2 < e1 / 1.5 and v2 < v1 / 1.5
    l1e, l1v, nsteps, t, _, _ = run_shock_tube(1000)
    assert t == 0.8 and 600 < nsteps < 1200
    assert l1e < 6e-3 and l1v < 1.5e-2


def test_more_musta_stages_reduce_error():
    errs = [run_shock_tube(500, stages=k)[0] for k in (1, 2, 3, 4)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_minbee_overshoots_less_than_superbee():
    """Sec. 3.2.1: Minbee removes most of the velocity overshoot, Superbee enhances it."""
    R = exact.Riemann()
    over = {lim: run_shock_tube(500, limiter=lim)[5].max() - R.v_star
            for lim in ("minmod", "superbee")}
    assert over["minmod"] < over["superbee"]


# ------------------------------------------------------------- smooth flow
def bjorken_error(n, limiter, rk_order, hancock, t0=2.0, t1=2.4):
    dx = 2.0 / n
    z = I.cell_centres(n, -1.0, dx)
    e, v = exact.bjorken(z, t0)
    o = O.Oracle(n, dx=dx, x0=-1.0, bc="outflow", limiter=limiter, rk_order=rk_order,
                 hancock=hancock, fixed_dt=0.2 * dx)
    zero = np.zeros((1, 1, n))
    U = o.prim2cons_field(e.reshape(1, 1, n), v.reshape(1, 1, n), zero, zero)
    o.run(U, 100000, t_end=t1, t=t0)
    ee, vv, _, _, _ = o.cons2prim_field(U)
    ex, vex = exact.bjorken(z, t1)
    m = np.abs(z) < 0.5          # outside the light cone of the boundaries
    return np.abs(ee.ravel() - ex)[m].mean(), np.abs(vv.ravel() - vex)[m].mean()


@pytest.mark.parametrize("limiter,rk_order,hancock,lo,hi", [
    ("none", 1, 1, 1.8, 2.6),     # single-stage MUSCL-Hancock: second order
    ("none", 2, 0, 1.8, 2.3),     # RK2 on the plain MUSCL operator: second order
    ("none", 3, 0, 1.8, 2.3),
    ("minmod", 1, 1, 1.8, 2.3),
    ("none", 2, 1, 0.9, 1.2),     # Hancock inside each RK2 stage: first order in time
])
def test_bjorken_convergence_order(limiter, rk_order, hancock, lo, hi):
    e1, v1 = bjorken_error(200, limiter, rk_order, hancock)
    e2, v2 = bjorken_error(400, limiter, rk_order, hancock)
    assert lo < math.log2(e1 / e2) < hi
    assert lo - 0.2 < math.log2(v1 / v2) < hi + 0.3


@pytest.mark.parametrize("axis", [1, 2])
def test_axis_embedding_equals_1d_run(axis):
    """A 1-D problem along y or z of a 3-D grid (uniform across) equals the 1-D
    run along x: the transverse sweeps change nothing, Strang gives two half
    steps along y, one full step along z."""
    n = 64
    dx = 2.0 / n
    z = I.cell_centres(n, -1.0, dx)
    e, v = exact.bjorken(z, 2.0)
    dt = 0.2 * dx
    ref = O.Oracle(n, dx=dx, x0=-1.0, bc="outflow", fixed_dt=dt / 2 if axis == 1 else dt)
    zero = np.zeros((1, 1, n))
    U1 = ref.prim2cons_field(e.reshape(1, 1, n), v.reshape(1, 1, n), zero, zero)
    ref.run(U1, 6 if axis == 1 else 3)
    shape = [4, 4, 4]
    shape[2 - axis] = n
    bc = ["periodic"] * 3
    bc[axis] = "outflow"
    o = O.Oracle(shape[2], shape[1], shape[0], dx=dx, bc=tuple(bc), fixed_dt=dt)
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    ee = np.broadcast_to(e[tuple(sl)], shape).copy()
    vv = np.broadcast_to(v[tuple(sl)], shape).copy()
    zz = np.zeros(shape)
    vel = [zz, zz, zz]
    vel[axis] = vv
    U3 = o.prim2cons_field(ee, *vel)
    o.run(U3, 3)
    line = [slice(None), 1, 1, 1]
    line[1 + (2 - axis)] = slice(None)
    got = U3[tuple(line)]
    assert np.array_equal(got[0], U1[0].ravel())
    assert np.array_equal(got[1 + axis], U1[1].ravel())
    others = [q for q in (1, 2, 3) if q != 1 + axis]
    assert not got[others].any()


def hubble_error(n, dx, dt, nsteps, t0=2.0, **kw):
    lo = -0.5 * n * dx
    c = I.cell_centres(n, lo, dx)
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(xx * xx + yy * yy + zz * zz)
    inside = r < t0 - 0.5                      # vacuum outside r < t - 0.5 fm
    e, vr = exact.hubble(np.where(inside, r, 0.0), t0)
    e = np.where(inside, e, 0.0)
    vr = np.where(inside, vr, 0.0)
    rs = np.where(r > 0, r, 1.0)
    o = O.Oracle(n, n, n, dx=dx, x0=lo, y0=lo, z0=lo, bc="outflow", fixed_dt=dt, **kw)
    U = o.prim2cons_field(e, vr * xx / rs, vr * yy / rs, vr * zz / rs)
    o.run(U, nsteps)
    ee, vx, vy, vz, _ = o.cons2prim_field(U)
    core = r < 0.5
    ex, vex = exact.hubble(r[core], t0 + nsteps * dt)
    vnum = (vx * xx + vy * yy + vz * zz)[core] / rs[core]
    return np.abs(ee[core] / ex - 1).max(), np.abs(vnum - vex).max()


@pytest.mark.slow
def test_hubble_expansion_interior_converges():
    """Sec. 3.2.2 (its table: e0 = 1, c_s^2 = 1/3, tau0 = 4, t0 = 2, dx = 0.1, dt = 0.03;
    vacuum outside r < t - 0.5), on a reduced box: the core follows
    e = e0 (tau0/tau)^4, v = r/t, and the error falls under refinement at fixed
    Courant number."""
    e1, v1 = hubble_error(32, 0.1, 0.03, 10)
    e2, v2 = hubble_error(64, 0.05, 0.015, 20)
    assert e1 < 0.04 and v1 < 0.01
    assert e2 < e1 / 2 and v2 < v1 / 2


# ------------------------------------------------------- splitting order
def vortex_error(n, lam=0.6, T=0.2, lie=False):
    """Mean |U(T) - U(0)| per field of the stationary vortex on n^2 cells of
    [-0.5, 0.5]^2 (periodic), single-stage MUSCL-Hancock (rk_order 1, second
    order per sweep), central slopes, fixed dt = lam dx.  lie: compose the
    oracle's own sweeps as X(dt) Y(dt) instead of taking its step."""
    dx = 1.0 / n
    c = I.cell_centres(n, -0.5, dx)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    e, vx, vy = exact.vortex(xx, yy)
    steps = int(round(T / (lam * dx)))
    dt = T / steps
    o = O.Oracle(n, n, 1, dx=dx, x0=-0.5, y0=-0.5, bc="periodic", limiter="none",
                 rk_order=1, hancock=1, fixed_dt=dt)
    U0 = o.prim2cons_field(e[None], vx[None], vy[None], np.zeros((1, n, n)))
    U = U0.copy()
    if lie:
        for _ in range(steps):
            o.sweep(U, 0, dt)
            o.sweep(U, 1, dt)
    else:
        o.run(U, steps)
    return np.abs(U - U0)[:3].mean(axis=(1, 2, 3))


@pytest.mark.slow
def test_strang_step_is_second_order_in_time():
    """The step's splitting is the symmetric Strang order (reading R7): on the
    stationary vortex (an exact 2-D solution whose x and y operators do not
    commute) its error falls at second order as dx and dt are halved
    together.  The oracle's own sweeps composed in Lie order X(dt) Y(dt) --
    the mistake this guards against -- fall at about first order and fail
    the same bound."""
    e1, e2 = vortex_error(64), vortex_error(128)
    order = np.log2(e1 / e2)
    assert (order > 1.8).all(), order
    assert (e2 < 3e-4).all(), e2
    l1, l2 = vortex_error(64, lie=True), vortex_error(128, lie=True)
    lie_order = np.log2(l1 / l2)
    assert (lie_order < 1.5).all(), lie_order
    assert (l2 > 2 * e2).all()


# --------------------------------------------------------- 3-D invariants
def blast_oracle(n, limiter="minmod"):
    g, prim = I.spherical_blast(n)
    o = O.Oracle(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic",
                 limiter=limiter, cfl=0.4)
    return o, o.prim2cons_field(*prim)


@pytest.mark.parametrize("limiter", ["minmod", "mc", "superbee"])
def test_periodic_blast_conserves_energy_momentum(limiter):
    o, U = blast_oracle(16, limiter)
    s0 = o.conservation_sums(U)
    o.run(U, 8)
    s1 = o.conservation_sums(U)
    assert abs(s1[0] - s0[0]) <= 1e-13 * s0[0]
    assert np.abs(s1[1:]).max() <= 1e-13 * s0[0]


def test_blast_mirror_symmetry():
    """Reflection x -> -x maps the solution to itself with M_x odd (Sec. 2.5, Eq. 22)."""
    o, U = blast_oracle(16)
    o.run(U, 6)
    scale = U[0].max()
    for ax in range(3):
        arr_ax = 3 - ax
        R = np.flip(U, axis=arr_ax).copy()
        R[1 + ax] *= -1.0
        assert np.abs(R - U).max() <= 1e-14 * scale


# ------------------------------------------------------------ tabulated EOS
def test_eos_closed_form_derivative_is_cs2():
    e = np.exp(np.linspace(math.log(1e-5), math.log(1e3), 400))
    h = 1e-6 * e
    dp = (I.eos_p_exact(e + h) - I.eos_p_exact(e - h)) / (2 * h)
    np.testing.assert_allclose(dp, I.eos_cs2_exact(e), rtol=1e-7, atol=1e-9)
    assert abs(I.eos_p_exact(1e-9) - 1e-9 / 3) < 1e-20       # p -> e/3 at low e


def test_eos_table_interpolation_error():
    tab = I.eos_table()
    o = O.Oracle(4, eos=tab)
    h = (tab["lne_max"] - tab["lne_min"]) / (tab["n"] - 1)
    for e in 10.0 ** RNG.uniform(-5.9, 3.9, size=400):
        p = o.eos_p(e)
        # linear interpolation in u = ln e: error <= h^2/8 max|d2p/du2|, d2p/du2 <= ~2e
        assert abs(p - I.eos_p_exact(e)) <= h * h / 8 * 2.0 * e * 1.01
        assert abs(o.eos_cs2(e) - I.eos_cs2_exact(e)) <= h * h / 8 * 2.0
    assert o.eos_p(1e-8) == 1e-8 / 3.0
    emax = math.exp(tab["lne_max"])
    assert abs(o.eos_p(2 * emax) - (tab["p"][-1] + tab["cs2"][-1] * emax)) < 1e-9 * emax


def test_newton_cons2prim_roundtrip_table_eos():
    tab = I.eos_table()
    for seed_kind in (0, 1):
        o = O.Oracle(4, eos=tab, seed_kind=seed_kind)
        for _ in range(300):
            e, v = random_prim(0.999)
            U = o.prim2cons(e, v)
            e2, v2, p2, st, it = o.cons2prim(U)
            g2 = 1.0 / (1.0 - v @ v)
            assert st == 0 and it < 50
            assert np.abs(v2 - v).max() < 1e-13 * g2
            assert abs(e2 - e) < 1e-12 * e * g2


def test_newton_root_matches_bracketed_solver():
    from scipy.optimize import brentq
    tab = I.eos_table()
    o = O.Oracle(4, eos=tab)
    for _ in range(100):
        e, v = random_prim(0.95)
        U = o.prim2cons(e, v)
        E, M = U[0], np.linalg.norm(U[1:])
        root = brentq(lambda w: w - M / (E + o.eos_p(E - M * w)), 0.0, M / E, xtol=1e-16,
                      rtol=1e-15)
        assert abs(np.linalg.norm(o.cons2prim(U)[1]) - root) < 1e-14


# ------------------------------------------------------------------- MLP
def test_mlp_gradient_matches_finite_differences():
    n = O.mlp_nparam()
    P = RNG.normal(size=n) * 0.3
    P[-4:] = [0.5, 2.0, 0.4, 0.3]
    X = np.column_stack([RNG.uniform(-5, 5, 40), RNG.uniform(0, 0.99, 40)])
    Y = RNG.uniform(0, 0.9, 40)
    loss, G = O.mlp_loss_grad(P, X, Y)
    for idx in list(RNG.choice(n - 4, 60, replace=False)):
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[idx] += h
        Pm[idx] -= h
        fd = (O.mlp_loss_grad(Pp, X, Y)[0] - O.mlp_loss_grad(Pm, X, Y)[0]) / (2 * h)
        assert abs(fd - G[idx]) <= 1e-6 * max(1e-4, abs(G).max())
    assert not G[-4:].any()


def _mlp_pack(W1, b1, W2, b2, W3, b3, nrm):
    """Parameters in the network's layout: W1[32][2] b1 W2[32][32] b2 W3 b3 mu0 s0 mu1 s1."""
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3], nrm])


def _conformal_root(x):
    """|v| of the p = e/3 state with |M|/E = x: for that EOS x = 4v / (3 + v^2),
    so v is the root in [0, 1] of x v^2 - 4 v + 3 x = 0 (library polynomial roots)."""
    out = []
    for xi in x:
        r = np.roots([xi, -4.0, 3.0 * xi]) if xi > 0 else np.array([0.0])
        out.append(min(float(np.real(t)) for t in r if -1e-12 <= np.real(t) <= 1.0 + 1e-12))
    return np.array(out)


def test_mlp_forward_reduces_to_matrix_products():
    """The Newton seed network's forward pass (FP64, unquantised) pinned to
    special cases that a matrix product gives: with the weights of layers 1
    and 2 zero it is v0 = vc + (x - vc) sigmoid(W3 . tanh(b2) + b3) exactly;
    with zero biases and layer-1 and layer-2 weights scaled by 1e-3, tanh and
    the sigmoid linearise and 4 (v0 - (vc + x) / 2) / (x - vc) = 1e-6 W3 . (B (A s))
    to a relative O(1e-6), s the standardised inputs; with layer 1 zero, the
    same with tanh(b1) for A s.  vc, the closed-form p = e/3 root, comes from
    the polynomial its defining relation gives.  A transposed weight matrix,
    a wrong parameter offset, a dropped bias or a wrong standardisation fails
    one of them."""
    H = 32
    rng = np.random.default_rng(41)
    nrm = np.array([0.7, 2.5, 0.45, 0.3])
    n = 64
    X = np.column_stack([rng.uniform(-6, 6, n), rng.uniform(0.2, 0.95, n)])
    x = X[:, 1]
    s = np.column_stack([(X[:, 0] - nrm[0]) / nrm[1], (x - nrm[2]) / nrm[3]])
    vc = _conformal_root(x)
    np.testing.assert_allclose(4 * vc / (3 + vc * vc), x, rtol=1e-14)
    b1, b2, W3 = rng.normal(size=H), rng.normal(size=H), rng.normal(size=H)
    A, B = rng.normal(size=(H, 2)), rng.normal(size=(H, H))
    # layers 1 and 2 without weights: exact
    b3 = 0.37
    P = _mlp_pack(np.zeros((H, 2)), b1, np.zeros((H, H)), b2, W3, b3, nrm)
    z = W3 @ np.tanh(b2) + b3
    want = vc + (x - vc) / (1.0 + np.exp(-z))
    np.testing.assert_allclose(O.mlp_forward(P, X), want, rtol=1e-13, atol=1e-15)
    # zero biases, small weights: the linearised product W3 B A s
    eps = 1e-3
    P = _mlp_pack(eps * A, np.zeros(H), eps * B, np.zeros(H), W3, 0.0, nrm)
    zl = eps * eps * (s @ A.T @ B.T @ W3)
    got = 4.0 * (O.mlp_forward(P, X) - 0.5 * (vc + x)) / (x - vc)
    np.testing.assert_allclose(got, zl, rtol=1e-4, atol=1e-12)
    # layer 1 without weights: its output tanh(b1) through the linearised rest
    P = _mlp_pack(np.zeros((H, 2)), b1, eps * B, np.zeros(H), W3, 0.0, nrm)
    zb = eps * (W3 @ (B @ np.tanh(b1)))
    got = 4.0 * (O.mlp_forward(P, X) - 0.5 * (vc + x)) / (x - vc)
    np.testing.assert_allclose(got, np.full(n, zb), rtol=1e-4)


def test_round_bf16_matches_library_conversion():
    import torch
    x = RNG.normal(size=2000) * 10.0 ** RNG.uniform(-10, 10, size=2000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.round_bf16(v) for v in x])
    assert np.array_equal(got, want)


# --------------------------------------------------------------- jet source
def test_jet_source_deposits_dedx_per_unit_time():
    n, dx = 48, 0.1
    lo = -0.5 * n * dx
    jet = np.array([0.3, -0.2, 0.1, 0.6, 0.8, 0.0, 5.0, 0.3])
    o = O.Oracle(n, n, n, dx=dx, x0=lo, y0=lo, z0=lo, jet=jet)
    U = np.zeros(o.shape)
    U[0] = 1.0
    s0 = o.conservation_sums(U)
    o.jet_source(U, 0.5, 0.02)
    ds = o.conservation_sums(U) - s0
    want = 0.02 * 5.0
    # the Gaussian's tail beyond the box edge (6 sigma away) is ~1e-9 of its mass
    assert abs(ds[0] - want) < 1e-8 * want
    np.testing.assert_allclose(ds[1:], want * jet[3:6], atol=1e-8 * want)


def test_jet_source_profile_moves_with_the_jet_and_has_width_sigma():
    """R12 beyond the integrals: the deposited energy is a Gaussian centred on
    x0 + n t (the jet has moved along n for the time t) with variance sigma^2
    per axis, and the momentum deposit is n times the energy deposit cell by
    cell.  Sampled on cells of dx = sigma / 3 a Gaussian's first and second
    moments are exact to far below the tolerances (Poisson summation), so a
    wrong direction or sign of the motion, a wrong width or a mixed-up axis
    fails here."""
    n, dx = 64, 0.1
    lo = -0.5 * n * dx
    sig = 0.3
    jet = np.array([0.3, -0.2, 0.1, 0.6, 0.0, -0.8, 5.0, sig])
    o = O.Oracle(n, n, n, dx=dx, x0=lo, y0=lo, z0=lo, jet=jet)
    U = np.zeros(o.shape)
    t, dt = 0.75, 0.02
    o.jet_source(U, t, dt)
    c = lo + (np.arange(n) + 0.5) * dx
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    w = U[0]
    mass = w.sum()
    centre = np.array([jet[0], jet[1], jet[2]]) + t * jet[3:6]
    got = np.array([(xx * w).sum(), (yy * w).sum(), (zz * w).sum()]) / mass
    np.testing.assert_allclose(got, centre, atol=1e-9)
    for a, x in zip(range(3), (xx, yy, zz)):
        var = ((x - centre[a]) ** 2 * w).sum() / mass
        assert abs(var - sig * sig) < 1e-8, (a, var)
    for k in range(3):
        np.testing.assert_allclose(U[1 + k], jet[3 + k] * U[0], rtol=0, atol=1e-15)
    # the peak deposit: dt dE/dx over (2 pi)^(3/2) sigma^3 at the centre, here
    # off the cell centres, so the largest cell value lies below it
    peak = dt * jet[6] / ((2 * np.pi) ** 1.5 * sig ** 3)
    assert w.max() < peak and w.max() > 0.8 * peak


# ----------------------------------------------- unsplit multi-D scheme (R16)
def test_unsplit_on_a_line_equals_the_1d_sweep():
    """With one active axis the unsplit scheme (Eq. 13 with only the F term)
    is the 1-D MUSCL-Hancock MUSTA-FORCE step: same faces, fluxes, RK stages
    and CFL dt (sum over one axis = max over one axis)."""
    for rk in (1, 2, 3):
        g, prim = I.shock_tube(200)
        kw = dict(dx=g["dx"], x0=-1.0, bc="outflow", alpha=3.0, rk_order=rk, cfl=0.4)
        a, b = O.Oracle(200, **kw), O.Oracle(200, unsplit=1, **kw)
        Ua = a.prim2cons_field(*prim)
        Ub = Ua.copy()
        a.run(Ua, 40)
        b.run(Ub, 40)
        assert np.array_equal(Ua, Ub), rk


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_unsplit_plane_wave_equals_1d_unsplit(axis):
    """Data varying along one axis only of a 3-D grid: the transverse half-step
    terms vanish (zero slopes give equal faces) and so do the transverse flux
    differences, so every line equals the 1-D unsplit run."""
    n = 48
    g, prim = I.shock_tube(n)
    dt = 0.1 * g["dx"]
    ref = O.Oracle(n, dx=g["dx"], x0=-1.0, bc="outflow", alpha=3.0, unsplit=1, fixed_dt=dt)
    U1 = ref.prim2cons_field(*prim)
    ref.run(U1, 12)
    shape = [5, 5, 5]
    shape[2 - axis] = n
    bc = ["periodic"] * 3
    bc[axis] = "outflow"
    o = O.Oracle(shape[2], shape[1], shape[0], dx=g["dx"], bc=tuple(bc), alpha=3.0, unsplit=1,
                 fixed_dt=dt)
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    e = np.broadcast_to(prim[0].ravel()[tuple(sl)], shape).copy()
    z = np.zeros(shape)
    U3 = o.prim2cons_field(e, z, z, z)
    o.run(U3, 12)
    line = [slice(None), 2, 2, 2]
    line[1 + (2 - axis)] = slice(None)
    got = U3[tuple(line)]
    assert np.array_equal(got[0], U1[0].ravel())
    assert np.array_equal(got[1 + axis], U1[1].ravel())
    others = [q for q in (1, 2, 3) if q != 1 + axis]
    assert not got[others].any()


def unsplit_blast(n, steps, limiter="minmod"):
    g, prim = I.spherical_blast(n)
    o = O.Oracle(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic",
                 limiter=limiter, cfl=0.4, alpha=3.0, unsplit=1)
    U = o.prim2cons_field(*prim)
    s0 = o.conservation_sums(U)
    o.run(U, steps)
    return o, U, s0


def test_unsplit_blast_conserves_and_is_symmetric():
    """Periodic flux form conserves E and M to roundoff; the blast stays
    symmetric under each reflection (M_d odd) and under exchange of two axes
    (the scheme treats the axes alike; only the order of the axis sums differs)."""
    o, U, s0 = unsplit_blast(16, 6)
    s1 = o.conservation_sums(U)
    assert abs(s1[0] - s0[0]) <= 1e-13 * s0[0]
    assert np.abs(s1[1:]).max() <= 1e-13 * s0[0]
    scale = U[0].max()
    for ax in range(3):
        R = np.flip(U, axis=3 - ax).copy()
        R[1 + ax] *= -1.0
        assert np.abs(R - U).max() <= 1e-14 * scale
    # exchange x and y: array axes 3 and 2, momentum components 1 and 2
    T = np.swapaxes(U, 2, 3)[[0, 2, 1, 3]]
    assert np.abs(T - U).max() <= 1e-13 * scale


def test_unsplit_and_strang_agree_on_the_blast():
    """Two consistent discretisations of the same flow: after the same physical
    time their energy densities differ by discretisation error only (small
    against the blast's jump of 9), and both keep E positive."""
    n = 24
    g, prim = I.spherical_blast(n)
    kw = dict(dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic", cfl=0.4)
    a = O.Oracle(n, n, n, **kw)
    b = O.Oracle(n, n, n, alpha=3.0, unsplit=1, **kw)
    Ua = a.prim2cons_field(*prim)
    Ub = Ua.copy()
    _, ta = a.run(Ua, 10)
    _, tb = b.run(Ub, 200, t_end=ta)
    assert tb == ta
    assert Ua[0].min() > 0 and Ub[0].min() > 0
    assert np.abs(Ua[0] - Ub[0]).mean() <= 0.05 * np.abs(Ua[0] - 1.0).mean() + 0.02


def test_unsplit_cfl_rate_sums_the_axes():
    """R16c: the rate is the sum over active axes of speed/dx; at rest with
    c_s^2 = 1/3 each axis contributes c_s/dx."""
    n = 8
    o = O.Oracle(n, n, n, dx=0.25, unsplit=1)
    U = o.prim2cons_field(np.ones((n, n, n)), *[np.zeros((n, n, n))] * 3)
    assert o.max_rate(U) == pytest.approx(3 * math.sqrt(1 / 3) / 0.25, rel=1e-14)
    o2 = O.Oracle(n, n, n, dx=0.25)
    assert o2.max_rate(U) == pytest.approx(math.sqrt(1 / 3) / 0.25, rel=1e-14)


@pytest.mark.slow
def test_unsplit_hubble_expansion_interior_converges():
    """The unsplit scheme (alpha = 3) on the same 3-D Hubble flow: the core
    follows the exact solution and the error falls under refinement at a fixed
    Courant number small enough for the unsplit stability limit."""
    e1, v1 = hubble_error(32, 0.1, 0.02, 15, alpha=3.0, unsplit=1)
    e2, v2 = hubble_error(64, 0.05, 0.01, 30, alpha=3.0, unsplit=1)
    assert e1 < 0.04 and v1 < 0.01
    assert e2 < e1 / 2 and v2 < v1 / 2


# ------------------------------------------- the paper's ellipsoidal flow (R17)
def ellipsoidal_1d_error(n, t0=2.0, t1=2.4, half=3.0):
    """The ellipsoidal flow of Sec. 3.2 along one axis (pressureless, c_s^2 = 0,
    vacuum outside |v| < 1) from t0 to t1; relative L1 error of e in |x| < 1.2."""
    dx = 2 * half / n
    x = I.cell_centres(n, -half, dx)
    e, (v,) = exact.ellipsoidal([x], t0)
    dt = 0.2 * dx
    steps = int(round((t1 - t0) / dt))
    o = O.Oracle(n, dx=dx, x0=-half, bc="outflow", cs2=0.0, fixed_dt=dt)
    z = np.zeros((1, 1, n))
    U = o.prim2cons_field(e.reshape(1, 1, n), v.reshape(1, 1, n), z, z)
    o.run(U, steps)
    en = o.cons2prim_field(U)[0].ravel()
    ex, _ = exact.ellipsoidal([x], t0 + steps * dt)
    core = np.abs(x) < 1.2
    return np.abs(en[core] - ex[core]).sum() / ex[core].sum()


def test_ellipsoidal_flow_1d_converges_to_the_exact_dust_solution():
    """p = 0 (the conformal EOS with c_s^2 = 0) keeps the exact ballistic
    expansion: the error is small and falls under refinement."""
    e1 = ellipsoidal_1d_error(120)
    e2 = ellipsoidal_1d_error(240)
    assert e1 < 2e-3
    assert e2 < e1 / 1.8


# ----------------------------------------------- op counting and timing builds
def test_op_count_of_a_sweep_follows_the_method_structure():
    """The op-counting build counts one square root and one division per flux
    evaluation of the p = c^2 e cons->prim (W from the quadratic, v_d = M_d/W),
    and a sweep makes 2 Hancock + 3k MUSTA-FORCE evaluations per cell and RK
    stage (Sec. 2.4): rk (2 + 3k) of each.  RK3's combination adds the
    division U/3 per field."""
    for stages, rk in ((1, 2), (2, 2), (3, 2), (2, 1), (4, 3)):
        d = O.opcount_sweep("minmod", stages, rk)
        evals = rk * (2 + 3 * stages)
        assert d["sqrt"] == evals, (stages, rk, d)
        assert d["div"] == evals + (4 if rk == 3 else 0), (stages, rk, d)
        # Minbee: one min per field and RK stage; no transcendental anywhere
        assert d["min"] == 4 * rk and d["max"] == 0
        assert d["exp"] == d["log"] == d["tanh"] == 0


def test_op_counts_pin_the_benchmark_flops():
    """The algorithmic flops the benchmark reports are the op-counting build's."""
    import bench
    for (lim, stages, rk), flops in bench.FLOPS_PER_CELL_SWEEP.items():
        assert O.opcount_sweep(lim, stages, rk)["flops"] == flops, (lim, stages, rk)
    for (stages, rk), flops in bench.FLOPS_PER_CELL_STAGE_UNSPLIT.items():
        assert O.opcount_unsplit(stages, rk)["flops"] == flops
        # uniform per cell: the same count on a larger periodic grid
        assert O.opcount_unsplit(stages, rk, n=10)["flops"] == flops


def test_openmp_timing_build_equals_the_oracle_bit_for_bit():
    g, prim = I.spherical_blast(20)
    o = O.Oracle(20, 20, 20, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic")
    U1 = o.prim2cons_field(*prim)
    U2 = U1.copy()
    o.run(U1, 2)
    o.run(U2, 2, threads=True)
    assert np.array_equal(U1, U2)


# ------------------------------------------------------------ conserved charge
def test_charge_flux_and_prim2cons_follow_eq_3_and_4():
    """R = n gamma (Eq. 4) and its flux R v_d (Eq. 3); the energy-momentum
    components are those of the four-field scheme."""
    o5 = O.Oracle(1, charge=1)
    o4 = O.Oracle(1)
    v = np.array([0.3, -0.4, 0.2])
    U5 = o5.prim2cons(2.0, v, n=0.7)
    g = 1.0 / math.sqrt(1.0 - v @ v)
    assert U5[4] == pytest.approx(0.7 * g, rel=1e-15)
    assert np.array_equal(U5[:4], o4.prim2cons(2.0, v))
    for d in range(3):
        F5 = o5.flux(d, U5)
        assert np.array_equal(F5[:4], o4.flux(d, U5[:4]))
        assert F5[4] == pytest.approx(U5[4] * v[d], rel=1e-14)


def charged_shock_tube(n, n_l=1.0, n_r=0.5):
    g, prim = I.shock_tube(n)
    o = O.Oracle(n, dx=g["dx"], x0=-1.0, bc="outflow", limiter="minmod", cfl=0.4, charge=1)
    x = I.cell_centres(n, -1.0, g["dx"])
    nn = np.where(x < 0.0, n_l, n_r).reshape(1, 1, n)
    U = o.prim2cons_field(*prim, n=nn)
    o.run(U, 100000, t_end=0.8)
    got = o.charge_density_field(U).ravel()
    want = exact.Riemann().sample_n(x, 0.8, n_l, n_r)
    return np.abs(got - want).sum() / np.abs(want).sum(), U


def test_charged_shock_tube_converges_to_the_exact_charge_density():
    """e_L = 10, e_R = 1, p = e/3 with n_L = 1, n_R = 0.5: the exact n has a
    rarefaction fan, a contact moving with v*, and the shock's compression.
    The energy-momentum fields are those of the four-field run bit for bit."""
    errs = [charged_shock_tube(n)[0] for n in (250, 500, 1000)]
    assert errs[0] < 0.05
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert errs[0] / errs[2] > 2.0      # at least half order through the contact
    _, U5 = charged_shock_tube(250)
    g, prim = I.shock_tube(250)
    o4 = O.Oracle(250, dx=g["dx"], x0=-1.0, bc="outflow", limiter="minmod", cfl=0.4)
    U4 = o4.prim2cons_field(*prim)
    o4.run(U4, 100000, t_end=0.8)
    assert np.array_equal(U5[:4], U4)


def test_charge_is_conserved_on_a_periodic_blast():
    n = 16
    g, prim = I.spherical_blast(n)
    c = I.cell_centres(n, -1.0, g["dx"])
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    nn = 1.0 + 0.5 * np.cos(np.pi * xx) * np.sin(np.pi * yy)
    o = O.Oracle(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic", charge=1)
    U = o.prim2cons_field(*prim, n=nn)
    s0 = o.conservation_sums(U)
    o.run(U, 4)
    s1 = o.conservation_sums(U)
    assert abs(s1[4] - s0[4]) <= 1e-13 * abs(s0[4])
    assert abs(s1[0] - s0[0]) <= 1e-13 * abs(s0[0])


def ellipsoidal_charge_error(n, t0=2.0, t1=2.4, half=3.0):
    """The ellipsoidal flow of Sec. 3.2 along one axis with its charge density
    n = C_n / prod(t + T_i) exp(-b_n^2 t^2/tau^2) (C_n = 0.75, b_n = 1):
    relative L1 error of n in |x| < 1.2."""
    dx = 2 * half / n
    x = I.cell_centres(n, -half, dx)
    e, (v,) = exact.ellipsoidal([x], t0)
    nn, _ = exact.ellipsoidal([x], t0, C=0.75, b=1.0)
    dt = 0.2 * dx
    steps = int(round((t1 - t0) / dt))
    o = O.Oracle(n, dx=dx, x0=-half, bc="outflow", cs2=0.0, fixed_dt=dt, charge=1)
    z = np.zeros((1, 1, n))
    U = o.prim2cons_field(e.reshape(1, 1, n), v.reshape(1, 1, n), z, z, n=nn.reshape(1, 1, n))
    o.run(U, steps)
    got = o.charge_density_field(U).ravel()
    want, _ = exact.ellipsoidal([x], t0 + steps * dt, C=0.75, b=1.0)
    core = np.abs(x) < 1.2
    return np.abs(got[core] - want[core]).sum() / want[core].sum()


def test_ellipsoidal_charge_density_converges_to_the_exact_solution():
    """The paper's third test carries n with the flow; the charge field
    follows its exact solution and the error falls under refinement."""
    e1 = ellipsoidal_charge_error(120)
    e2 = ellipsoidal_charge_error(240)
    assert e1 < 2e-3
    assert e2 < e1 / 1.8
