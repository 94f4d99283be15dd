"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (reading R13): FP64 <= 1e-10 max relative per cell; FP32 and
mixed <= 1e-4 relative L1 per field.  Sizes are small enough for the oracle
and span several blocks, several pencil segments and ragged tails.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_06340_b300 import inputs as I
from tests import exact
from tests.metrics import max_rel_per_cell, rel_l1

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
F32_TOL = 1e-4


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1510_06340_b300 import build, hydro
    build.build(verbose=False)
    return hydro


def pair(H, g, prim, prec="fp64", bc="periodic", limiter="minmod", stages=2, rk_order=2,
         hancock=1, cfl=0.4, fixed_dt=0.0, eos=None, seed="zero", jet=None, newton_tol=0.0):
    """A GPU handle and an oracle on the same grid and initial state."""
    grid = H.make_grid(g["nx"], g.get("ny", 1), g.get("nz", 1), dx=g["dx"], x0=g.get("x0", 0.0),
                       y0=g.get("y0", 0.0), z0=g.get("z0", 0.0), bc=bc, prec=prec,
                       rk_order=rk_order, hancock=hancock, cfl=cfl, fixed_dt=fixed_dt)
    h = H.Hydro(grid, H.make_eos(eos, seed=seed, newton_tol=newton_tol), limiter=limiter,
                stages=stages)
    o = O.Oracle(g["nx"], g.get("ny", 1), g.get("nz", 1), dx=g["dx"], x0=g.get("x0", 0.0),
                 y0=g.get("y0", 0.0), z0=g.get("z0", 0.0), bc=bc, limiter=limiter,
                 stages=stages, rk_order=rk_order, hancock=hancock, cfl=cfl, fixed_dt=fixed_dt,
                 eos=eos, seed_kind=H.SEEDS[seed], jet=jet)
    U0 = o.prim2cons_field(*prim)
    h.set_conserved(U0.astype(h.dtype))
    if jet is not None:
        h.set_jet(jet)
    return h, o, U0


def check(h, U_ref, prec):
    U = h.get_conserved()
    if prec == "fp64":
        err = max_rel_per_cell(U, U_ref)
        assert err <= F64_TOL, err
    else:
        err = max(rel_l1(U, U_ref))
        assert err <= F32_TOL, err
    return err


# ------------------------------------------------------------------ 1-D shock tube
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shock_tube_to_t08(H, prec):
    """1000 cells, e_L = 10, e_R = 1, outflow, CFL 0.4, minmod, 2 stages, RK2, t = 0.8."""
    g, prim = I.shock_tube(1000)
    h, o, U = pair(H, g, prim, prec=prec, bc="outflow")
    n_or, t_or = o.run(U, 100000, t_end=0.8)
    t = h.step(100000, t_end=0.8)
    assert t == 0.8 and t_or == 0.8
    check(h, U, prec)
    # and the GPU solution is close to the exact one
    e, vx, _, _ = h.get_primitives()
    x = I.cell_centres(1000, -1.0, g["dx"])
    ex, _ = exact.Riemann().sample(x, 0.8)
    assert np.abs(e.ravel() - ex).sum() / np.abs(ex).sum() < 6e-3


@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "superbee", "vanleer", "vanalbada"])
@pytest.mark.parametrize("rk_order,hancock,stages", [(2, 1, 2), (1, 1, 3), (3, 0, 1), (3, 1, 4)])
def test_scheme_variants_1d(H, limiter, rk_order, hancock, stages):
    n = 203   # ragged against every segment length
    rng = np.random.default_rng(7)
    x = I.cell_centres(n, -1.0, 2.0 / n)
    e = 1.0 + 0.5 * np.sin(3 * np.pi * x) + (x > 0.3) * 2.0 + 0.05 * rng.random(n)
    v = 0.3 * np.cos(2 * np.pi * x) * (np.abs(x) < 0.7)
    z = np.zeros(n)
    prim = tuple(a.reshape(1, 1, n) for a in (e, v, 0.2 * v, z))
    g = dict(nx=n, dx=2.0 / n, x0=-1.0)
    for bc in ("periodic", "outflow"):
        h, o, U = pair(H, g, prim, bc=bc, limiter=limiter, stages=stages, rk_order=rk_order,
                       hancock=hancock, fixed_dt=0.3 * 2.0 / n)
        for segs in (1, 4):
            h.force_launch(0, 64, segs)
            h.set_conserved(U)
            h.set_time(0.0)
            h.step(12)
            Uo = U.copy()
            o.run(Uo, 12)
            check(h, Uo, "fp64")


# ------------------------------------------------------------------ 3-D blast
@pytest.mark.parametrize("limiter", ["minmod", "mc", "superbee"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blast_3d(H, limiter, prec):
    g, prim = I.spherical_blast(32)
    h, o, U = pair(H, g, prim, prec=prec, limiter=limiter)
    o.run(U, 10)
    h.step(10)
    check(h, U, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cap_acts_in_the_specialised_sweeps(H, prec):
    """Cells set with |M| > E (not admissible, R9): their faces fall back to
    the cell average and the fluxes of those states take the |M| cap.  The
    specialised kernels evaluate a group of fluxes without the cap and redo
    the group where a state exceeded it; the result must be the oracle's.  A
    second run with counters (the runtime-limiter kernels, which cap in every
    evaluation) confirms that the cap acted."""
    n = 24
    g = dict(nx=n, ny=n, nz=n, dx=2.0 / n, x0=-1.0, y0=-1.0, z0=-1.0)
    c = I.cell_centres(n, -1.0, g["dx"])
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    e = 1.0 + 0.5 * np.exp(-8.0 * (xx * xx + yy * yy + zz * zz))
    prim = (e, 0.3 * np.sin(np.pi * yy), 0.2 * np.cos(np.pi * xx), 0.1 * np.sin(np.pi * zz))
    delta = 1e-12 if prec == "fp64" else 1e-6
    h, o, U = pair(H, g, prim, prec=prec, fixed_dt=0.25 * g["dx"])
    o = O.Oracle(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, fixed_dt=0.25 * g["dx"],
                 delta=delta)
    rng = np.random.default_rng(5)
    idx = rng.choice(n ** 3, 40, replace=False)
    Uf = U.reshape(4, -1)
    for i in idx:   # |M| = 1.2 E along a random direction
        d = rng.normal(size=3)
        Uf[1:, i] = 1.2 * Uf[0, i] * d / np.linalg.norm(d)
    h.set_conserved(U.astype(h.dtype))
    U0 = U.copy()
    o.run(U, 3)
    h.step(3)
    check(h, U, prec)
    hc = H.Hydro(H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec=prec,
                             fixed_dt=0.25 * g["dx"]))
    hc.enable_counters(True)
    hc.set_conserved(U0.astype(hc.dtype))
    hc.step(3)
    assert hc.counters()["capped"] > 0
    a, b = hc.get_conserved().astype(np.float64), h.get_conserved().astype(np.float64)
    if prec == "fp64":
        assert max_rel_per_cell(a, b) <= 1e-13
    else:
        assert max(rel_l1(a, b)) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["outflow", "periodic"])
def test_blob_in_vacuum_through_the_specialised_sweeps(H, prec, bc):
    """A moving blob in exact vacuum (E = M = 0 outside) through the RK2 Minbee
    sweeps with the CFL step: every group of flux evaluations that meets a
    vacuum state is redone with the guarded cons->prim, and the result must
    be the oracle's, dt included."""
    n = 16
    dx = 0.25
    lo = -0.5 * n * dx
    g = dict(nx=n, ny=n, nz=n, dx=dx, x0=lo, y0=lo, z0=lo)
    spots = np.array([[0.3, -0.2, 0.1, 2.0, 0.6, 0.3, -0.2]])
    e, vx, vy, vz = I.hotspot_primitives(g, spots, sigma=0.5, e_bg=0.0)
    inside = e > 1e-3 * e.max()
    prim = [np.where(inside, a, 0.0) for a in (e, vx, vy, vz)]
    assert not inside.all()
    h, o, U = pair(H, g, prim, prec=prec, bc=bc, cfl=0.3)
    _, t = o.run(U, 4)
    h.step(4)
    assert h.time() == pytest.approx(t, rel=1e-12 if prec == "fp64" else 1e-6)
    check(h, U, prec)


def test_blast_3d_ragged_shapes_bitwise(H):
    """Launch shape (threads per block, pencil segments) changes no bit."""
    g = dict(nx=37, ny=29, nz=23, dx=2.0 / 37, x0=-1.0, y0=-0.8, z0=-0.6)
    c = [I.cell_centres(g[k], g[o], g["dx"]) for k, o in (("nz", "z0"), ("ny", "y0"), ("nx", "x0"))]
    zz, yy, xx = np.meshgrid(*c, indexing="ij")
    e = np.where(xx ** 2 + yy ** 2 + zz ** 2 < 0.3, 8.0, 1.0)
    zero = np.zeros_like(e)
    prim = (e, 0.1 * np.sin(3 * yy), zero, 0.05 * np.cos(2 * xx))
    ref = None
    for threads, segs in ((256, 1), (64, 3), (96, 5), (32, 2)):
        h, o, U = pair(H, g, prim, bc=("periodic", "outflow", "periodic"))
        for ax in range(3):
            h.force_launch(ax, threads, segs)
        h.step(4)
        out = h.get_conserved()
        if ref is None:
            ref = out
            o.run(U, 4)
            assert max_rel_per_cell(out, U) <= F64_TOL
        else:
            assert np.array_equal(out, ref), (threads, segs)


@pytest.mark.parametrize("dims", [1, 3])
def test_graph_and_eager_steps_agree_bitwise(H, dims):
    """Steps replayed from CUDA graphs equal single steps bit for bit, also
    when calls with odd step counts alternate the starting state buffer."""
    if dims == 3:
        g, prim = I.spherical_blast(24)
    else:
        g, prim = I.shock_tube(300)
    h1, _, U = pair(H, g, prim, bc="outflow")
    for _ in range(9):
        h1.step(1)   # single steps (no graph)
    h2, _, _ = pair(H, g, prim, bc="outflow")
    for n in (3, 2, 4):
        h2.step(n)   # graph launches of two steps plus odd single steps
    assert np.array_equal(h1.get_conserved(), h2.get_conserved())
    h3, _, _ = pair(H, g, prim, bc="outflow")
    h3.step(9, t_end=10.0)   # chunked stepping with a (distant) end time
    assert np.array_equal(h1.get_conserved(), h3.get_conserved())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_conservation(H, prec):
    g, prim = I.spherical_blast(32)
    h, o, U = pair(H, g, prim, prec=prec)
    s0 = h.conservation_sums()
    np.testing.assert_allclose(s0, o.conservation_sums(U.astype(h.dtype).astype(np.float64)),
                               rtol=1e-12, atol=1e-12 * s0[0])
    h.step(20)
    s1 = h.conservation_sums()
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert abs(s1[0] - s0[0]) <= tol * s0[0]
    assert np.abs(s1[1:]).max() <= tol * s0[0]


def test_cfl_rate_matches_oracle(H):
    g = I.event_grid(20, 0.1)
    spots = I.hotspots(3, flow_max=0.9)
    prim = I.hotspot_primitives(g, spots)
    h, o, U = pair(H, g, prim, bc="outflow")
    r = h.max_rate()
    assert abs(r - o.max_rate(U)) <= 1e-14 * r


# ------------------------------------------------------------------ outflow + flow + jet
@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_hotspots_with_flow_and_jet(H, prec):
    g = I.event_grid(24, 0.1)
    spots = I.hotspots(11, flow_max=0.95)
    prim = I.hotspot_primitives(g, spots)
    jet = I.jet(11)
    jet[:3] = [0.2, -0.3, 0.0]    # start inside this small box
    h, o, U = pair(H, g, prim, prec=prec, bc="outflow", jet=jet)
    o.run(U, 8)
    h.step(8)
    check(h, U, prec)


def test_hotspot_initial_state_matches_generator(H):
    g = I.event_grid(18, 0.1)
    spots = I.hotspots(5, flow_max=0.9)
    e, vx, vy, vz = I.hotspot_primitives(g, spots)
    grid = H.make_grid(18, 18, 18, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow")
    h = H.Hydro(grid)
    h.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    eg, vxg, vyg, vzg = h.get_primitives()
    np.testing.assert_allclose(eg, e, rtol=1e-12)
    for a, b in ((vxg, vx), (vyg, vy), (vzg, vz)):
        np.testing.assert_allclose(a, b, atol=1e-12)


# ------------------------------------------------------------------ full-size sweeps, sampled
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_size_blast_sweeps_sampled(H, prec):
    """256^3 blast in the benchmark's launch configuration: after two steps,
    one sweep per axis on the GPU; sampled pencils recomputed one by one by
    the oracle from the same input state."""
    n = 256
    g, prim = I.spherical_blast(n)
    grid = H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec=prec)
    h = H.Hydro(grid)
    h.set_primitives(*[a.astype(h.dtype) for a in prim])
    h.step(2)
    rng = np.random.default_rng(3)
    dt = 0.4 * g["dx"] * 0.5
    for axis in range(3):
        U_in = h.get_conserved()
        h.sweep(axis, dt)
        U_out = h.get_conserved()
        for _ in range(12):
            a, b = rng.integers(0, n, size=2)
            idx = [a, b]
            idx.insert(2 - axis, slice(None))
            pen = U_in[(slice(None),) + tuple(idx)].astype(np.float64)   # [4][n]
            shape = [1, 1, 1]
            shape[axis] = n
            o = O.Oracle(*shape, dx=g["dx"], bc="periodic")
            Up = pen.reshape((4,) + tuple(shape[::-1])).copy()
            o.sweep(Up, axis, dt)
            got = U_out[(slice(None),) + tuple(idx)]
            if prec == "fp64":
                assert max_rel_per_cell(got, Up.reshape(4, n)) <= F64_TOL
            else:
                assert max(rel_l1(got, Up.reshape(4, n))) <= F32_TOL


# ------------------------------------------------------------------ batch
def test_batch_equals_single_runs_bitwise(H):
    sizes = [17, 24, 31, 20]
    grids, prims = [], []
    for k, n in enumerate(sizes):
        g = I.event_grid(n, 0.1)
        grids.append(H.make_grid(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                                 bc="outflow", prec="fp32"))
        prims.append(I.hotspot_primitives(g, I.hotspots(k, nspots=40)))
    b = H.Batch(grids)
    for k, p in enumerate(prims):
        b.set_primitives(k, *[a.astype(np.float32) for a in p])
    b.step(6)
    times = b.times()
    for k, p in enumerate(prims):
        h = H.Hydro(grids[k])
        h.set_primitives(*[a.astype(np.float32) for a in p])
        h.step(6)
        assert h.time() == times[k]
        assert np.array_equal(h.get_conserved(), b.get_conserved(k)), k


def test_batch_hotspots_jets_against_oracle(H):
    sizes = [16, 22, 19]
    grids, jets, spots = [], [], []
    for k, n in enumerate(sizes):
        g = I.event_grid(n, 0.1)
        grids.append(H.make_grid(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                                 bc="outflow", prec="fp64"))
        j = I.jet(k)
        j[:3] = [0.1 * k, -0.2, 0.0]
        jets.append(j)
        spots.append(I.hotspots(k, nspots=64))
    b = H.Batch(grids)
    b.init_hotspots(np.stack(spots), I.SPOT_SIGMA, I.E_BACKGROUND)
    b.set_jets(np.stack(jets))
    b.step(5)
    for k, n in enumerate(sizes):
        g = I.event_grid(n, 0.1)
        o = O.Oracle(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow",
                     jet=jets[k])
        U = o.prim2cons_field(*I.hotspot_primitives(g, spots[k]))
        o.run(U, 5)
        assert max_rel_per_cell(b.get_conserved(k), U) <= F64_TOL


# ------------------------------------------------------------------ tabulated EOS
@pytest.mark.parametrize("seed", ["zero", "conformal"])
def test_table_eos_fp64(H, seed):
    tab = I.eos_table()
    g = I.event_grid(16, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(2, nspots=60, flow_max=0.8))
    h, o, U = pair(H, g, prim, bc="outflow", eos=tab, seed=seed)
    o.run(U, 4)
    h.step(4)
    check(h, U, "fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("max_iter", [0, 1])
def test_paired_newton_solves_equal_single_solves(H, prec, max_iter):
    """The tabulated-EOS sweeps run the cons->prim Newton solves of two flux
    evaluations in one loop; each state must get the |v|, p and iteration
    count of its own solve, bit for bit: both seeds, both reciprocal forms,
    states below, inside and above the table, at rest, at the |M| cap and in
    vacuum, with the default iteration cap and with a cap of one that leaves
    most solves unconverged. The single solves with divisions must also be
    those of hydro_c2p_newton."""
    import torch
    tab = I.eos_table()
    grid = H.make_grid(4, 4, 4, dx=0.1, prec=prec)
    h = H.Hydro(grid, H.make_eos(tab, newton_max_iter=max_iter))
    rng = np.random.default_rng(21)
    n = 4096
    E = np.exp(rng.uniform(np.log(1e-7), np.log(1e5), n))
    x = rng.uniform(0.0, 0.9999, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    E[:4] = [0.0, -1.0, 1e-30, 1e-12]
    x[8:24] = 0.0
    x[24:40] = 1.0
    U = np.stack([E, *(x * E * d)]).astype(h.dtype)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ut = torch.from_numpy(U).cuda()
    bits = torch.int64 if prec == "fp64" else torch.int32
    for seed in ("zero", "conformal"):
        for rcp in (0, 1):
            v = torch.zeros((2, n), dtype=dt, device="cuda")
            p = torch.zeros((2, n), dtype=dt, device="cuda")
            it = torch.zeros((2, n), dtype=torch.int32, device="cuda")
            h.c2p_newton_pairs(Ut, seed, rcp, v, p, it)
            assert torch.equal(v[0].view(bits), v[1].view(bits)), (seed, rcp)
            assert torch.equal(p[0].view(bits), p[1].view(bits)), (seed, rcp)
            assert torch.equal(it[0], it[1]), (seed, rcp)
            assert torch.isfinite(v).all() and torch.isfinite(p).all()
            if max_iter == 1:
                assert int((it[0] == 1).sum()) > n // 2
            if rcp == 0:
                vs = torch.zeros(n, dtype=dt, device="cuda")
                its = torch.zeros(n, dtype=torch.int32, device="cuda")
                h.c2p_newton(Ut, seed, vs, its)
                assert torch.equal(vs.view(bits), v[0].view(bits))
                assert torch.equal(its, it[0])


def test_table_eos_fp32(H):
    tab = I.eos_table()
    g = I.event_grid(16, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(2, nspots=60, flow_max=0.8))
    h, o, U = pair(H, g, prim, prec="fp32", bc="outflow", eos=tab)
    o.run(U, 4)
    h.step(4)
    check(h, U, "fp32")


def test_table_eos_mixed(H):
    """Mixed precision with the tabulated EOS: FP32 Newton, redone in FP64
    (seeded by the FP32 root) where |v| > 0.99."""
    tab = I.eos_table()
    g = I.event_grid(16, 0.1)
    # one fast spot (|u| = 0.999) on the background: cells near its centre
    # move with |v| > 0.99
    spots = np.array([[0.05, -0.05, 0.0, 2.0, 0.999, 0.0, 0.0]])
    prim = I.hotspot_primitives(g, spots)
    assert np.sqrt(sum(a * a for a in prim[1:])).max() > 0.99
    h, o, U = pair(H, g, prim, prec="mixed", bc="outflow", eos=tab, cfl=0.3)
    o.run(U, 4)
    h.step(4)
    check(h, U, "mixed")


def test_table_eos_fp32_generic_kernel(H):
    """The runtime-limiter table kernels: MC, RK3, four MUSTA stages."""
    tab = I.eos_table()
    g = I.event_grid(14, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(3, nspots=60, flow_max=0.6))
    h, o, U = pair(H, g, prim, prec="fp32", bc="outflow", eos=tab, limiter="mc",
                   rk_order=3, stages=4)
    o.run(U, 3)
    h.step(3)
    check(h, U, "fp32")


# ------------------------------------------------------------------ failure reporting
def test_nonfinite_state_is_reported(H):
    g, prim = I.spherical_blast(8)
    h, o, U = pair(H, g, prim)
    h.check_finite()
    U[0, 1, 2, 3] = np.nan
    h.set_conserved(U)
    with pytest.raises(H.HydroError) as ei:
        h.check_finite()
    assert ei.value.status == 6


def test_invalid_configurations_are_rejected(H):
    with pytest.raises(H.HydroError) as ei:
        H.Hydro(H.make_grid(0, 1, 1, dx=0.1))
    assert ei.value.status == 1
    with pytest.raises(H.HydroError):
        H.Hydro(H.make_grid(8, dx=0.1), limiter=9)
    with pytest.raises(H.HydroError):
        H.Hydro(H.make_grid(8, dx=0.1), stages=0)
    with pytest.raises(H.HydroError):
        H.Hydro(H.make_grid(8, dx=0.1, rk_order=4))
    # the largest grids: 536,870,911 cells (32-bit field offsets), 429,496,729
    # with the charge; refused before any state is allocated
    with pytest.raises(H.HydroError) as ei:
        H.Hydro(H.make_grid(1024, 1024, 513, dx=0.1))
    assert "536,870,911" in str(ei.value)
    with pytest.raises(H.HydroError) as ei:
        H.Hydro(H.make_grid(1024, 1024, 410, dx=0.1, charge=True))
    assert "429,496,729" in str(ei.value)
    # a non-positive cell size on an axis of more than one cell
    with pytest.raises(H.HydroError):
        H.Hydro(H.make_grid(8, 8, 1, dx=0.1, dy=0.0))


def test_empty_inputs_are_no_ops(H):
    """Zero samples for the network and the Newton hook launch nothing and
    succeed; a zero-step call leaves the state as it is."""
    import torch
    P = torch.zeros(H.mlp_nparam(), dtype=torch.float32, device="cuda")
    X = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros(0, dtype=torch.float32, device="cuda")
    H.mlp_forward(P, X, out)
    H.mlp_hidden(P, X, torch.zeros((0, 32), dtype=torch.float32, device="cuda"))
    h = H.Hydro(H.make_grid(8, dx=0.1), H.make_eos(I.eos_table()))
    U = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    h.c2p_newton(U, "zero", torch.zeros(0, dtype=torch.float64, device="cuda"),
                 torch.zeros(0, dtype=torch.int32, device="cuda"))
    g, prim = I.spherical_blast(8)
    hb, _, U0 = pair(H, g, prim)
    hb.step(0)
    assert np.array_equal(hb.get_conserved(), U0)


# ------------------------------------------------------------------ the paper's own settings
@pytest.mark.parametrize("limiter", ["minmod", "vanalbada"])
def test_hubble_expansion_paper_settings(H, limiter):
    """Sec. 3.2.2 Hubble-like expansion (e0 = 1, c_s^2 = 1/3, tau0 = 4, t0 = 2,
    dx = 0.1, dt = 0.03, vacuum outside r < t - 0.5) with the paper's four MUSTA
    stages and RK3 (Sec. 3.2), on a reduced 32^3 box."""
    n, dx, t0 = 32, 0.1, 2.0
    lo = -0.5 * n * dx
    c = I.cell_centres(n, lo, dx)
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(xx * xx + yy * yy + zz * zz)
    inside = r < t0 - 0.5
    e, vr = exact.hubble(np.where(inside, r, 0.0), t0)
    e = np.where(inside, e, 0.0)
    vr = np.where(inside, vr, 0.0)
    rs = np.where(r > 0, r, 1.0)
    prim = (e, vr * xx / rs, vr * yy / rs, vr * zz / rs)
    g = dict(nx=n, ny=n, nz=n, dx=dx, x0=lo, y0=lo, z0=lo)
    h, o, U = pair(H, g, prim, bc="outflow", limiter=limiter, stages=4, rk_order=3,
                   fixed_dt=0.03)
    o.run(U, 5)
    h.step(5)
    Ug = h.get_conserved()
    live = U[0] > 1e-3 * U[0].max()          # skip vacuum cells (E = 0)
    err = (np.abs(Ug - U)[:, live] / U[0][live][None]).max()
    assert err <= F64_TOL, err
    assert np.abs(Ug[:, ~live] - U[:, ~live]).max() <= 1e-12 * U[0].max()


def test_get_primitives_into_pinned_and_device_buffers(H):
    """The same primitives land in new arrays, pinned host tensors and CUDA
    tensors; a host output that cannot be written in place is refused."""
    import torch
    g, prim = I.spherical_blast(24)
    grid = H.make_grid(24, 24, 24, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec="fp32")
    h = H.Hydro(grid)
    h.set_primitives(*[a.astype(np.float32) for a in prim])
    h.step(2)
    ref = h.get_primitives()
    pinned = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in ref]
    dev = [torch.empty(a.shape, dtype=torch.float32, device="cuda") for a in ref]
    h.get_primitives(out=pinned)
    h.get_primitives(out=dev)
    for r, p, d in zip(ref, pinned, dev):
        assert np.array_equal(r, p.numpy())
        assert np.array_equal(r, d.cpu().numpy())
    with pytest.raises(ValueError):
        h.get_primitives(out=[np.empty(a.shape, dtype=np.float64) for a in ref])
