"""GPU parity of the unsplit scheme (the paper's multi-D MUSCL-Hancock of
Eq. 13 with every flux term, FORCE alpha = 3; reading R16) against the
oracle's unsplit step, through the C ABI.

Tolerances as for the split path (reading R13): FP64 <= 1e-10 max relative
per cell, FP32 and mixed <= 1e-4 relative L1 per field.  Sizes span several
work items and ragged grids; both boundary conditions, every RK order, a
runtime limiter, the tabulated EOS and batches are covered.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_06340_b300 import inputs as I
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


def pair(H, shape, dx, lo, prim, prec="fp64", bc="periodic", limiter="minmod", stages=2,
         rk_order=2, cfl=0.4, fixed_dt=0.0, eos=None, seed="zero"):
    nz, ny, nx = shape
    grid = H.make_grid(nx, ny, nz, dx=dx, x0=lo[0], y0=lo[1], z0=lo[2], bc=bc, prec=prec,
                       rk_order=rk_order, cfl=cfl, fixed_dt=fixed_dt, unsplit=True)
    h = H.Hydro(grid, H.make_eos(eos, seed=seed), limiter=limiter, stages=stages)
    o = O.Oracle(nx, ny, nz, dx=dx, x0=lo[0], y0=lo[1], z0=lo[2], bc=bc, limiter=limiter,
                 stages=stages, rk_order=rk_order, cfl=cfl, fixed_dt=fixed_dt, alpha=3.0,
                 unsplit=1, eos=eos, seed_kind=H.SEEDS[seed])
    U0 = o.prim2cons_field(*prim)
    h.set_conserved(U0.astype(h.dtype))
    return h, o, U0


def check(h, U_ref, prec):
    U = h.get_conserved().astype(np.float64)
    if prec == "fp64":
        err = max_rel_per_cell(U, U_ref)
        assert err <= F64_TOL, err
    else:
        err = max(rel_l1(U, U_ref))
        assert err <= F32_TOL, err
    return err


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_unsplit_blast_matches_oracle(H, prec):
    n = 20
    g, prim = I.spherical_blast(n)
    h, o, U = pair(H, (n, n, n), g["dx"], (-1.0, -1.0, -1.0), prim, prec=prec)
    _, t = o.run(U, 5)
    h.step(5)
    check(h, U, prec)
    assert h.time() == pytest.approx(t, rel=1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("rk", [1, 2, 3])
def test_unsplit_ragged_outflow_hot_spots(H, rk):
    """A ragged grid (13 x 11 x 9, several work items, uneven lines) with hot
    spots and random flow, outflow on every side."""
    shape = (9, 11, 13)
    dx = 0.4
    lo = (-0.5 * 13 * dx, -0.5 * 11 * dx, -0.5 * 9 * dx)
    g = dict(nx=13, ny=11, nz=9, dx=dx, x0=lo[0], y0=lo[1], z0=lo[2])
    prim = I.hotspot_primitives(g, I.hotspots(5, nspots=40, flow_max=0.7))
    h, o, U = pair(H, shape, dx, lo, prim, bc="outflow", rk_order=rk, cfl=0.3)
    o.run(U, 4)
    h.step(4)
    check(h, U, "fp64")


@pytest.mark.parametrize("limiter", ["mc", "vanleer", "none"])
def test_unsplit_runtime_limiters(H, limiter):
    n = 12
    g, prim = I.spherical_blast(n)
    h, o, U = pair(H, (n, n, n), g["dx"], (-1.0, -1.0, -1.0), prim, limiter=limiter,
                   fixed_dt=0.1 * g["dx"])
    o.run(U, 3)
    h.step(3)
    check(h, U, "fp64")


def test_unsplit_2d_and_1d_grids(H):
    """Inactive axes take no faces or fluxes: a 2-D grid and a 1-D line."""
    g, prim = I.shock_tube(64)
    h, o, U = pair(H, (1, 1, 64), g["dx"], (-1.0, 0.0, 0.0), prim, bc="outflow")
    o.run(U, 10)
    h.step(10)
    check(h, U, "fp64")
    n = 24
    dx = 2.0 / n
    c = I.cell_centres(n, -1.0, dx)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    e = np.where(xx * xx + yy * yy < 0.1, 10.0, 1.0).reshape(1, n, n)
    z = np.zeros_like(e)
    h, o, U = pair(H, (1, n, n), dx, (-1.0, -1.0, 0.0), (e, z, z, z))
    o.run(U, 6)
    h.step(6)
    check(h, U, "fp64")


def test_unsplit_table_eos(H):
    tab = I.eos_table()
    shape = (10, 10, 10)
    dx = 0.5
    lo = (-2.5, -2.5, -2.5)
    g = dict(nx=10, ny=10, nz=10, dx=dx, x0=lo[0], y0=lo[1], z0=lo[2])
    prim = I.hotspot_primitives(g, I.hotspots(7, nspots=30, flow_max=0.6))
    h, o, U = pair(H, shape, dx, lo, prim, bc="outflow", eos=tab, cfl=0.3)
    o.run(U, 3)
    h.step(3)
    check(h, U, "fp64")


def test_unsplit_conserves_and_rate_sums_axes(H):
    n = 16
    g, prim = I.spherical_blast(n)
    h, o, U = pair(H, (n, n, n), g["dx"], (-1.0, -1.0, -1.0), prim)
    assert h.max_rate() == pytest.approx(o.max_rate(U), rel=1e-12)
    s0 = h.conservation_sums()
    h.step(6)
    s1 = h.conservation_sums()
    assert abs(s1[0] - s0[0]) <= 1e-12 * s0[0]
    assert np.abs(s1[1:]).max() <= 1e-12 * s0[0]


def test_unsplit_graph_steps_equal_single_steps(H):
    """Steps replayed from a CUDA graph equal steps enqueued one by one."""
    n = 16
    g, prim = I.spherical_blast(n)
    outs = []
    for chunks in ([5], [1] * 5):
        h, _, _ = pair(H, (n, n, n), g["dx"], (-1.0, -1.0, -1.0), prim, prec="fp32")
        for k in chunks:
            h.step(k)
        outs.append(h.get_conserved())
    assert np.array_equal(outs[0], outs[1])


def test_unsplit_batch_equals_single_runs(H):
    """Uneven events in one batch take the same arithmetic as alone."""
    sizes = [9, 14, 11]
    grids, prims = [], []
    for k, n in enumerate(sizes):
        g = I.event_grid(n, 0.4)
        grids.append(H.make_grid(n, n, n, dx=0.4, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                                 bc="outflow", prec="fp32", cfl=0.3, unsplit=True))
        prims.append(I.hotspot_primitives(g, I.hotspots(20 + k, nspots=30, flow_max=0.5)))
    b = H.Batch(grids)
    for e, p in enumerate(prims):
        b.set_primitives(e, *[a.astype(np.float32) for a in p])
    b.step(3)
    for e, p in enumerate(prims):
        h = H.Hydro(grids[e])
        h.set_primitives(*[a.astype(np.float32) for a in p])
        h.step(3)
        assert np.array_equal(h.get_conserved(), b.get_conserved(e)), e


def test_unsplit_rejects_mixed_schemes_in_a_batch(H):
    g1 = H.make_grid(8, 8, 8, dx=0.1, unsplit=True)
    g2 = H.make_grid(8, 8, 8, dx=0.1)
    with pytest.raises(Exception):
        H.Batch([g1, g2])


def test_unsplit_cfl_step_with_vacuum_matches_oracle(H):
    """A fast blob (|v| = 0.9) in vacuum under the CFL step: the summed rate of
    the vacuum cells (3 c / dx) exceeds the blob's, so dt is set by the vacuum
    rule (R18: v = 0, speed c) and must equal the oracle's."""
    n = 16
    dx = 0.25
    lo = -0.5 * n * dx
    g = dict(nx=n, ny=n, nz=n, dx=dx, x0=lo, y0=lo, z0=lo)
    spots = np.array([[0.0, 0.0, 0.0, 2.0, 0.9, 0.0, 0.0]])
    e, vx, vy, vz = I.hotspot_primitives(g, spots, sigma=0.5, e_bg=0.0)
    inside = e > 1e-3 * e.max()          # vacuum (e = v = 0) outside the blob
    prim = [np.where(inside, a, 0.0) for a in (e, vx, vy, vz)]
    assert not inside.all()
    h, o, U = pair(H, (n, n, n), dx, (lo, lo, lo), prim, bc="outflow", cfl=0.3)
    assert h.max_rate() == pytest.approx(o.max_rate(U), rel=1e-12)
    _, t = o.run(U, 4)
    h.step(4)
    assert h.time() == pytest.approx(t, rel=1e-12)
    check(h, U, "fp64")
