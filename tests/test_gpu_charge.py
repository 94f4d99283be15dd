"""GPU parity of the conserved charge R = n gamma (Eq. 1, 3, 4) carried as a
fifth field: the CUDA sweeps through the C ABI against the FP64 CPU oracle
(FP64 <= 1e-10 relative per cell, FP32 <= 1e-4 relative L1 per field, the
tolerances of the four-field tests), the charge sum, the density readout,
and the batch path."""
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


def rel_charge(got, want):
    """max |R - R_ref| / max(|R_ref|, 1e-12 max |R_ref|)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.maximum(np.abs(want), 1e-12 * np.abs(want).max())
    return float((np.abs(got - want) / scale).max())


def check(U, Uo, prec):
    if prec == "fp64":
        assert max_rel_per_cell(U[:4], Uo[:4]) <= F64_TOL
        assert rel_charge(U[4], Uo[4]) <= F64_TOL
    else:
        err = rel_l1(U, Uo)
        assert max(err) <= F32_TOL, err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_charged_shock_tube_matches_oracle(H, prec):
    """1000 cells to t = 0.8 with n_L = 1, n_R = 0.5; the GPU's n is also
    close to the exact solution."""
    n = 1000
    g, prim = I.shock_tube(n)
    x = I.cell_centres(n, -1.0, g["dx"])
    nn = np.where(x < 0.0, 1.0, 0.5).reshape(1, 1, n)
    o = O.Oracle(n, dx=g["dx"], x0=-1.0, bc="outflow", cfl=0.4, charge=1)
    U0 = o.prim2cons_field(*prim, n=nn)
    grid = H.make_grid(n, dx=g["dx"], x0=-1.0, bc="outflow", prec=prec, cfl=0.4, charge=True)
    h = H.Hydro(grid)
    h.set_conserved(U0.astype(h.dtype))
    t = h.step(100000, t_end=0.8)
    Uo = U0.copy()
    o.run(Uo, 100000, t_end=0.8)
    assert t == 0.8
    check(h.get_conserved(), Uo, prec)
    dens = h.charge_density().astype(np.float64).ravel()
    want = o.charge_density_field(Uo).ravel()
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert np.abs(dens - want).sum() / np.abs(want).sum() <= tol
    ex = exact.Riemann().sample_n(x, 0.8, 1.0, 0.5)
    assert np.abs(dens - ex).sum() / ex.sum() < 0.02


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("rk", [1, 2, 3])
def test_charged_blast_matches_oracle_and_conserves_charge(H, prec, rk):
    """3-D blast, periodic, a smooth charge density, Superbee; 24^3 spans
    several blocks and pencil segments with a ragged tail."""
    n = 24
    g, prim = I.spherical_blast(n)
    c = I.cell_centres(n, -1.0, g["dx"])
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    nn = 1.0 + 0.5 * np.cos(np.pi * xx) * np.sin(np.pi * yy) + 0.2 * zz
    o = O.Oracle(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, bc="periodic",
                 limiter="superbee", rk_order=rk, charge=1)
    U0 = o.prim2cons_field(*prim, n=nn)
    grid = H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec=prec,
                       rk_order=rk, charge=True)
    h = H.Hydro(grid, limiter="superbee")
    h.set_primitives(*[a.astype(h.dtype) for a in prim], n=nn.astype(h.dtype))
    np.testing.assert_allclose(h.get_conserved().astype(np.float64), U0,
                               rtol=1e-14 if prec == "fp64" else 1e-6)
    q0 = h.charge_sum()
    h.step(3)
    Uo = U0.copy()
    o.run(Uo, 3)
    check(h.get_conserved(), Uo, prec)
    q1 = h.charge_sum()
    want = o.conservation_sums(Uo)[4]
    assert abs(q1 - want) <= (1e-12 if prec == "fp64" else 1e-6) * abs(want)
    assert abs(q1 - q0) <= (1e-12 if prec == "fp64" else 1e-6) * abs(q0)


def test_charged_sweeps_with_the_tabulated_eos_match_oracle(H):
    """Hot spots with flow, the tabulated EOS (Newton cons->prim), FP64."""
    tab = I.eos_table()
    n = 16
    g = I.event_grid(n, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(2, nspots=40, flow_max=0.6))
    nn = 0.3 * prim[0] ** 0.75
    o = O.Oracle(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow", eos=tab,
                 charge=1)
    U0 = o.prim2cons_field(*prim, n=nn)
    grid = H.make_grid(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow",
                       prec="fp64", charge=True)
    h = H.Hydro(grid, H.make_eos(tab))
    h.set_conserved(U0)
    h.step(3)
    Uo = U0.copy()
    o.run(Uo, 3)
    check(h.get_conserved(), Uo, "fp64")


def test_charged_ellipsoidal_flow_matches_oracle_and_exact_n(H):
    """The paper's ellipsoidal flow (p = 0) with its charge density, 1-D along
    x, FP64: equal to the oracle, and n close to the exact solution."""
    n, half, t0 = 240, 3.0, 2.0
    dx = 2 * half / n
    x = I.cell_centres(n, -half, dx)
    e, (v,) = exact.ellipsoidal([x], t0)
    nn, _ = exact.ellipsoidal([x], t0, C=0.75, b=1.0)
    dt = 0.2 * dx
    steps = 20
    o = O.Oracle(n, dx=dx, x0=-half, bc="outflow", cs2=0.0, fixed_dt=dt, charge=1)
    z = np.zeros((1, 1, n))
    U0 = o.prim2cons_field(e.reshape(1, 1, n), v.reshape(1, 1, n), z, z,
                           n=nn.reshape(1, 1, n))
    grid = H.make_grid(n, dx=dx, x0=-half, bc="outflow", prec="fp64", fixed_dt=dt,
                       charge=True)
    h = H.Hydro(grid, H.make_eos(cs2=0.0))
    h.set_conserved(U0)
    h.step(steps)
    Uo = U0.copy()
    o.run(Uo, steps)
    check(h.get_conserved(), Uo, "fp64")
    got = h.charge_density().ravel()
    want, _ = exact.ellipsoidal([x], t0 + steps * dt, C=0.75, b=1.0)
    core = np.abs(x) < 1.2
    assert np.abs(got[core] - want[core]).sum() / want[core].sum() < 1e-3


def test_charged_batch_equals_single_runs(H):
    """Two charged events of different sizes in one batch give the single
    handles' results bit for bit; their charge sums likewise."""
    outs, sums, grids, states = [], [], [], []
    for k, n in enumerate((18, 27)):
        g, prim = I.spherical_blast(n)
        c = I.cell_centres(n, -1.0, g["dx"])
        zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
        nn = (1.0 + 0.3 * np.sin(np.pi * (xx + k * yy))).astype(np.float32)
        grid = H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec="fp32",
                           charge=True)
        h = H.Hydro(grid)
        h.set_primitives(*[a.astype(np.float32) for a in prim], n=nn)
        states.append(h.get_conserved())
        h.step(2)
        outs.append(h.get_conserved())
        sums.append(h.charge_sum())
        grids.append(grid)
    b = H.Batch(grids)
    for e, U in enumerate(states):
        b.set_conserved(e, U)
    b.step(2)
    for e in range(2):
        assert np.array_equal(b.get_conserved(e), outs[e])
    np.testing.assert_allclose(b.charge_sums(), sums, rtol=1e-12)


def test_charge_is_rejected_where_it_is_not_built(H):
    g = H.make_grid(8, 8, 8, dx=0.1, charge=True, unsplit=True)
    with pytest.raises(H.HydroError):
        H.Hydro(g)
    h = H.Hydro(H.make_grid(8, dx=0.1))
    with pytest.raises(H.HydroError):
        h.charge_sum()
