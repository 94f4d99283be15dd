"""GPU tests of the mixed-precision path: FP32 state and fluxes, cons->prim
redone in FP64 where the FP32 estimate gives |v| > 0.99, FP64 conservation
sums.  Errors are stated per field against an FP64 run of the same problem
(relative L1, reading R13)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_06340_b300 import inputs as I
from tests.metrics import rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1510_06340_b300 import build, hydro
    build.build(verbose=False)
    return hydro


def run(H, g, prim, prec, steps, counters=False):
    grid = H.make_grid(g["nx"], g.get("ny", 1), g.get("nz", 1), dx=g["dx"], x0=g.get("x0", 0.0),
                       y0=g.get("y0", 0.0), z0=g.get("z0", 0.0), bc="outflow", prec=prec,
                       fixed_dt=g.get("dt", 0.0))
    h = H.Hydro(grid)
    if counters:
        h.enable_counters(True)
    h.set_primitives(*[np.ascontiguousarray(a, dtype=h.dtype) for a in prim])
    h.step(steps)
    return h.get_conserved().astype(np.float64), (h.counters() if counters else None)


def test_hotspots_with_random_flow_mixed_vs_fp64(H):
    """The config-4 recipe (hot spots, |u_j| <= 0.95) at 48^3: per-field errors."""
    g = I.event_grid(48, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(21, flow_max=0.95))
    ref, _ = run(H, g, prim, "fp64", 20)
    mixed, cnt = run(H, g, prim, "mixed", 20, counters=True)
    f32, _ = run(H, g, prim, "fp32", 20)
    err_m, err_f = rel_l1(mixed, ref), rel_l1(f32, ref)
    print("rel L1 per field vs FP64: mixed", err_m, "fp32", err_f, "counters", cnt)
    assert max(err_m) <= 1e-4 and max(err_f) <= 1e-4


def test_fp64_redo_in_ultrarelativistic_cells(H):
    """At v = 0.9999 the rest-frame e = E - M.v cancels to ~1e-4 of E.  On the
    same FP32 state, FP32 cons->prim loses those digits; the mixed path redoes
    the cell in FP64 and matches the FP64 recovery.  The redo also runs in the
    sweeps (counted)."""
    n = 256
    dx = 2.0 / n
    x = I.cell_centres(n, -1.0, dx)
    e = np.where(np.abs(x) < 0.3, 1.0, 0.5) * (1.0 + 0.1 * np.cos(4 * x))
    v = np.where(np.abs(x) < 0.3, 0.9999, 0.2)
    z = np.zeros(n)
    prim = tuple(a.reshape(1, 1, n) for a in (e, v, z, z))
    g = dict(nx=n, dx=dx, x0=-1.0, dt=0.2 * dx)
    state, _ = run(H, g, prim, "fp64", 10)
    _, cnt = run(H, g, prim, "mixed", 10, counters=True)
    assert cnt["f64_redo"] > 0
    U32 = state.astype(np.float32)
    out = {}
    for prec in ("fp64", "mixed", "fp32"):
        grid = H.make_grid(n, dx=dx, x0=-1.0, bc="outflow", prec=prec)
        h = H.Hydro(grid)
        h.set_conserved(U32.astype(h.dtype))      # the same values in every handle
        out[prec] = h.get_primitives()[0].astype(np.float64).ravel()
    fast = np.abs(x) < 0.25
    rel = {k: np.abs(out[k][fast] / out["fp64"][fast] - 1).max() for k in ("mixed", "fp32")}
    print("max relative error of e in the v = 0.9999 cells:", rel, cnt)
    assert rel["mixed"] <= 1e-6
    assert rel["fp32"] >= 10 * rel["mixed"]


def test_mixed_conservation_sums_are_fp64(H):
    g, prim = I.spherical_blast(32)
    grid = H.make_grid(32, 32, 32, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec="mixed")
    h = H.Hydro(grid)
    h.set_primitives(*[a.astype(np.float32) for a in prim])
    U = h.get_conserved().astype(np.float64)
    o = O.Oracle(32, 32, 32, dx=g["dx"])
    np.testing.assert_allclose(h.conservation_sums(), o.conservation_sums(U), rtol=1e-13)
