"""GPU tests of the per-event status words: the kernels record a Newton solve
that hits its iteration cap and an inadmissible state (|M| >= (1 - delta) E)
that they repaired, and the host reads both after the step.  The failures are
made on the host (an iteration cap of 1, a state with |M| > E); nothing waits
or traps on the device."""
import numpy as np
import pytest

from paper_1510_06340_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1510_06340_b300 import build, hydro
    build.build(verbose=False)
    return hydro


def flowing_line(n=64):
    """A smooth 1-D state with |v| up to 0.9, so that every Newton solve of
    the tabulated EOS needs several iterations."""
    x = I.cell_centres(n, -1.0, 2.0 / n)
    e = (1.0 + 0.5 * np.sin(np.pi * x)).reshape(1, 1, n)
    vx = (0.9 * np.cos(np.pi * x)).reshape(1, 1, n)
    z = np.zeros_like(e)
    return e, vx, z, z.copy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_newton_cap_sets_the_newton_status(H, prec):
    tab = I.eos_table()
    n = 64
    codes = {}
    for cap in (0, 1):      # 0: the default cap of 50
        grid = H.make_grid(n, dx=2.0 / n, x0=-1.0, bc="periodic", prec=prec)
        h = H.Hydro(grid, H.make_eos(tab, seed="zero", newton_max_iter=cap))
        prim = [a.astype(h.dtype) for a in flowing_line(n)]
        h.set_primitives(*prim)
        h.step(2)
        codes[cap] = h.status()
        with pytest.raises(H.HydroError) if cap else _nothing():
            H._check(H.lib().hydro_check_status(h.h, None))
    assert codes[0] == (0, 0), codes
    assert codes[1][0] == 5 and codes[1][1] & H.FLAG_NEWTON, codes


class _nothing:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def smooth_3d(n):
    """A smooth periodic state at rest (no face comes near inadmissibility)."""
    c = I.cell_centres(n, -1.0, 2.0 / n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    e = 1.0 + 0.3 * np.sin(np.pi * x) * np.cos(np.pi * y) + 0.1 * np.sin(np.pi * z)
    zero = np.zeros_like(e)
    return dict(dx=2.0 / n), (e, zero, zero.copy(), zero.copy())


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_inadmissible_state_sets_the_unphysical_status(H, prec):
    """One cell with |M| = 1.5 E: cons->prim caps it and its faces fall back
    (the admissibility rule); the state stays finite and the status says
    UNPHYSICAL.  The same grid without that cell stays OK, and setting the
    state again clears the word."""
    n = 32
    g, prim = smooth_3d(n)
    grid = H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec=prec)
    h = H.Hydro(grid)
    h.set_primitives(*[a.astype(h.dtype) for a in prim])
    U = h.get_conserved()
    h.step(2)
    assert h.status() == (0, 0)
    bad = U.copy()
    bad[1, 5, 7, 9] = 1.5 * bad[0, 5, 7, 9]
    h.set_conserved(bad)
    h.step(2)
    code, flags = h.status()
    assert code == 4 and flags == H.FLAG_UNPHYSICAL, (code, flags)
    h.check_finite()
    h.set_conserved(U)
    assert h.status() == (0, 0)


def test_batch_reports_each_event(H):
    """Three events; only event 1 holds the inadmissible cell."""
    n = 24
    g, prim = smooth_3d(n)
    grids = [H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec="fp32")
             for _ in range(3)]
    b = H.Batch(grids)
    for e in range(3):
        b.set_primitives(e, *[a.astype(np.float32) for a in prim])
    U = b.get_conserved(1)
    U[2, 3, 4, 5] = -1.2 * U[0, 3, 4, 5]
    b.set_conserved(1, U)
    b.step(2)
    codes, flags = b.event_flags()
    assert list(codes) == [0, 4, 0], (codes, flags)
    assert list(flags) == [0, H.FLAG_UNPHYSICAL, 0]
    assert list(b.event_status()) == [0, 4, 0]
