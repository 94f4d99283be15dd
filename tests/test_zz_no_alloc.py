"""hydro_conservation_sums_noalloc: the conservation sums for callers that
cannot allocate device memory (for example code running where another
allocator already holds the whole device, or a loop that must never call
cudaMalloc because it can synchronise the device).  Its output must match
hydro_conservation_sums on the same state, call after call.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_sums_match_the_handle_sums_twice(H, prec):
    import torch
    n = 40
    g, prim = I.spherical_blast(n)
    grid = H.make_grid(n, n, n, dx=g["dx"], x0=-1.0, y0=-1.0, z0=-1.0, prec=prec)
    h = H.Hydro(grid)
    h.set_primitives(*[a.astype(h.dtype) for a in prim])
    for step in range(2):
        h.step(3)
        want = h.conservation_sums()
        U = torch.empty((4, n, n, n), dtype=torch.float64 if prec == "fp64" else torch.float32,
                        device="cuda")
        h.get_conserved(out=U)
        torch.cuda.synchronize()
        for _ in range(2):   # two calls in a row share the library's scratch array
            got = H.conservation_sums_noalloc(U, prec, n, n, n, g["dx"])
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * abs(want[0]))


def test_noalloc_one_axis_grid_uses_the_handle_cell_volume(H):
    """A 1-D grid created with dy = dz = 0: the handle counts those axes as 1,
    and so does the no-allocation call."""
    import torch
    n = 64
    g, prim = I.shock_tube(n)
    grid = H.make_grid(n, dx=g["dx"], dy=0.0, dz=0.0, x0=-1.0, bc="outflow")
    h = H.Hydro(grid)
    h.set_primitives(*prim)
    h.step(5)
    want = h.conservation_sums()
    U = torch.empty((4, 1, 1, n), dtype=torch.float64, device="cuda")
    h.get_conserved(out=U)
    torch.cuda.synchronize()
    got = H.conservation_sums_noalloc(U, "fp64", n, 1, 1, g["dx"], 0.0, 0.0)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * abs(want[0]))


def _raw_call(H, U, prec, nx, ny, nz, dx, dy, dz):
    """The entry point itself, without the binding's own size checks."""
    import ctypes as C
    out = (C.c_double * 4)()
    return H.lib().hydro_conservation_sums_noalloc(C.c_void_p(U.data_ptr()), prec, nx, ny, nz,
                                                   dx, dy, dz, out, None)


def test_noalloc_rejects_grids_over_its_limit_and_bad_cell_sizes(H):
    import torch
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert _raw_call(H, U, 0, 1 << 15, 1 << 14, 1, 0.1, 0.1, 0.1) == 1
    assert "limit" in H.lib().hydro_last_error().decode()
    assert _raw_call(H, U, 0, 2, 2, 1, 0.1, 0.0, 0.1) == 1
    assert _raw_call(H, U, 0, 2, 2, 1, float("nan"), 0.1, 0.1) == 1


def test_fp32_sums_widen_every_float_class_exactly(H):
    """The FP32 sums widen each value to FP64 from its bit layout. Values
    spread over the whole normal exponent range, signed zeros and subnormals
    must sum as their exact FP64 values do (math.fsum of the same doubles;
    the kernel's own order differs, so the bound is a few ulps of the
    summed magnitudes, and a subnormal, below 1.2e-38, is invisible at it);
    an infinity and a NaN must come through."""
    import math
    import torch
    rng = np.random.default_rng(11)
    n = 4096
    mant = rng.uniform(1.0, 2.0, size=(4, n))
    expo = rng.integers(-126, 100, size=(4, n))
    sign = rng.choice([-1.0, 1.0], size=(4, n))
    U = (sign * np.ldexp(mant, expo)).astype(np.float32)
    U[1, :8] = np.array([0.0, -0.0, 1e-40, -1e-41, 1.1754944e-38, -1.1754944e-38,
                         3.4028235e38, -3.4028235e38], dtype=np.float32)
    U[2, 5] = np.nan
    U[3, 7] = np.inf
    dev = torch.from_numpy(U.reshape(4, 1, 1, n)).cuda()
    got = H.conservation_sums_noalloc(dev, "fp32", n, 1, 1, 1.0, 0.0, 0.0)
    for q in (0, 1):
        vals = U[q].astype(np.float64)
        want = math.fsum(vals)
        scale = float(np.abs(vals).sum())
        assert abs(got[q] - want) <= 1e-14 * scale, (q, got[q], want)
    assert math.isnan(got[2])
    assert got[3] == math.inf
