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


def test_noalloc_rejects_grids_over_its_limit(H):
    import torch
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HydroError) as ei:
        H.conservation_sums_noalloc(U, "fp64", 1 << 15, 1 << 14, 1, 0.1)
    assert ei.value.status == 1 and "limit" in str(ei.value)
