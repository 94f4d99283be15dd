"""Full-size checks in the launch configurations the benchmark times, by
properties that hold at any size (the oracle cannot run these sizes):

* the 512-event batch (grids 64^3..160^3, hot spots, jets, one persistent
  launch per sweep over all events) equals separate single-event runs bit
  for bit, for its first and last events;
* the 512^3 mixed-precision event stays within 1e-4 relative L1 per field of
  an FP64 run from the same state;
* the 128-event x 128^3 tabulated-EOS batch gives the same state with the
  learned Newton seed as with the plain one (polishing removes the seed).
"""
import numpy as np
import pytest

from paper_1510_06340_b300 import inputs as I
from tests.metrics import rel_l1

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1510_06340_b300 import build, hydro
    build.build(verbose=False)
    return hydro


def event_grid(H, n, prec="fp32"):
    g = I.event_grid(int(n), 0.1)
    return H.make_grid(int(n), int(n), int(n), dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                       bc="outflow", prec=prec, cfl=0.4)


def test_full_batch_events_equal_single_runs(H):
    nev = 512
    sizes = I.event_sizes(nev)
    spots = np.stack([I.hotspots(e) for e in range(nev)])
    jets = np.stack([I.jet(e) for e in range(nev)])
    b = H.Batch([event_grid(H, n) for n in sizes])
    b.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    b.set_jets(jets)
    b.step(3)
    codes, flags = b.event_flags()
    # no NaN/Inf and no Newton trouble (conformal EOS); cells repaired by the
    # admissibility rule are reported, not failures
    assert not np.isin(codes, (5, 6)).any(), codes
    print("events with an inadmissible state repaired:", int((codes == 4).sum()))
    times = b.times()
    for e in (0, nev - 1):
        h = H.Hydro(event_grid(H, sizes[e]))
        h.init_hotspots(spots[e], I.SPOT_SIGMA, I.E_BACKGROUND)
        h.set_jet(jets[e])
        h.step(3)
        assert h.time() == times[e]
        assert np.array_equal(h.get_conserved(), b.get_conserved(e)), e


def test_512_cubed_mixed_against_fp64(H):
    spots = I.hotspots(0, flow_max=0.95)
    hm = H.Hydro(event_grid(H, 512, "mixed"))
    hm.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
    U0 = hm.get_conserved()
    hm.step(2)
    Um = hm.get_conserved()
    del hm
    hd = H.Hydro(event_grid(H, 512, "fp64"))
    hd.set_conserved(U0.astype(np.float64))
    hd.step(2)
    err = rel_l1(Um, hd.get_conserved())
    print("512^3 mixed vs FP64, rel L1 per field:", err)
    assert max(err) <= 1e-4


def test_learned_batch_equals_plain_seed(H):
    import torch
    rng = np.random.default_rng(3)
    P = rng.normal(size=H.mlp_nparam()) * 0.3       # any seed network: Newton polishes
    P[-4:] = [0.0, 3.0, 0.3, 0.3]
    tab = I.eos_table()
    spots = np.stack([I.hotspots(e) for e in range(128)])
    out = {}
    for seed in ("zero", "mlp"):
        b = H.Batch([event_grid(H, 128) for _ in range(128)],
                    H.make_eos(tab, seed=seed, mlp_params=P))
        b.init_hotspots(spots, I.SPOT_SIGMA, I.E_BACKGROUND)
        b.step(2)
        out[seed] = [b.get_conserved(e).astype(np.float64) for e in (0, 77, 127)]
        del b
        torch.cuda.synchronize()
    for a, z in zip(out["mlp"], out["zero"]):
        assert max(rel_l1(a, z)) <= 1e-5
