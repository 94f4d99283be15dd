"""GPU tests of the learned cons->prim seed for the tabulated EOS.

* forward (tensor cores, bf16 weights and layer-2 inputs) against the oracle's
  FP64 forward with the same bf16 rounding;
* loss gradient against the oracle's FP64 gradient (rounding passed through);
* training on (T^{0mu}, v) pairs generated by the solver's own Newton solve
  lowers the loss, and the trained seed cuts Newton iterations;
* with the learned seed the polished result equals the plain Newton result
  (<= 1e-12 in FP64), inside cons->prim and inside whole sweeps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1510_06340_b300 import inputs as I
from tests.metrics import max_rel_per_cell, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1510_06340_b300 import build, hydro
    build.build(verbose=False)
    return hydro


def random_params(rng, n):
    P = rng.normal(size=n) * 0.4
    P[-4:] = [1.0, 3.0, 0.5, 0.3]     # mu0, s0, mu1, s1
    return P


def random_inputs(rng, n):
    return np.column_stack([rng.uniform(-6, 8, n), rng.uniform(0.0, 0.99, n)])


def test_mlp_forward_matches_oracle(H):
    """Layer by layer.  Layer 1: the GPU's bf16-rounded activations equal the
    oracle's, or differ by one bf16 step where FP32 and FP64 tanh straddle a
    rounding boundary.  Layers 2-3: the oracle fed the GPU's own activations
    gives the GPU's output to FP32 accuracy.  Whole forward: the two differ
    only by those rare rounding steps."""
    import torch
    rng = np.random.default_rng(11)
    nP = H.mlp_nparam()
    P = random_params(rng, nP).astype(np.float32).astype(np.float64)
    X = random_inputs(rng, 1000)
    Xf = X.astype(np.float32).astype(np.float64)
    Pd = torch.tensor(P, dtype=torch.float32, device="cuda")
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    out = torch.empty(1000, dtype=torch.float32, device="cuda")
    H.mlp_forward(Pd, Xd, out)
    got = out.cpu().numpy().astype(np.float64)
    H1d = torch.empty(1000, 32, dtype=torch.float32, device="cuda")
    H.mlp_hidden(Pd, Xd, H1d)
    H1 = H1d.cpu().numpy().astype(np.float64)
    H1o = O.mlp_hidden(P, Xf, quantize=1)
    step = np.abs(H1 - H1o)
    # one bf16 step at |h|: 2^(floor(log2 |h|) - 7) (8 significant bits)
    big = np.maximum(np.abs(H1), np.abs(H1o))
    ulp = np.exp2(np.floor(np.log2(np.where(big > 0, big, 1.0))) - 7)
    print("layer 1: entries one bf16 step apart:", (step > 0).mean(),
          "max steps:", (step / ulp).max())
    assert (step <= ulp).all(), (step / ulp).max()
    assert (step > 0).mean() < 0.01, (step > 0).mean()
    want_h1 = O.mlp_forward_h1(P, Xf, H1, quantize=1)
    err23 = np.abs(got - want_h1)
    print("layers 2-3 max |GPU - oracle(GPU h1)|:", err23.max())
    assert err23.max() <= 2e-5, err23.max()
    want = O.mlp_forward(P, Xf, quantize=1)
    err = np.abs(got - want)
    same = (step == 0).all(axis=1)          # samples whose layer 1 matched exactly
    assert err[same].max() <= 2e-5, err[same].max()
    assert err.max() <= 3e-3 and err.mean() <= 2e-4, (err.max(), err.mean())


# parameter blocks of the seed network, each checked on its own scale
BLOCKS = {"W1": (0, 64), "b1": (64, 96), "W2": (96, 1120), "b2": (1120, 1152),
          "W3": (1152, 1184), "b3": (1184, 1185)}


def test_mlp_gradient_matches_oracle(H):
    """Element by element, each parameter block on its own scale:
    |G_i - G_oracle,i| <= 1e-5 |G_oracle,i| + 1e-6 max_block |G_oracle|
    (FP32 accumulation over 2048 samples against FP64)."""
    import torch
    rng = np.random.default_rng(12)
    nP = H.mlp_nparam()
    assert nP == 1189 and BLOCKS["b3"][1] == nP - 4
    P = random_params(rng, nP).astype(np.float32).astype(np.float64)
    X = random_inputs(rng, 2048).astype(np.float32).astype(np.float64)
    Y = (X[:, 1] * rng.uniform(0.7, 1.0, 2048)).astype(np.float32).astype(np.float64)
    loss_o, G_o = O.mlp_loss_grad(P, X, Y, quantize=1)
    grad = torch.empty(nP, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    H.mlp_loss_grad(torch.tensor(P, dtype=torch.float32, device="cuda"),
                    torch.tensor(X, dtype=torch.float32, device="cuda"),
                    torch.tensor(Y, dtype=torch.float32, device="cuda"), grad, loss)
    G = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - loss_o) <= 1e-4 * loss_o
    assert not G[-4:].any()
    worst = {}
    for name, (a, b) in BLOCKS.items():
        g, go = G[a:b], G_o[a:b]
        scale = np.abs(go).max()
        assert scale > 0, name
        bound = 1e-5 * np.abs(go) + 1e-6 * scale
        worst[name] = float((np.abs(g - go) / bound).max())
    print("gradient error / bound per block:", worst)
    assert max(worst.values()) <= 1.0, worst


def solver_pairs(H, tab, n, rng):
    """(T^{0mu}, v) pairs made by the solver itself: states from the tabulated
    EOS's prim->cons on the device, targets from its plain Newton solve."""
    import torch
    e = np.exp(rng.uniform(np.log(1e-3), np.log(1e2), n))
    v = 0.95 * rng.uniform(0, 1, n) ** 0.5
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    grid = H.make_grid(n, dx=1.0, prec="fp64")
    h = H.Hydro(grid, H.make_eos(tab, seed="zero"))
    h.set_primitives(e.reshape(1, 1, n), (v * d[0]).reshape(1, 1, n),
                     (v * d[1]).reshape(1, 1, n), (v * d[2]).reshape(1, 1, n))
    U = torch.tensor(h.get_conserved().reshape(4, n), device="cuda")
    vmag = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    h.c2p_newton(U, "zero", vmag, it)
    Uh = U.cpu().numpy()
    E, M = Uh[0], np.linalg.norm(Uh[1:], axis=0)
    X = np.column_stack([np.log(E), M / E])
    return U, X, vmag.cpu().numpy(), it.cpu().numpy()


@pytest.fixture(scope="module")
def trained(H):
    import torch
    rng = np.random.default_rng(13)
    tab = I.eos_table()
    U, X, Y, _ = solver_pairs(H, tab, 65536, rng)
    nP = H.mlp_nparam()
    P = rng.normal(size=nP) * 0.3
    P[-4:] = [X[:, 0].mean(), X[:, 0].std(), X[:, 1].mean(), X[:, 1].std()]
    params = torch.tensor(P, dtype=torch.float32, device="cuda")
    hist = torch.zeros(150, dtype=torch.float32, device="cuda")
    H.mlp_train(params, torch.tensor(X, dtype=torch.float32, device="cuda"),
                torch.tensor(Y, dtype=torch.float32, device="cuda"), 512, 150, 3e-3, 7, hist)
    print("training loss by epoch:", hist.cpu().numpy()[::10])
    return tab, params.cpu().numpy(), hist.cpu().numpy()


def test_training_on_solver_pairs_lowers_the_loss(H, trained):
    _, _, hist = trained
    assert hist[-1] < hist[0] / 100, hist
    assert hist[-1] < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_learned_seed_cuts_newton_iterations_and_keeps_the_root(H, trained, prec):
    import torch
    tab, P, _ = trained
    rng = np.random.default_rng(14)
    U, X, Y, it_plain = solver_pairs(H, tab, 20000, rng)
    grid = H.make_grid(8, dx=1.0, prec=prec)
    h = H.Hydro(grid, H.make_eos(tab, seed="mlp", mlp_params=P))
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ud = U.to(dt).contiguous()
    res = {}
    for seed in ("zero", "conformal", "mlp"):
        v = torch.empty(U.shape[1], dtype=dt, device="cuda")
        it = torch.empty(U.shape[1], dtype=torch.int32, device="cuda")
        h.c2p_newton(Ud, seed, v, it)
        res[seed] = (v.cpu().numpy().astype(np.float64), it.cpu().numpy())
    mean_it = {k: r[1].mean() for k, r in res.items()}
    print("mean Newton iterations per solve:", mean_it)
    # the paper's fixed-point start (v0 = 0) is the method without the network
    assert mean_it["mlp"] < 0.85 * mean_it["zero"], mean_it
    assert mean_it["mlp"] <= mean_it["conformal"] + 0.15, mean_it
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(res["mlp"][0] - res["zero"][0]).max() <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sweeps_with_learned_seed_match_plain_and_oracle(H, trained, prec):
    """The seed runs warp-wide on the tensor cores inside the sweep kernels."""
    tab, P, _ = trained
    g = I.event_grid(16, 0.1)
    prim = I.hotspot_primitives(g, I.hotspots(4, nspots=60, flow_max=0.8))
    o = O.Oracle(16, 16, 16, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"], bc="outflow", eos=tab)
    U0 = o.prim2cons_field(*prim)
    outs = {}
    for seed in ("zero", "mlp"):
        grid = H.make_grid(16, 16, 16, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                           bc="outflow", prec=prec)
        h = H.Hydro(grid, H.make_eos(tab, seed=seed, mlp_params=P))
        h.set_conserved(U0.astype(h.dtype))
        h.step(4)
        outs[seed] = h.get_conserved().astype(np.float64)
    Uo = U0.copy()
    o.run(Uo, 4)
    if prec == "fp64":
        assert max_rel_per_cell(outs["mlp"], outs["zero"]) <= 1e-12
        assert max_rel_per_cell(outs["mlp"], Uo) <= 1e-10
    else:
        assert max(rel_l1(outs["mlp"], Uo)) <= 1e-4
