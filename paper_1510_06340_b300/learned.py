"""Training of the Newton-seed network for a tabulated EOS on states that the
solver itself produces (orchestration only: every step runs in libhydro's
kernels -- the sweeps, the plain Newton solve that makes the targets, and the
network's forward, backward and Adam update).

1. harvest: run hot-spot events with the tabulated EOS (closed-form seed) for
   a few steps and take the conserved states of their cells, keeping those in
   the network's range (E above hydro_mlp_seed_emin, where the EOS departs
   from p = e/3);
2. label: solve cons->prim for them with the plain Newton solve (FP64, v0 = 0);
3. train: fit the network to (ln E, |M|/E) -> v on the GPU.
"""
from __future__ import annotations

import numpy as np

from . import hydro
from . import inputs as I


def harvest_states(table, n=64, events=(0, 1), steps=4, flow_max=0.5, stream=None,
                   keep_all=False):
    """Conserved states [4][N] (float64, host) of the cells of hot-spot events
    (n^3, dx 0.1 fm, outflow, FP64, the tabulated EOS) after `steps` steps,
    restricted to E above the network's range start unless keep_all; and
    that start."""
    import torch
    g = I.event_grid(n, 0.1)
    grids = [hydro.make_grid(n, n, n, dx=0.1, x0=g["x0"], y0=g["y0"], z0=g["z0"],
                             bc="outflow", prec="fp64", cfl=0.4) for _ in events]
    b = hydro.Batch(grids, hydro.make_eos(table, seed="conformal"), stream=stream)
    b.init_hotspots(np.stack([I.hotspots(e, flow_max=flow_max) for e in events]),
                    I.SPOT_SIGMA, I.E_BACKGROUND)
    b.step(steps)
    torch.cuda.synchronize()
    h = hydro.Hydro(hydro.make_grid(8, dx=1.0, prec="fp64"), hydro.make_eos(table))
    emin = h.mlp_seed_emin()
    states = []
    for e in range(len(events)):
        U = b.get_conserved(e).reshape(4, -1)
        states.append(U if keep_all else U[:, U[0] > emin])
    return np.concatenate(states, axis=1), emin


def solver_pairs(table, U):
    """(X, v, iterations): inputs (ln E, |M|/E) and the plain Newton root
    (FP64, v0 = 0) of the states U [4][N] on the device."""
    import torch
    n = U.shape[1]
    h = hydro.Hydro(hydro.make_grid(8, dx=1.0, prec="fp64"), hydro.make_eos(table, seed="zero"))
    Ud = torch.tensor(np.ascontiguousarray(U), dtype=torch.float64, device="cuda")
    v = torch.empty(n, dtype=torch.float64, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    h.c2p_newton(Ud, "zero", v, it)
    E, M = U[0], np.linalg.norm(U[1:], axis=0)
    X = np.column_stack([np.log(E), M / E])
    return X, v.cpu().numpy(), it.cpu().numpy()


def train_seed(X, Y, epochs=150, batch=512, lr=3e-3, seed=13, shuffle_seed=7):
    """Train the seed network on the GPU (Adam, half-cosine learning rate);
    returns (parameters, loss per epoch)."""
    import torch
    rng = np.random.default_rng(seed)
    P = rng.normal(size=hydro.mlp_nparam()) * 0.3
    P[-4:] = [X[:, 0].mean(), X[:, 0].std() + 1e-12, X[:, 1].mean(), X[:, 1].std() + 1e-12]
    params = torch.tensor(P, dtype=torch.float32, device="cuda")
    hist = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    hydro.mlp_train(params, torch.tensor(X, dtype=torch.float32, device="cuda"),
                    torch.tensor(Y, dtype=torch.float32, device="cuda"), batch, epochs, lr,
                    shuffle_seed, hist)
    torch.cuda.synchronize()
    return params.cpu().numpy(), hist.cpu().numpy()


def seed_iterations(table, params, U, prec="fp32"):
    """Mean Newton iterations per solve of the states U for each seed (zero,
    conformal, mlp), and the largest root difference of mlp against zero."""
    import torch
    h = hydro.Hydro(hydro.make_grid(8, dx=1.0, prec=prec),
                    hydro.make_eos(table, seed="mlp", mlp_params=params))
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ud = torch.tensor(np.ascontiguousarray(U), dtype=dt, device="cuda")
    n = U.shape[1]
    out, roots = {}, {}
    for s in ("zero", "conformal", "mlp"):
        v = torch.empty(n, dtype=dt, device="cuda")
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        h.c2p_newton(Ud, s, v, it)
        out[s] = float(it.double().mean().item())
        roots[s] = v.cpu().numpy().astype(np.float64)
    return out, float(np.abs(roots["mlp"] - roots["zero"]).max())
