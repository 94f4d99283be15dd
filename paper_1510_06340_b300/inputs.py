"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds only workload recipes -- grids, initial primitive fields
(e, v), hot-spot lists, jet parameters, the equation-of-state table -- and
none of the method's arithmetic (no prim<->cons transform, no flux, no
limiter).  Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), so any side can reproduce a draw from (seed, stream, index).

The paper runs on external heavy-ion initial-condition models (Sec. 2.2);
the hot-spot recipe below is a synthetic stand-in for Monte-Carlo Glauber
events: 416 = 2 x 208 nucleon-sized Gaussians (sigma 0.5 fm) in a disc of
radius 6.6 fm (about a lead nucleus), on a zero-velocity background.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

BASE_SEED = 20151020
_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """U[0,1) doubles: SplitMix64 output for counter `index` of key (seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream + 1) * _G)
        idx = np.asarray(index, dtype=np.uint64)
        z = _mix(key + (idx + np.uint64(1)) * _G)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# grids and simple initial states
# --------------------------------------------------------------------------
def cell_centres(n: int, lo: float, dx: float) -> np.ndarray:
    return lo + (np.arange(n) + 0.5) * dx


def shock_tube(n: int = 1000, e_left: float = 10.0, e_right: float = 1.0):
    """1-D Riemann problem on [-1, 1]: e_L for x < 0, e_R for x > 0, v = 0."""
    dx = 2.0 / n
    x = cell_centres(n, -1.0, dx)
    e = np.where(x < 0.0, e_left, e_right).reshape(1, 1, n)
    z = np.zeros_like(e)
    return dict(nx=n, ny=1, nz=1, dx=dx, x0=-1.0, y0=0.0, z0=0.0), (e, z, z.copy(), z.copy())


def spherical_blast(n: int = 256, e_in: float = 10.0, e_out: float = 1.0, radius: float = 0.2):
    """3-D blast on [-1, 1]^3: e_in inside r < radius, e_out outside, v = 0."""
    dx = 2.0 / n
    c = cell_centres(n, -1.0, dx)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    e = np.where(x * x + y * y + z * z < radius * radius, e_in, e_out)
    zero = np.zeros_like(e)
    return dict(nx=n, ny=n, nz=n, dx=dx, x0=-1.0, y0=-1.0, z0=-1.0), (e, zero, zero.copy(),
                                                                      zero.copy())


# --------------------------------------------------------------------------
# event-by-event hot-spot workload
# --------------------------------------------------------------------------
HOTSPOTS = 416
SPOT_SIGMA = 0.5      # fm
SPOT_AMPL = 2.0       # GeV/fm^3
DISC_RADIUS = 6.6     # fm
E_BACKGROUND = 0.01   # GeV/fm^3
JET_DEDX = 5.0        # GeV/fm
JET_SIGMA = 0.3       # fm


def event_sizes(nevents: int, lo: int = 64, hi: int = 160, seed: int = BASE_SEED) -> np.ndarray:
    """Cubic grid edge per event, uniform on {lo..hi}."""
    u = uniform(seed, 0, np.arange(nevents))
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def hotspots(event: int, nspots: int = HOTSPOTS, flow_max: float = 0.0,
             seed: int = BASE_SEED) -> np.ndarray:
    """Per hot spot: (cx, cy, cz, amplitude, ux, uy, uz).

    Centres are uniform in the disc of radius DISC_RADIUS at z = 0; with
    flow_max > 0 each spot carries a velocity uniform in the ball |u| <= flow_max.
    """
    i = np.arange(nspots, dtype=np.uint64) * np.uint64(8)
    s = 1000 + event
    r = DISC_RADIUS * np.sqrt(uniform(seed, s, i))
    th = 2.0 * np.pi * uniform(seed, s, i + np.uint64(1))
    out = np.zeros((nspots, 7))
    out[:, 0] = r * np.cos(th)
    out[:, 1] = r * np.sin(th)
    out[:, 3] = SPOT_AMPL
    if flow_max > 0.0:
        rad = flow_max * np.cbrt(uniform(seed, s, i + np.uint64(2)))
        ct = 2.0 * uniform(seed, s, i + np.uint64(3)) - 1.0
        ph = 2.0 * np.pi * uniform(seed, s, i + np.uint64(4))
        st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
        out[:, 4] = rad * st * np.cos(ph)
        out[:, 5] = rad * st * np.sin(ph)
        out[:, 6] = rad * ct
    return out


def jet(event: int, seed: int = BASE_SEED) -> np.ndarray:
    """(x0, y0, z0, nx, ny, nz, dE/dx, sigma): start uniform in the disc, direction in xy."""
    s = 500000 + event
    u = uniform(seed, s, np.arange(3))
    r = DISC_RADIUS * math.sqrt(u[0])
    th = 2.0 * math.pi * u[1]
    ph = 2.0 * math.pi * u[2]
    return np.array([r * math.cos(th), r * math.sin(th), 0.0, math.cos(ph), math.sin(ph), 0.0,
                     JET_DEDX, JET_SIGMA])


def event_grid(n: int, dx: float = 0.1):
    """Cubic grid of edge n centred on the origin."""
    lo = -0.5 * n * dx
    return dict(nx=n, ny=n, nz=n, dx=dx, x0=lo, y0=lo, z0=lo)


def hotspot_primitives(grid: dict, spots: np.ndarray, sigma: float = SPOT_SIGMA,
                       e_bg: float = E_BACKGROUND):
    """e = e_bg + sum_j A_j g_j,  v = sum_j A_j g_j u_j / e  (|v| <= max |u_j|)."""
    xs = cell_centres(grid["nx"], grid["x0"], grid["dx"])
    ys = cell_centres(grid["ny"], grid["y0"], grid["dx"])
    zs = cell_centres(grid["nz"], grid["z0"], grid["dx"])
    shape = (grid["nz"], grid["ny"], grid["nx"])
    e = np.full(shape, e_bg)
    px = np.zeros(shape)
    py = np.zeros(shape)
    pz = np.zeros(shape)
    inv = 1.0 / (2.0 * sigma * sigma)
    for s in spots:
        gx = np.exp(-(xs - s[0]) ** 2 * inv)
        gy = np.exp(-(ys - s[1]) ** 2 * inv)
        gz = np.exp(-(zs - s[2]) ** 2 * inv)
        g = s[3] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        e += g
        if s[4] or s[5] or s[6]:
            px += g * s[4]
            py += g * s[5]
            pz += g * s[6]
    return e, px / e, py / e, pz / e


# --------------------------------------------------------------------------
# tabulated non-conformal equation of state
# --------------------------------------------------------------------------
EOS_E0 = 0.5
EOS_W = 0.5


def eos_cs2_exact(e):
    """c_s^2(e) = 1/3 - 0.25 exp(-(ln(e/e0))^2 / w)."""
    le = np.log(np.asarray(e, dtype=np.float64) / EOS_E0)
    return 1.0 / 3.0 - 0.25 * np.exp(-le * le / EOS_W)


def eos_p_exact(e):
    """p(e) = int_0^e c_s^2 de' in closed form (substitute u = ln(e'/e0)):
    p = e/3 - (1/8) e0 exp(w/4) sqrt(pi w) [1 + erf((ln(e/e0) - w/2)/sqrt(w))]."""
    e = np.asarray(e, dtype=np.float64)
    le = np.log(e / EOS_E0)
    return e / 3.0 - 0.125 * EOS_E0 * math.exp(EOS_W / 4.0) * math.sqrt(math.pi * EOS_W) * (
        1.0 + erf((le - EOS_W / 2.0) / math.sqrt(EOS_W)))


def eos_table(n: int = 4096, lne_min: float = math.log(1e-6), lne_max: float = math.log(1e4)):
    """Nodes uniform in ln e; returns the dict the solver and the oracle take."""
    lne = np.linspace(lne_min, lne_max, n)
    e = np.exp(lne)
    return dict(n=n, lne_min=lne_min, lne_max=lne_max, cs2=eos_cs2_exact(e), p=eos_p_exact(e))
