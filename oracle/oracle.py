"""Python handle on the plain FP64 CPU oracle (``musta_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  Nothing here imports the
CUDA package; the oracle shares no code with it.  Arithmetic lives in the C
file; this module only marshals numpy arrays through ctypes.

Every function here is pinned by a CPU test; the MLP forward pass through
special cases that reduce to matrix products, its gradient by finite
differences.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "musta_oracle.c")
_LIB = os.path.join(_HERE, "libmusta_oracle.so")
# the same source with its pencil loops split over threads (timing only)
_LIB_OMP = os.path.join(_HERE, "libmusta_oracle_omp.so")
# the same source compiled as C++ with an operation-counting double
_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_LIB_OPC = os.path.join(_HERE, "libmusta_opcount.so")

LIMITERS = {"none": 0, "minmod": 1, "mc": 2, "superbee": 3, "vanleer": 4, "vanalbada": 5}
BC = {"periodic": 0, "outflow": 1}


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s)
                                          for s in srcs)


def _compile(cmd, lib):
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(cmd + ["-o", tmp])
    os.replace(tmp, lib)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction),
    its OpenMP timing build and its op-counting build."""
    if force or _stale(_LIB, [_SRC]):
        _compile(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-ffp-contract=off",
                  "-shared", _SRC, "-lm"], _LIB)
    if force or _stale(_LIB_OMP, [_SRC]):
        _compile(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-ffp-contract=off",
                  "-fopenmp", "-DOR_OPENMP", "-shared", _SRC, "-lm"], _LIB_OMP)
    if force or _stale(_LIB_OPC, [_SRC, _OPC_SRC]):
        _compile(["g++", "-O1", "-std=c++17", "-D_DEFAULT_SOURCE", "-fPIC", "-ffp-contract=off",
                  "-shared", _OPC_SRC], _LIB_OPC)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
        ("bc", C.c_int * 3),
        ("limiter", C.c_int), ("stages", C.c_int), ("rk_order", C.c_int), ("hancock", C.c_int),
        ("alpha", C.c_double), ("cfl", C.c_double), ("fixed_dt", C.c_double),
        ("delta", C.c_double),
        ("eos_kind", C.c_int), ("cs2", C.c_double),
        ("tab_n", C.c_int), ("lne_min", C.c_double), ("lne_max", C.c_double),
        ("cs2_tab", C.POINTER(C.c_double)), ("p_tab", C.POINTER(C.c_double)),
        ("seed_kind", C.c_int), ("mlp", C.POINTER(C.c_double)), ("mlp_quantize", C.c_int),
        ("newton_tol", C.c_double),
        ("jet_on", C.c_int), ("jet", C.c_double * 8),
        ("unsplit", C.c_int), ("charge", C.c_int),
    ]


_lib = None
_lib_omp = None
_lib_opc = None
_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def lib_omp():
    """The OpenMP timing build (pencils of a sweep split over all host threads);
    the same arithmetic per pencil, without the diagnostics counters."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = _bind(C.CDLL(_LIB_OMP))
    return _lib_omp


def _bind(L):
    if True:
        P = C.POINTER(_Cfg)
        L.or_limiter.restype = C.c_double
        L.or_limiter.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_cons2prim.restype = C.c_int
        L.or_cons2prim.argtypes = [P, _dp, _dp, _dp, _dp, C.POINTER(C.c_int)]
        L.or_prim2cons.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        L.or_flux.argtypes = [P, C.c_int, _dp, _dp]
        L.or_musta_force.argtypes = [P, C.c_int, C.c_double, _dp, _dp, _dp]
        L.or_hancock_faces.argtypes = [P, C.c_int, C.c_double, _dp, _dp, _dp, _dp, _dp]
        L.or_sweep.argtypes = [P, _dp, C.c_int, C.c_double]
        L.or_signal_speed.restype = C.c_double
        L.or_signal_speed.argtypes = [P, _dp, C.c_int]
        L.or_max_rate.restype = C.c_double
        L.or_max_rate.argtypes = [P, _dp]
        L.or_max_rate_unsplit.restype = C.c_double
        L.or_max_rate_unsplit.argtypes = [P, _dp]
        L.or_jet_source.argtypes = [P, _dp, C.c_double, C.c_double]
        L.or_step.restype = C.c_double
        L.or_step.argtypes = [P, _dp, C.c_double, C.c_double]
        L.or_run.restype = C.c_int
        L.or_run.argtypes = [P, _dp, C.c_int, C.c_double, _dp]
        L.or_conservation_sums.argtypes = [P, _dp, _dp]
        L.or_prim2cons_field.argtypes = [P, C.c_long, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_prim2cons_n.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double, _dp]
        L.or_charge_density_field.argtypes = [P, C.c_long, _dp, _dp]
        L.or_cons2prim_field.argtypes = [P, C.c_long, _dp, _dp, _dp, _dp, _dp,
                                         C.POINTER(C.c_int)]
        L.or_eos_p.restype = C.c_double
        L.or_eos_p.argtypes = [P, C.c_double]
        L.or_eos_cs2.restype = C.c_double
        L.or_eos_cs2.argtypes = [P, C.c_double]
        L.or_mlp_nparam.restype = C.c_int
        L.or_round_bf16.restype = C.c_double
        L.or_round_bf16.argtypes = [C.c_double]
        L.or_mlp_forward.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp]
        L.or_mlp_hidden.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp]
        L.or_mlp_forward_h1.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, _dp]
        L.or_mlp_loss_grad.restype = C.c_double
        L.or_mlp_loss_grad.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, _dp]
        L.or_get_counters.argtypes = [C.POINTER(C.c_long)]
        L.or_threads.restype = C.c_int
    return L


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Oracle:
    """One grid plus scheme parameters; methods mirror the C entry points."""

    def __init__(self, nx, ny=1, nz=1, dx=1.0, dy=None, dz=None, x0=0.0, y0=0.0, z0=0.0,
                 bc=("periodic", "periodic", "periodic"), limiter="minmod", stages=2,
                 rk_order=2, hancock=1, alpha=1.0, cfl=0.4, fixed_dt=0.0, delta=1e-12, eos=None,
                 cs2=1.0 / 3.0, seed_kind=0, mlp=None, mlp_quantize=0, newton_tol=1e-13,
                 jet=None, unsplit=0, charge=0):
        self.keep = []
        c = _Cfg()
        c.nx, c.ny, c.nz = nx, ny, nz
        c.dx = dx
        c.dy = dx if dy is None else dy
        c.dz = dx if dz is None else dz
        c.x0, c.y0, c.z0 = x0, y0, z0
        if isinstance(bc, str):
            bc = (bc, bc, bc)
        for i in range(3):
            c.bc[i] = BC[bc[i]] if isinstance(bc[i], str) else int(bc[i])
        c.limiter = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
        c.stages, c.rk_order, c.hancock = stages, rk_order, hancock
        c.alpha, c.cfl, c.fixed_dt, c.delta = alpha, cfl, fixed_dt, delta
        c.cs2 = cs2
        if eos is None:
            c.eos_kind = 0
        else:
            c.eos_kind = 1
            cs2_tab = np.ascontiguousarray(eos["cs2"], dtype=np.float64)
            p_tab = np.ascontiguousarray(eos["p"], dtype=np.float64)
            self.keep += [cs2_tab, p_tab]
            c.tab_n = len(p_tab)
            c.lne_min, c.lne_max = eos["lne_min"], eos["lne_max"]
            c.cs2_tab, c.p_tab = _ptr(cs2_tab), _ptr(p_tab)
        c.seed_kind = seed_kind
        if mlp is not None:
            m = np.ascontiguousarray(mlp, dtype=np.float64)
            self.keep.append(m)
            c.mlp = _ptr(m)
        c.mlp_quantize = mlp_quantize
        c.newton_tol = newton_tol
        if jet is not None:
            c.jet_on = 1
            for i in range(8):
                c.jet[i] = float(jet[i])
        c.unsplit = int(unsplit)
        c.charge = int(charge)
        self.c = c
        self.nq = 5 if charge else 4
        self.shape = (self.nq, nz, ny, nx)

    @property
    def cells(self):
        return self.c.nx * self.c.ny * self.c.nz

    # --- pointwise pieces -------------------------------------------------
    def limiter(self, a, b):
        return lib().or_limiter(self.c.limiter, a, b)

    def cons2prim(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        e, p = C.c_double(), C.c_double()
        v = np.zeros(3)
        it = C.c_int()
        st = lib().or_cons2prim(C.byref(self.c), _ptr(U), C.byref(e), _ptr(v), C.byref(p),
                                C.byref(it))
        return e.value, v, p.value, st, it.value

    def prim2cons(self, e, v, n=0.0):
        U = np.zeros(self.nq)
        lib().or_prim2cons_n(C.byref(self.c), e, v[0], v[1], v[2], n, _ptr(U))
        return U

    def flux(self, d, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.size >= self.nq
        F = np.zeros(self.nq)
        lib().or_flux(C.byref(self.c), d, _ptr(U), _ptr(F))
        return F

    def musta_force(self, d, lam, UL, UR):
        UL = np.ascontiguousarray(UL, dtype=np.float64)
        UR = np.ascontiguousarray(UR, dtype=np.float64)
        assert UL.size >= self.nq and UR.size >= self.nq
        F = np.zeros(self.nq)
        lib().or_musta_force(C.byref(self.c), d, lam, _ptr(UL), _ptr(UR), _ptr(F))
        return F

    def signal_speed(self, U, d):
        U = np.ascontiguousarray(U, dtype=np.float64)
        return lib().or_signal_speed(C.byref(self.c), _ptr(U), d)

    def eos_p(self, e):
        return lib().or_eos_p(C.byref(self.c), e)

    def eos_cs2(self, e):
        return lib().or_eos_cs2(C.byref(self.c), e)

    # --- whole-field operations --------------------------------------------
    def prim2cons_field(self, e, vx, vy, vz, n=None):
        """Conserved fields from (e, v) and, with the charge, the rest-frame
        charge density n (None: zero)."""
        cells = self.cells
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (e, vx, vy, vz)]
        nn = None
        if n is not None:
            nn = np.ascontiguousarray(n, dtype=np.float64).reshape(-1)
            assert nn.size == cells
        U = np.zeros(self.shape)
        lib().or_prim2cons_field(C.byref(self.c), cells, *[_ptr(a) for a in arrs],
                                 _ptr(nn) if nn is not None else None, _ptr(U))
        return U

    def charge_density_field(self, U):
        """n = R / gamma per cell (needs charge=1)."""
        assert self.nq == 5
        U = np.ascontiguousarray(U, dtype=np.float64)
        n = np.zeros(self.shape[1:])
        lib().or_charge_density_field(C.byref(self.c), self.cells, _ptr(U), _ptr(n))
        return n

    def cons2prim_field(self, U):
        n = self.cells
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = [np.zeros(self.shape[1:]) for _ in range(4)]
        it = np.zeros(self.shape[1:], dtype=np.int32)
        lib().or_cons2prim_field(C.byref(self.c), n, _ptr(U), *[_ptr(a) for a in out],
                                 it.ctypes.data_as(C.POINTER(C.c_int)))
        return out[0], out[1], out[2], out[3], it

    def sweep(self, U, d, dt):
        assert U.shape == self.shape
        lib().or_sweep(C.byref(self.c), _ptr(U), d, dt)

    def max_rate(self, U):
        """The rate whose inverse times cfl is dt: max over axes (split) or the
        sum over axes (unsplit, R16c)."""
        self._field(U)
        if self.c.unsplit:
            return lib().or_max_rate_unsplit(C.byref(self.c), _ptr(U))
        return lib().or_max_rate(C.byref(self.c), _ptr(U))

    def jet_source(self, U, t, dt):
        lib().or_jet_source(C.byref(self.c), _ptr(U), t, dt)

    def _field(self, U):
        assert U.dtype == np.float64 and U.size == self.nq * self.cells, (U.shape, self.shape)

    def step(self, U, t=0.0, t_end=0.0):
        self._field(U)
        return lib().or_step(C.byref(self.c), _ptr(U), t, t_end)

    def run(self, U, nsteps, t_end=0.0, t=0.0, threads=False):
        """Advance U in place; threads=True runs the OpenMP timing build."""
        self._field(U)
        tt = C.c_double(t)
        L = lib_omp() if threads else lib()
        n = L.or_run(C.byref(self.c), _ptr(U), nsteps, t_end, C.byref(tt))
        return n, tt.value

    def conservation_sums(self, U):
        self._field(U)
        out = np.zeros(self.nq)
        lib().or_conservation_sums(C.byref(self.c), _ptr(U), _ptr(out))
        return out


def counters():
    out = (C.c_long * 5)()
    lib().or_get_counters(out)
    keys = ("newton_calls", "newton_iters", "newton_fail", "capped", "face_fallback")
    return dict(zip(keys, list(out)))


def reset_counters():
    lib().or_reset_counters()


def mlp_nparam():
    return lib().or_mlp_nparam()


def round_bf16(x):
    return lib().or_round_bf16(float(x))


def mlp_forward(params, X, quantize=0):
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0])
    lib().or_mlp_forward(_ptr(P), quantize, X.shape[0], _ptr(X), _ptr(out))
    return out


def mlp_hidden(params, X, quantize=0):
    """First-layer activations [n][32] (bf16-rounded with quantize=1)."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    H1 = np.zeros((X.shape[0], 32))
    lib().or_mlp_hidden(_ptr(P), quantize, X.shape[0], _ptr(X), _ptr(H1))
    return H1


def mlp_forward_h1(params, X, H1, quantize=0):
    """Layers 2 and 3 of the forward fed with the given activations H1 [n][32]."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    H1 = np.ascontiguousarray(H1, dtype=np.float64)
    out = np.zeros(X.shape[0])
    lib().or_mlp_forward_h1(_ptr(P), quantize, X.shape[0], _ptr(X), _ptr(H1), _ptr(out))
    return out


def mlp_loss_grad(params, X, Y, quantize=0):
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    G = np.zeros_like(P)
    loss = lib().or_mlp_loss_grad(_ptr(P), quantize, X.shape[0], _ptr(X), _ptr(Y), _ptr(G))
    return loss, G


# ------------------------------------------------------------ op counting
OP_KINDS = ("leaf", "add", "sub", "mul", "div", "sqrt", "min", "max", "exp", "log", "tanh",
            "abs", "neg", "floor")
FLOP_KINDS = ("add", "sub", "mul", "div", "sqrt", "min", "max")


def _opc():
    global _lib_opc
    if _lib_opc is None:
        build()
        L = C.CDLL(_LIB_OPC)
        L.or_opcount_nkind.restype = C.c_int
        L.or_opcount_sweep.restype = C.c_int
        L.or_opcount_sweep.argtypes = [C.c_int] * 6 + [C.POINTER(C.c_longlong)]
        L.or_opcount_unsplit.restype = C.c_int
        L.or_opcount_unsplit.argtypes = [C.c_int] * 4 + [C.POINTER(C.c_longlong)]
        assert L.or_opcount_nkind() == len(OP_KINDS)
        _lib_opc = L
    return _lib_opc


def opcount_sweep(limiter="minmod", stages=2, rk_order=2, hancock=1, n1=32, n2=64):
    """Operations per cell of one oracle sweep (conformal EOS), by kind, from
    the op-counting build: distinct operations on state-derived values that
    the output depends on.  'flops' sums FLOP_KINDS."""
    out = (C.c_longlong * len(OP_KINDS))()
    lim = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
    rc = _opc().or_opcount_sweep(lim, stages, rk_order, hancock, n1, n2, out)
    if rc != 0:
        raise RuntimeError("operation count is not a whole number per cell")
    d = dict(zip(OP_KINDS, out[:]))
    d["flops"] = sum(d[k] for k in FLOP_KINDS)
    return d


def opcount_unsplit(stages=2, rk_order=2, hancock=1, n=8):
    """Operations per cell and RK stage of the unsplit scheme, counted the same way."""
    out = (C.c_longlong * len(OP_KINDS))()
    rc = _opc().or_opcount_unsplit(stages, rk_order, hancock, n, out)
    if rc != 0:
        raise RuntimeError("operation count is not a whole number per cell and stage")
    d = dict(zip(OP_KINDS, out[:]))
    d["flops"] = sum(d[k] for k in FLOP_KINDS)
    return d
