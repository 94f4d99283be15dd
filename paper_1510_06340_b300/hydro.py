"""ctypes binding of libhydro.so (include/hydro.h).  Argument marshalling only.

Arrays may be numpy arrays (host, on_device=0) or CUDA torch tensors (device,
on_device=1).  The element type must match the handle's precision: float64
for "fp64", float32 for "fp32" and "mixed".  Every call raises HydroError on a
non-zero status; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhydro.so")

LIMITERS = {"none": 0, "minmod": 1, "mc": 2, "superbee": 3, "vanleer": 4, "vanalbada": 5}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}
BCS = {"periodic": 0, "outflow": 1}
SEEDS = {"zero": 0, "conformal": 1, "mlp": 2}
STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "UNPHYSICAL", 5: "NEWTON",
          6: "NONFINITE"}
COUNTERS = ("capped", "face_fallback", "newton_calls", "newton_iters", "newton_fail", "f64_redo")
FLAG_NEWTON, FLAG_UNPHYSICAL = 1, 2


class HydroError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hydro status {STATUS.get(status, status)}: {msg}")
        self.status = status


class GridT(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("bc", C.c_int * 3), ("prec", C.c_int), ("rk_order", C.c_int),
                ("hancock", C.c_int), ("cfl", C.c_double), ("fixed_dt", C.c_double),
                ("alpha", C.c_double), ("unsplit", C.c_int), ("charge", C.c_int)]


class EosT(C.Structure):
    _fields_ = [("kind", C.c_int), ("cs2", C.c_double), ("n", C.c_int),
                ("lne_min", C.c_double), ("lne_max", C.c_double),
                ("cs2_tab", C.POINTER(C.c_double)), ("p_tab", C.POINTER(C.c_double)),
                ("seed", C.c_int), ("mlp_params", C.POINTER(C.c_float)),
                ("newton_tol", C.c_double), ("newton_max_iter", C.c_int)]


_lib = None


def lib():
    """Load libhydro.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_1510_06340_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, ip, dp, i, d = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int, C.c_double
        H = C.c_void_p
        L.hydro_last_error.restype = C.c_char_p
        sig = {
            "hydro_create": [C.POINTER(GridT), C.POINTER(EosT), i, i, C.POINTER(H)],
            "hydro_set_stream": [H, vp],
            "hydro_set_primitives": [H, vp, vp, vp, vp, i],
            "hydro_set_conserved": [H, vp, i],
            "hydro_set_primitives_charged": [H, vp, vp, vp, vp, vp, i],
            "hydro_get_charge_density": [H, vp, i],
            "hydro_charge_sum": [H, dp],
            "hydro_batch_set_primitives_charged": [H, i, vp, vp, vp, vp, vp, i],
            "hydro_batch_charge_sums": [H, dp],
            "hydro_get_conserved": [H, vp, i],
            "hydro_get_primitives": [H, vp, vp, vp, vp, i],
            "hydro_init_hotspots": [H, dp, i, d, d],
            "hydro_set_jet": [H, dp],
            "hydro_step": [H, i, d, dp],
            "hydro_sweep": [H, i, d],
            "hydro_max_rate": [H, dp],
            "hydro_conservation_sums": [H, dp],
            "hydro_get_time": [H, dp],
            "hydro_set_time": [H, d],
            "hydro_enable_counters": [H, i],
            "hydro_counters": [H, C.POINTER(C.c_longlong)],
            "hydro_check_finite": [H],
            "hydro_check_status": [H, C.POINTER(C.c_uint)],
            "hydro_batch_event_flags": [H, ip, C.POINTER(C.c_uint)],
            "hydro_force_launch": [H, i, i, i],
            "hydro_set_kernel_timing": [H, i],
            "hydro_get_kernel_timing": [H, dp, C.POINTER(C.c_longlong)],
            "hydro_batch_set_kernel_timing": [H, i],
            "hydro_batch_get_kernel_timing": [H, dp, C.POINTER(C.c_longlong)],
            "hydro_get_launch": [H, i, ip, ip],
            "hydro_c2p_newton": [H, vp, i, i, vp, vp],
            "hydro_c2p_newton_pairs": [H, vp, i, i, i, vp, vp, vp],
            "hydro_mlp_seed_emin": [H, dp],
            "hydro_batch_create": [C.POINTER(GridT), i, C.POINTER(EosT), i, i, C.POINTER(H)],
            "hydro_batch_set_stream": [H, vp],
            "hydro_batch_init_hotspots": [H, dp, i, d, d],
            "hydro_batch_set_primitives": [H, i, vp, vp, vp, vp, i],
            "hydro_batch_set_jets": [H, dp],
            "hydro_batch_step": [H, i, i],
            "hydro_batch_set_conserved": [H, i, vp, i],
            "hydro_batch_get_conserved": [H, i, vp, i],
            "hydro_batch_get_primitives": [H, i, vp, vp, vp, vp, i],
            "hydro_batch_times": [H, dp],
            "hydro_batch_conservation_sums": [H, dp],
            "hydro_batch_event_status": [H, ip],
            "hydro_batch_enable_counters": [H, i],
            "hydro_batch_counters": [H, C.POINTER(C.c_longlong)],
            "hydro_conservation_sums_noalloc": [vp, i, i, i, i, d, d, d, dp, vp],
            "hydro_mlp_forward": [vp, vp, i, vp, vp],
            "hydro_mlp_hidden": [vp, vp, i, vp, vp],
            "hydro_mlp_loss_grad": [vp, vp, vp, i, vp, vp, vp],
            "hydro_mlp_train": [vp, vp, vp, i, i, i, C.c_float, C.c_ulonglong, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.hydro_destroy.argtypes = [H]
        L.hydro_destroy.restype = None
        L.hydro_batch_destroy.argtypes = [H]
        L.hydro_batch_destroy.restype = None
        L.hydro_mlp_nparam.restype = C.c_int
        L.hydro_mlp_nparam.argtypes = []
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise HydroError(status, lib().hydro_last_error().decode())


def _is_tensor(a):
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


_TORCH_DTYPES = {np.float64: "torch.float64", np.float32: "torch.float32",
                 np.int32: "torch.int32"}


def _arg(a, dtype, numel=None):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA tensor.
    numel: the element count the call reads or writes; a shorter buffer is
    rejected before any pointer reaches the library."""
    if _is_tensor(a):
        if not a.is_cuda:
            a = a.numpy()
        else:
            want = _TORCH_DTYPES[dtype]
            if str(a.dtype) != want:
                raise TypeError(f"tensor dtype {a.dtype}, expected {want}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if numel is not None and a.numel() < numel:
                raise ValueError(f"tensor holds {a.numel()} elements, the call needs {numel}")
            return C.c_void_p(a.data_ptr()), 1, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if numel is not None and arr.size < numel:
        raise ValueError(f"array holds {arr.size} elements, the call needs {numel}")
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _dev(t, dtype, numel, name="tensor"):
    """Pointer of a CUDA tensor that a device-only call reads or writes:
    checked for device, dtype, contiguity and size first."""
    if not _is_tensor(t) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    want = _TORCH_DTYPES[dtype]
    if str(t.dtype) != want:
        raise TypeError(f"{name} dtype {t.dtype}, expected {want}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {numel}")
    return C.c_void_p(t.data_ptr())


def _out_arg(o, dtype, numel=None):
    """_arg for an output: a host output must be written in place."""
    p, dev, keep = _arg(o, dtype, numel)
    if not dev:
        base = o.numpy() if _is_tensor(o) else o
        if not (isinstance(base, np.ndarray) and np.shares_memory(keep, base)):
            raise ValueError("host output must be a contiguous array of the handle's dtype")
    return p, dev, keep


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def make_grid(nx, ny=1, nz=1, dx=1.0, dy=None, dz=None, x0=0.0, y0=0.0, z0=0.0,
              bc="periodic", prec="fp64", rk_order=2, hancock=1, cfl=0.4, fixed_dt=0.0,
              alpha=None, unsplit=False, charge=False):
    """hydro_grid_t; alpha defaults to 1 for split sweeps and 3 for the
    unsplit scheme (the paper's 3-D value)."""
    g = GridT()
    g.nx, g.ny, g.nz = nx, ny, nz
    g.dx = dx
    g.dy = dx if dy is None else dy
    g.dz = dx if dz is None else dz
    g.x0, g.y0, g.z0 = x0, y0, z0
    if isinstance(bc, str):
        bc = (bc, bc, bc)
    for k in range(3):
        g.bc[k] = BCS[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    g.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    g.rk_order, g.hancock = rk_order, hancock
    g.cfl, g.fixed_dt = cfl, fixed_dt
    g.alpha = (3.0 if unsplit else 1.0) if alpha is None else alpha
    g.unsplit = 1 if unsplit else 0
    g.charge = 1 if charge else 0
    return g


def make_eos(table=None, cs2=1.0 / 3.0, seed="zero", mlp_params=None, newton_tol=0.0,
             newton_max_iter=0):
    """Conformal EOS (table=None) or a table dict from inputs.eos_table()."""
    e = EosT()
    keep = []
    if table is None:
        e.kind, e.cs2 = 0, cs2
    else:
        e.kind = 1
        c2 = np.ascontiguousarray(table["cs2"], dtype=np.float64)
        p = np.ascontiguousarray(table["p"], dtype=np.float64)
        keep += [c2, p]
        e.n = len(p)
        e.lne_min, e.lne_max = table["lne_min"], table["lne_max"]
        e.cs2_tab = c2.ctypes.data_as(C.POINTER(C.c_double))
        e.p_tab = p.ctypes.data_as(C.POINTER(C.c_double))
    e.seed = SEEDS[seed] if isinstance(seed, str) else int(seed)
    if mlp_params is not None:
        m = np.ascontiguousarray(mlp_params, dtype=np.float32)
        keep.append(m)
        e.mlp_params = m.ctypes.data_as(C.POINTER(C.c_float))
    e.newton_tol = newton_tol
    e.newton_max_iter = newton_max_iter
    return e, keep


class _Base:
    _dtype = np.float64

    def _t(self):
        return self._dtype

    @property
    def dtype(self):
        return self._dtype


class Hydro(_Base):
    """One grid: hydro_create ... hydro_destroy."""

    def __init__(self, grid: GridT, eos=None, limiter="minmod", stages=2, stream=None):
        eos_t, self._keep = (eos if eos is not None else make_eos())
        self.grid = grid
        h = C.c_void_p()
        lim = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
        _check(lib().hydro_create(C.byref(grid), C.byref(eos_t), lim, stages, C.byref(h)))
        self.h = h
        self._dtype = np.float64 if grid.prec == 0 else np.float32
        self.nq = 5 if grid.charge else 4
        self.shape = (self.nq, grid.nz, grid.ny, grid.nx)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "h", None):
            lib().hydro_destroy(self.h)
            self.h = None

    __del__ = close

    def set_stream(self, stream):
        _check(lib().hydro_set_stream(self.h, _stream_ptr(stream)))

    @property
    def cells(self):
        return self.grid.nx * self.grid.ny * self.grid.nz

    def set_primitives(self, e, vx, vy, vz, n=None):
        """(e, v) and, on a charged handle, the rest-frame charge density n."""
        fields = (e, vx, vy, vz) if n is None else (e, vx, vy, vz, n)
        args = [_arg(a, self._dtype, self.cells) for a in fields]
        if len({a[1] for a in args}) != 1:
            raise ValueError("inputs must be all on the host or all on the device")
        if n is None:
            _check(lib().hydro_set_primitives(self.h, *[a[0] for a in args], args[0][1]))
        else:
            _check(lib().hydro_set_primitives_charged(self.h, *[a[0] for a in args],
                                                      args[0][1]))

    def charge_density(self, out=None):
        """n = R / gamma [nz][ny][nx] (charged handles)."""
        if out is None:
            out = np.empty(self.shape[1:], dtype=self._dtype)
        p, dev, _ = _out_arg(out, self._dtype, self.cells)
        _check(lib().hydro_get_charge_density(self.h, p, dev))
        return out

    def charge_sum(self):
        out = C.c_double()
        _check(lib().hydro_charge_sum(self.h, C.byref(out)))
        return out.value

    def set_conserved(self, U):
        p, dev, keep = _arg(U, self._dtype, self.nq * self.cells)
        _check(lib().hydro_set_conserved(self.h, p, dev))

    def get_conserved(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self._dtype)
        p, dev, _ = _arg(out, self._dtype, self.nq * self.cells)
        if not dev and not (isinstance(out, np.ndarray) and out.flags["C_CONTIGUOUS"]):
            raise ValueError("host output must be a contiguous numpy array")
        _check(lib().hydro_get_conserved(self.h, p, dev))
        return out

    def get_primitives(self, out=None):
        """(e, vx, vy, vz) as new host arrays, or written into `out`: four
        contiguous host arrays / CPU tensors (pinned ones copy at full speed) or
        four CUDA tensors, of the handle's dtype."""
        if out is None:
            out = [np.empty(self.shape[1:], dtype=self._dtype) for _ in range(4)]
        args = [_out_arg(o, self._dtype, self.cells) for o in out]
        if len({a[1] for a in args}) != 1:
            raise ValueError("outputs must be all on the host or all on the device")
        _check(lib().hydro_get_primitives(self.h, *[a[0] for a in args], args[0][1]))
        return out

    def init_hotspots(self, spots, sigma, e_bg):
        s = np.ascontiguousarray(spots, dtype=np.float64)
        _check(lib().hydro_init_hotspots(self.h, s.ctypes.data_as(C.POINTER(C.c_double)),
                                         s.shape[0], sigma, e_bg))

    def set_jet(self, jet):
        j = np.ascontiguousarray(jet, dtype=np.float64)
        _check(lib().hydro_set_jet(self.h, j.ctypes.data_as(C.POINTER(C.c_double))))

    def step(self, nsteps, t_end=0.0):
        t = C.c_double()
        _check(lib().hydro_step(self.h, nsteps, t_end, C.byref(t)))
        return t.value

    def sweep(self, axis, dt):
        _check(lib().hydro_sweep(self.h, axis, dt))

    def max_rate(self):
        r = C.c_double()
        _check(lib().hydro_max_rate(self.h, C.byref(r)))
        return r.value

    def conservation_sums(self):
        out = (C.c_double * 4)()
        _check(lib().hydro_conservation_sums(self.h, out))
        return np.array(out[:])

    def time(self):
        t = C.c_double()
        _check(lib().hydro_get_time(self.h, C.byref(t)))
        return t.value

    def set_time(self, t):
        _check(lib().hydro_set_time(self.h, t))

    def enable_counters(self, on=True):
        _check(lib().hydro_enable_counters(self.h, int(on)))

    def counters(self):
        out = (C.c_longlong * 6)()
        _check(lib().hydro_counters(self.h, out))
        return dict(zip(COUNTERS, out[:]))

    def check_finite(self):
        _check(lib().hydro_check_finite(self.h))

    def status(self):
        """(code, flags): the hydro_check_status code (0, or 4 UNPHYSICAL,
        5 NEWTON, 6 NONFINITE) and the raw FLAG_* bits, without raising."""
        fl = C.c_uint()
        code = lib().hydro_check_status(self.h, C.byref(fl))
        if code not in (0, 4, 5, 6):
            _check(code)
        return code, fl.value

    def set_kernel_timing(self, on=True):
        _check(lib().hydro_set_kernel_timing(self.h, int(on)))

    def kernel_timing(self):
        """((sweep_ms, other_ms), (sweep_launches, other_launches)) since the last call."""
        ms = (C.c_double * 2)()
        n = (C.c_longlong * 2)()
        _check(lib().hydro_get_kernel_timing(self.h, ms, n))
        return tuple(ms[:]), tuple(n[:])

    def force_launch(self, axis, threads, segments=1):
        _check(lib().hydro_force_launch(self.h, axis, threads, segments))

    def get_launch(self, axis):
        t, s = C.c_int(), C.c_int()
        _check(lib().hydro_get_launch(self.h, axis, C.byref(t), C.byref(s)))
        return t.value, s.value

    def mlp_seed_emin(self):
        """E above which the MLP seeds Newton (tabulated EOS)."""
        out = C.c_double()
        _check(lib().hydro_mlp_seed_emin(self.h, C.byref(out)))
        return out.value

    def c2p_newton(self, U, seed, vmag, iters):
        """Device tensors: U [4][n], vmag [n] (handle dtype), iters [n] int32."""
        n = U.shape[-1]
        pU = _dev(U, self._dtype, 4 * n, "U")
        pv = _dev(vmag, self._dtype, n, "vmag")
        pi = _dev(iters, np.int32, n, "iters")
        _check(lib().hydro_c2p_newton(self.h, pU, n,
                                      SEEDS[seed] if isinstance(seed, str) else seed, pv, pi))

    def c2p_newton_pairs(self, U, seed, rcp, vmag, p, iters):
        """Device tensors: U [4][n] (n even), vmag and p [2][n] (handle dtype),
        iters [2][n] int32; row 0 single solves, row 1 the paired solve."""
        n = U.shape[-1]
        pU = _dev(U, self._dtype, 4 * n, "U")
        pv = _dev(vmag, self._dtype, 2 * n, "vmag")
        pp = _dev(p, self._dtype, 2 * n, "p")
        pi = _dev(iters, np.int32, 2 * n, "iters")
        _check(lib().hydro_c2p_newton_pairs(self.h, pU, n,
                                            SEEDS[seed] if isinstance(seed, str) else seed,
                                            int(rcp), pv, pp, pi))


class Batch(_Base):
    """Many events of uneven size: hydro_batch_create ... hydro_batch_destroy."""

    def __init__(self, grids, eos=None, limiter="minmod", stages=2, stream=None):
        eos_t, self._keep = (eos if eos is not None else make_eos())
        arr = (GridT * len(grids))(*grids)
        self.grids = list(grids)
        h = C.c_void_p()
        lim = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
        _check(lib().hydro_batch_create(arr, len(grids), C.byref(eos_t), lim, stages, C.byref(h)))
        self.h = h
        self.nevents = len(grids)
        self._dtype = np.float64 if grids[0].prec == 0 else np.float32
        self.nq = 5 if grids[0].charge else 4
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "h", None):
            lib().hydro_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def shape(self, event):
        g = self.grids[event]
        return (self.nq, g.nz, g.ny, g.nx)

    def set_stream(self, stream):
        _check(lib().hydro_batch_set_stream(self.h, _stream_ptr(stream)))

    def init_hotspots(self, spots, sigma, e_bg):
        s = np.ascontiguousarray(spots, dtype=np.float64)
        assert s.ndim == 3 and s.shape[0] == self.nevents and s.shape[2] == 7
        _check(lib().hydro_batch_init_hotspots(self.h, s.ctypes.data_as(C.POINTER(C.c_double)),
                                               s.shape[1], sigma, e_bg))

    def _cells(self, event):
        if not 0 <= event < self.nevents:
            raise ValueError(f"event {event} out of range")
        g = self.grids[event]
        return g.nx * g.ny * g.nz

    def set_primitives(self, event, e, vx, vy, vz):
        args = [_arg(a, self._dtype, self._cells(event)) for a in (e, vx, vy, vz)]
        if len({a[1] for a in args}) != 1:
            raise ValueError("inputs must be all on the host or all on the device")
        _check(lib().hydro_batch_set_primitives(self.h, event, *[a[0] for a in args], args[0][1]))

    def set_jets(self, jets):
        j = np.ascontiguousarray(jets, dtype=np.float64)
        _check(lib().hydro_batch_set_jets(self.h, j.ctypes.data_as(C.POINTER(C.c_double))))

    def step(self, nsteps, use_graph=True):
        _check(lib().hydro_batch_step(self.h, nsteps, int(use_graph)))

    def set_conserved(self, event, U):
        p, dev, keep = _arg(U, self._dtype, self.nq * self._cells(event))
        _check(lib().hydro_batch_set_conserved(self.h, event, p, dev))

    def get_conserved(self, event, out=None):
        if out is None:
            out = np.empty(self.shape(event), dtype=self._dtype)
        p, dev, _ = _out_arg(out, self._dtype, self.nq * self._cells(event))
        _check(lib().hydro_batch_get_conserved(self.h, event, p, dev))
        return out

    def get_primitives(self, event):
        outs = [np.empty(self.shape(event)[1:], dtype=self._dtype) for _ in range(4)]
        _check(lib().hydro_batch_get_primitives(self.h, event,
                                                *[o.ctypes.data_as(C.c_void_p) for o in outs], 0))
        return outs

    def times(self):
        out = (C.c_double * self.nevents)()
        _check(lib().hydro_batch_times(self.h, out))
        return np.array(out[:])

    def conservation_sums(self):
        out = (C.c_double * (4 * self.nevents))()
        _check(lib().hydro_batch_conservation_sums(self.h, out))
        return np.array(out[:]).reshape(self.nevents, 4)

    def charge_sums(self):
        out = (C.c_double * self.nevents)()
        _check(lib().hydro_batch_charge_sums(self.h, out))
        return np.array(out[:])

    def set_primitives_charged(self, event, e, vx, vy, vz, n):
        args = [_arg(a, self._dtype, self._cells(event)) for a in (e, vx, vy, vz, n)]
        if len({a[1] for a in args}) != 1:
            raise ValueError("inputs must be all on the host or all on the device")
        _check(lib().hydro_batch_set_primitives_charged(self.h, event, *[a[0] for a in args],
                                                        args[0][1]))

    def event_status(self):
        out = (C.c_int * self.nevents)()
        _check(lib().hydro_batch_event_status(self.h, out))
        return np.array(out[:])

    def event_flags(self):
        """(codes, flags) per event: hydro_check_status codes and FLAG_* bits."""
        st = (C.c_int * self.nevents)()
        fl = (C.c_uint * self.nevents)()
        _check(lib().hydro_batch_event_flags(self.h, st, fl))
        return np.array(st[:]), np.array(fl[:])

    def enable_counters(self, on=True):
        _check(lib().hydro_batch_enable_counters(self.h, int(on)))

    def set_kernel_timing(self, on=True):
        _check(lib().hydro_batch_set_kernel_timing(self.h, int(on)))

    def kernel_timing(self):
        ms = (C.c_double * 2)()
        n = (C.c_longlong * 2)()
        _check(lib().hydro_batch_get_kernel_timing(self.h, ms, n))
        return tuple(ms[:]), tuple(n[:])

    def counters(self):
        out = (C.c_longlong * 6)()
        _check(lib().hydro_batch_counters(self.h, out))
        return dict(zip(COUNTERS, out[:]))


def conservation_sums_noalloc(U, prec, nx, ny, nz, dx, dy=None, dz=None, stream=None):
    """FP64 sums of a caller-held device state U [4][nz][ny][nx] without any
    device allocation by the library (see hydro_conservation_sums_noalloc)."""
    out = (C.c_double * 4)()
    pr = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    if pr not in (0, 1, 2):
        raise ValueError(f"unknown precision {prec}")
    pU = _dev(U, np.float64 if pr == 0 else np.float32, 4 * nx * ny * nz, "U")
    _check(lib().hydro_conservation_sums_noalloc(
        pU, pr,
        nx, ny, nz, dx, dx if dy is None else dy, dx if dz is None else dz, out,
        _stream_ptr(stream)))
    return np.array(out[:])


# ------------------------------------------------------------------ MLP
def mlp_nparam():
    return lib().hydro_mlp_nparam()


def _mlp_args(params, X):
    n = X.shape[0]
    return n, _dev(params, np.float32, mlp_nparam(), "params"), _dev(X, np.float32, 2 * n, "X")


def mlp_forward(params, X, out, stream=None):
    """Device float32 tensors: params [nparam], X [n][2], out [n]."""
    n, pp, px = _mlp_args(params, X)
    _check(lib().hydro_mlp_forward(pp, px, n, _dev(out, np.float32, n, "out"),
                                   _stream_ptr(stream)))


def mlp_hidden(params, X, H1, stream=None):
    """Device float32 tensors: params [nparam], X [n][2], H1 [n][32] receives
    the bf16-rounded first-layer activations the forward feeds to the tensor
    cores."""
    n, pp, px = _mlp_args(params, X)
    _check(lib().hydro_mlp_hidden(pp, px, n, _dev(H1, np.float32, 32 * n, "H1"),
                                  _stream_ptr(stream)))


def mlp_loss_grad(params, X, Y, grad, loss, stream=None):
    n, pp, px = _mlp_args(params, X)
    _check(lib().hydro_mlp_loss_grad(pp, px, _dev(Y, np.float32, n, "Y"), n,
                                     _dev(grad, np.float32, mlp_nparam(), "grad"),
                                     _dev(loss, np.float32, 1, "loss"), _stream_ptr(stream)))


def mlp_train(params, X, Y, batch, epochs, lr, seed, loss_hist, stream=None):
    n, pp, px = _mlp_args(params, X)
    _check(lib().hydro_mlp_train(pp, px, _dev(Y, np.float32, n, "Y"), n, batch, epochs, lr,
                                 seed, _dev(loss_hist, np.float32, epochs, "loss_hist"),
                                 _stream_ptr(stream)))
