"""ctypes binding of include/kfbim.h: argument marshalling only."""
import ctypes
import os

import numpy as np

from .build import LIB

c_int, c_double, c_int64, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p

STATUS = {0: "OK", -1: "E_INVALID", -2: "E_GEOMETRY", -3: "E_NOCONV", -4: "E_NONFINITE",
          -5: "E_CUDA", -6: "E_OOM"}
KINDS = {"sphere": 0, "ellipsoid": 1, "star": 2, "torus": 3}


class KfbimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("kind", c_int), ("center", c_double * 3), ("rot", c_double * 9),
                ("params", c_double * 8)]


class Grid(ctypes.Structure):
    _fields_ = [("N", c_int), ("lo", c_double), ("hi", c_double)]


class Options(ctypes.Structure):
    _fields_ = [("mu", c_double), ("precision", c_int), ("gmres_tol", c_double),
                ("gmres_max", c_int), ("cg_tol", c_double), ("cg_max", c_int),
                ("refine_tol", c_double), ("refine_max", c_int), ("inner_tol", c_double),
                ("pde", c_int), ("lam", c_double), ("transforms", c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("gmres_iters", c_int), ("interface_solves", c_int), ("cg_iters", c_int),
                ("refine_sweeps", c_int), ("gmres_residual", c_double),
                ("kernel_launches", c_int64)]


SYMBOLS = {
    "kfbim_default_options": (None, [ctypes.POINTER(Options)]),
    "kfbim_setup": (c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(Grid), ctypes.POINTER(Options),
                            ctypes.POINTER(c_void_p)]),
    "kfbim_setup_host": (c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(Grid),
                                 ctypes.POINTER(Options), ctypes.POINTER(c_void_p)]),
    "kfbim_destroy": (c_int, [c_void_p]),
    "kfbim_last_error": (ctypes.c_char_p, [c_void_p]),
    "kfbim_sizes": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                            ctypes.POINTER(c_int)]),
    "kfbim_table_sizes": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                  ctypes.POINTER(c_int64)]),
    "kfbim_points": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_sides": (c_int, [c_void_p, c_int, c_void_p]),
    "kfbim_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                            ctypes.POINTER(Stats), c_void_p]),
    "kfbim_solve_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, ctypes.POINTER(Stats), c_void_p]),
    "kfbim_solve_batch": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, ctypes.POINTER(Stats), c_void_p]),
    "kfbim_transform_f32": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_int,
                                    c_void_p]),
    "kfbim_transforms_info": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_apply_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_solve_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(Stats), c_void_p]),
    "kfbim_pressure_trace": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_jumps": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_interface": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_trace": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_poisson": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "kfbim_schur_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_poisson_noalloc": (c_int, [c_int, c_int, c_double, c_double, c_void_p, c_void_p,
                                      c_void_p]),
    "kfbim_profile": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p]),
}

_lib = None


def library_path():
    return LIB


def load_library():
    """Load libkfbim.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libkfbim.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2303_04992_gb300.build" % LIB)
        lib = ctypes.CDLL(LIB)
        for name, (res, args) in SYMBOLS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def poisson_noalloc(c, N, lo, hi, r, u):
    """Allocation-free FFT Poisson solve on face grid c (N <= 64): r, u are
    caller-owned float64 CUDA tensors of N^3 values; torch's current stream."""
    import torch
    lib = load_library()
    st = lib.kfbim_poisson_noalloc(c, N, lo, hi, _ptr(r), _ptr(u),
                                   c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise KfbimError(st, "kfbim_poisson_noalloc failed (see stderr)")
    return u


def _geometry(desc):
    g = Geometry()
    g.kind = KINDS[desc["kind"]]
    for i, v in enumerate(desc.get("center", (0.0, 0.0, 0.0))):
        g.center[i] = v
    rot = desc.get("rotation", np.eye(3).reshape(-1).tolist())
    for i, v in enumerate(np.asarray(rot, dtype=np.float64).reshape(-1)):
        g.rot[i] = v
    if desc["kind"] == "sphere":
        params = [desc["radius"]]
    elif desc["kind"] == "ellipsoid":
        params = list(desc["axes"])
    elif desc["kind"] == "torus":
        params = [desc["a"], desc["c"]]
    else:
        params = [desc["r0"], desc["eps"], desc["m"], desc["n"]]
    for i, v in enumerate(params):
        g.params[i] = v
    return g


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(c_void_p)


class Solver:
    """One geometry + grid.  Device arguments are torch float64 CUDA tensors
    (contiguous); work goes on torch's current CUDA stream."""

    def __init__(self, geom, grid, mu=1.0, precision=0, device=True, lam=None, **opts):
        """lam = None: Stokes; lam = Lame lambda: Navier (Lame) problem."""
        lib = load_library()
        o = Options()
        lib.kfbim_default_options(ctypes.byref(o))
        o.mu = mu
        o.precision = precision
        if lam is not None:
            o.pde = 1
            o.lam = lam
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        gr = Grid(int(grid["N"]), float(grid["lo"]), float(grid["hi"]))
        ctx = c_void_p()
        fn = lib.kfbim_setup if device else lib.kfbim_setup_host
        st = fn(ctypes.byref(_geometry(geom)), ctypes.byref(gr), ctypes.byref(o), ctypes.byref(ctx))
        if st != 0:
            raise KfbimError(st, "setup failed (see stderr)")
        self._lib, self._ctx = lib, ctx
        n_all, n_prim, N = c_int64(), c_int64(), c_int()
        lib.kfbim_sizes(ctx, ctypes.byref(n_all), ctypes.byref(n_prim), ctypes.byref(N))
        self.n_points, self.n_primary, self.N = n_all.value, n_prim.value, N.value
        self.lo, self.hi = float(grid["lo"]), float(grid["hi"])
        self.h = (self.hi - self.lo) / self.N
        self.mu = mu
        self.lam = lam
        self.last_stats = None

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.kfbim_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise KfbimError(st, self._lib.kfbim_last_error(self._ctx).decode())

    @staticmethod
    def _stream():
        import torch
        return c_void_p(torch.cuda.current_stream().cuda_stream)

    # ------------------------------------------------------------ host data
    def points(self):
        n = self.n_points
        xyz = np.zeros((n, 3))
        comp = np.zeros(n, np.int32)
        axis = np.zeros(n, np.int32)
        prim = np.zeros(n, np.int32)
        self._check(self._lib.kfbim_points(self._ctx, _np_ptr(xyz), _np_ptr(comp), _np_ptr(axis),
                                           _np_ptr(prim)))
        return xyz, comp, axis, prim.astype(bool)

    def sides(self, c):
        s = np.zeros(self.N ** 3, np.uint8)
        self._check(self._lib.kfbim_sides(self._ctx, c, _np_ptr(s)))
        return s.reshape(self.N, self.N, self.N).astype(bool)

    def table_sizes(self):
        a, b, c = c_int64(), c_int64(), c_int64()
        self._check(self._lib.kfbim_table_sizes(self._ctx, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)))
        return a.value, b.value, c.value

    # ----------------------------------------------------------- device ops
    def apply(self, phi, out):
        self._check(self._lib.kfbim_apply(self._ctx, _ptr(phi), _ptr(out), self._stream()))
        return out

    def solve(self, g, phi, fpts=None, fgrid=None, u=None, p=None):
        st = Stats()
        self._check(self._lib.kfbim_solve(self._ctx, _ptr(g), _ptr(fpts), _ptr(fgrid), _ptr(phi),
                                          _ptr(u), _ptr(p), ctypes.byref(st), self._stream()))
        self.last_stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        return phi

    def solve_host(self, g, phi, fpts=None, fgrid=None, u=None, p=None):
        """Host (numpy float64) buffers; copies happen inside the library call."""
        st = Stats()
        self._check(self._lib.kfbim_solve_host(self._ctx, _np_ptr(g), _np_ptr(fpts), _np_ptr(fgrid),
                                               _np_ptr(phi), _np_ptr(u), _np_ptr(p), ctypes.byref(st),
                                               self._stream()))
        self.last_stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        return phi

    def solve_batch(self, g, phi, fpts=None, fgrid=None, u=None, p=None):
        """B solves in one call: g, phi are (B, n_primary) device tensors, fpts
        (B, 3 n_points), fgrid (B, 3 N^3), u (B, 3 N^3), p (B, N^3); each
        contiguous.  last_stats becomes a list of B dicts."""
        B = int(g.shape[0])
        st = (Stats * B)()
        self._check(self._lib.kfbim_solve_batch(self._ctx, B, _ptr(g), _ptr(fpts), _ptr(fgrid), _ptr(phi),
                                                _ptr(u), _ptr(p), st, self._stream()))
        self.last_stats = [{k: getattr(st[b], k) for k, _ in Stats._fields_} for b in range(B)]
        return phi

    def apply_adjoint(self, lam, out):
        self._check(self._lib.kfbim_apply_adjoint(self._ctx, _ptr(lam), _ptr(out), self._stream()))
        return out

    def solve_adjoint(self, ubar, gbar):
        """gbar = dL/dg for ubar = dL/du (3 N^3 face-grid values)."""
        st = Stats()
        self._check(self._lib.kfbim_solve_adjoint(self._ctx, _ptr(ubar), _ptr(gbar), ctypes.byref(st),
                                                  self._stream()))
        self.last_stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        return gbar

    def jumps(self, phi, J, fpts=None):
        self._check(self._lib.kfbim_jumps(self._ctx, _ptr(phi), _ptr(fpts), _ptr(J), self._stream()))
        return J

    def interface(self, phi, u, p, fpts=None, fgrid=None):
        self._check(self._lib.kfbim_interface(self._ctx, _ptr(phi), _ptr(fpts), _ptr(fgrid), _ptr(u),
                                              _ptr(p), self._stream()))
        return u, p

    def pressure_trace(self, p, J, out):
        self._check(self._lib.kfbim_pressure_trace(self._ctx, _ptr(p), _ptr(J), _ptr(out), self._stream()))
        return out

    def trace(self, u, J, out):
        self._check(self._lib.kfbim_trace(self._ctx, _ptr(u), _ptr(J), _ptr(out), self._stream()))
        return out

    def transform_f32(self, xform, axis, inp, out, backend, wmode=0, wc=0):
        self._check(self._lib.kfbim_transform_f32(self._ctx, xform, axis, wmode, wc, _ptr(inp), _ptr(out),
                                                  backend, self._stream()))
        return out

    def transforms_info(self):
        """{"plain": 0|1, "fused": 0|1 (1 = tensor core), "tune_ms": [4 floats]}."""
        pl, fu = c_int(), c_int()
        ms = (ctypes.c_float * 4)()
        self._check(self._lib.kfbim_transforms_info(self._ctx, ctypes.byref(pl), ctypes.byref(fu), ms))
        return {"plain": pl.value, "fused": fu.value, "tune_ms": [round(float(x), 4) for x in ms]}

    def poisson(self, c, r, u):
        self._check(self._lib.kfbim_poisson(self._ctx, c, _ptr(r), _ptr(u), self._stream()))
        return u

    def profile(self, enable):
        """enable True/False starts/stops kernel timing; None reads it:
        {"fp64"|"fp32": (ms, launches, bytes)}."""
        if enable is not None:
            self._check(self._lib.kfbim_profile(self._ctx, 1 if enable else 0, *([None] * 6)))
            return None
        v = [c_double(), c_int64(), c_double(), c_double(), c_int64(), c_double()]
        self._check(self._lib.kfbim_profile(self._ctx, -1, *[ctypes.byref(x) for x in v]))
        return {"fp64": (v[0].value, v[1].value, v[2].value),
                "fp32": (v[3].value, v[4].value, v[5].value)}

    def schur_apply(self, d, q):
        self._check(self._lib.kfbim_schur_apply(self._ctx, _ptr(d), _ptr(q), self._stream()))
        return q
