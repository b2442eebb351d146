"""ctypes binding of include/kfbim.h: argument marshalling only."""
import ctypes
import os

import numpy as np

from .build import LIB

c_int, c_double, c_int64, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p

STATUS = {0: "OK", -1: "E_INVALID", -2: "E_GEOMETRY", -3: "E_NOCONV", -4: "E_NONFINITE",
          -5: "E_CUDA", -6: "E_OOM"}
KINDS = {"sphere": 0, "ellipsoid": 1, "star": 2, "torus": 3, "callback": 4}


class KfbimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


LEVEL_FN = ctypes.CFUNCTYPE(c_double, ctypes.POINTER(c_double), c_void_p)
LEVEL_DERIVS_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double), c_void_p)


class Geometry(ctypes.Structure):
    _fields_ = [("kind", c_int), ("center", c_double * 3), ("rot", c_double * 9),
                ("params", c_double * 8), ("F", LEVEL_FN), ("derivs", LEVEL_DERIVS_FN),
                ("user", c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, ctypes.c_size_t, c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


def torch_allocator(device):
    """kfbim_allocator over torch's CUDA caching allocator on `device`: the
    context's workspace is then part of torch's memory pool (and of
    torch.cuda.memory_allocated).  Returns the ctypes struct; it holds the
    callbacks, which must stay referenced while the context lives."""
    import torch

    def alloc(nbytes, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device))
        except Exception:   # the library reports E_OOM
            return None

    def free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator()
    a.alloc, a.free = ALLOC_FN(alloc), FREE_FN(free)
    return a


class Grid(ctypes.Structure):
    _fields_ = [("N", c_int), ("lo", c_double), ("hi", c_double)]


class Options(ctypes.Structure):
    _fields_ = [("mu", c_double), ("precision", c_int), ("gmres_tol", c_double),
                ("gmres_max", c_int), ("cg_tol", c_double), ("cg_max", c_int),
                ("refine_tol", c_double), ("refine_max", c_int), ("inner_tol", c_double),
                ("pde", c_int), ("lam", c_double), ("transforms", c_int), ("relax", c_double)]


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
    "kfbim_setup_async": (c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(Grid), ctypes.POINTER(Options),
                                  c_void_p, ctypes.POINTER(c_void_p)]),
    "kfbim_setup_ex": (c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(Grid), ctypes.POINTER(Options),
                               c_void_p, ctypes.POINTER(Allocator), ctypes.POINTER(c_void_p)]),
    "kfbim_control_points": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64), c_void_p, c_void_p]),
    "kfbim_jump_points": (c_int, [c_void_p, ctypes.POINTER(c_int64), c_void_p]),
    "kfbim_destroy": (c_int, [c_void_p]),
    "kfbim_last_error": (ctypes.c_char_p, [c_void_p]),
    "kfbim_sizes": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                            ctypes.POINTER(c_int)]),
    "kfbim_table_sizes": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                  ctypes.POINTER(c_int64)]),
    "kfbim_points": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_sides": (c_int, [c_void_p, c_int, c_void_p]),
    "kfbim_normals": (c_int, [c_void_p, c_void_p]),
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
    "kfbim_schur_apply_f32": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "kfbim_poisson_noalloc": (c_int, [c_int, c_int, c_double, c_double, c_void_p, c_void_p,
                                      c_void_p]),
    "kfbim_profile": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p]),
    "kfbim_profile_kernels": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
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
    n = max(int(N), 0) ** 3
    st = lib.kfbim_poisson_noalloc(c, N, lo, hi, _ptr(r, n, "r"), _ptr(u, n, "u"),
                                   c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise KfbimError(st, "kfbim_poisson_noalloc failed (see stderr)")
    return u


def _level_callbacks(desc, errors):
    """C callbacks for a "callback" geometry: desc["F"](x) -> float and
    desc["derivs"](x) -> (gradient (3,), Hessian (3, 3)) at a point x (3
    floats).  An exception cannot cross the C call: the first one is kept in
    `errors` and the callback returns NaN values.  The returned objects must
    stay referenced while setup runs."""
    F, derivs = desc["F"], desc["derivs"]

    def f_c(x, user):
        try:
            return float(F((x[0], x[1], x[2])))
        except Exception as e:  # re-raised by the caller after setup
            errors.append(e)
            return float("nan")

    def d_c(x, g, H, user):
        try:
            gv, Hv = derivs((x[0], x[1], x[2]))
            gv = np.asarray(gv, dtype=np.float64).reshape(3)
            Hv = np.asarray(Hv, dtype=np.float64).reshape(9)
        except Exception as e:  # re-raised by the caller after setup
            errors.append(e)
            gv, Hv = np.full(3, np.nan), np.full(9, np.nan)
        for i in range(3):
            g[i] = gv[i]
        for i in range(9):
            H[i] = Hv[i]

    return LEVEL_FN(f_c), LEVEL_DERIVS_FN(d_c)


def _geometry(desc, errors=None):
    g = Geometry()
    g.kind = KINDS[desc["kind"]]
    if desc["kind"] == "callback":
        g.F, g.derivs = _level_callbacks(desc, [] if errors is None else errors)
        return g
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


E_INVALID = -1


def _ptr(t, n=0, name="tensor", dtype="float64", device=None):
    """Device pointer of torch tensor t, after checking that the library may
    access n values of it: dtype, C-contiguous, at least n elements, a CUDA
    tensor (on CUDA device `device` when given).  None stays None (nullable
    arguments).  A bad argument raises KfbimError(E_INVALID) before any call."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise KfbimError(E_INVALID, "%s: expected a torch tensor, got %s" % (name, type(t).__name__))
    if t.dtype != getattr(torch, dtype):
        raise KfbimError(E_INVALID, "%s: dtype %s, expected torch.%s" % (name, t.dtype, dtype))
    if not t.is_contiguous():
        raise KfbimError(E_INVALID, "%s: not contiguous" % name)
    if t.numel() < n:
        raise KfbimError(E_INVALID, "%s: %d values, at least %d needed" % (name, t.numel(), n))
    if not t.is_cuda:
        raise KfbimError(E_INVALID, "%s: not a CUDA tensor" % name)
    if device is not None and t.device.index != device:
        raise KfbimError(E_INVALID, "%s: on cuda:%s, the solver is on cuda:%d" % (name, t.device.index, device))
    return c_void_p(t.data_ptr())


def _np_ptr(a, n=0, name="array", dtype=np.float64):
    """Host pointer of numpy array a after the same checks (dtype,
    C-contiguous, at least n elements); None stays None."""
    if a is None:
        return None
    if not isinstance(a, np.ndarray):
        raise KfbimError(E_INVALID, "%s: expected a numpy array, got %s" % (name, type(a).__name__))
    if a.dtype != dtype:
        raise KfbimError(E_INVALID, "%s: dtype %s, expected %s" % (name, a.dtype, np.dtype(dtype)))
    if not a.flags.c_contiguous:
        raise KfbimError(E_INVALID, "%s: not C-contiguous" % name)
    if a.size < n:
        raise KfbimError(E_INVALID, "%s: %d values, at least %d needed" % (name, a.size, n))
    return a.ctypes.data_as(c_void_p)


class Solver:
    """One geometry + grid on the CUDA device current at construction.  Device
    arguments are contiguous torch float64 CUDA tensors on that device with at
    least as many values as include/kfbim.h gives for the call (checked before
    the call); work goes on torch's current CUDA stream of that device."""

    def __init__(self, geom, grid, mu=1.0, precision=0, device=True, lam=None, allocator=None, **opts):
        """lam = None: Stokes; lam = Lame lambda: Navier (Lame) problem.
        allocator = "torch": the context's device workspace comes from torch's
        caching allocator (kfbim_setup_ex) instead of cudaMalloc."""
        lib = load_library()
        self._device = None
        if device:
            import torch
            self._device = torch.cuda.current_device()
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
        errors = []
        gm = _geometry(geom, errors)   # holds the ctypes callbacks of a "callback" geometry during setup
        self._allocator = None
        if device:
            # device work of the setup on torch's current stream
            import torch
            stream = c_void_p(torch.cuda.current_stream(self._device).cuda_stream)
            if allocator == "torch":
                self._allocator = torch_allocator(self._device)
                st = lib.kfbim_setup_ex(ctypes.byref(gm), ctypes.byref(gr), ctypes.byref(o), stream,
                                        ctypes.byref(self._allocator), ctypes.byref(ctx))
            elif allocator is None:
                st = lib.kfbim_setup_async(ctypes.byref(gm), ctypes.byref(gr), ctypes.byref(o), stream,
                                           ctypes.byref(ctx))
            else:
                raise KfbimError(E_INVALID, "allocator: None or 'torch'")
        else:
            st = lib.kfbim_setup_host(ctypes.byref(gm), ctypes.byref(gr), ctypes.byref(o), ctypes.byref(ctx))
        if errors:
            if st == 0:
                lib.kfbim_destroy(ctx)
            raise errors[0]
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

    def _stream(self):
        import torch
        return c_void_p(torch.cuda.current_stream(self._device).cuda_stream)

    def _d(self, t, n, name, dtype="float64"):
        return _ptr(t, n, name, dtype, self._device)

    # ------------------------------------------------------------ host data
    def points(self):
        n = self.n_points
        xyz = np.zeros((n, 3))
        comp = np.zeros(n, np.int32)
        axis = np.zeros(n, np.int32)
        prim = np.zeros(n, np.int32)
        self._check(self._lib.kfbim_points(self._ctx, _np_ptr(xyz, 3 * n, "xyz"), _np_ptr(comp, n, "comp", np.int32),
                                           _np_ptr(axis, n, "axis", np.int32), _np_ptr(prim, n, "prim", np.int32)))
        return xyz, comp, axis, prim.astype(bool)

    def control_points(self, comp):
        """(xyz (n, 3), outward normals (n, 3)) of component comp's density
        unknowns, in the order of that component's block of g and phi."""
        n = c_int64()
        self._check(self._lib.kfbim_control_points(self._ctx, comp, ctypes.byref(n), None, None))
        xyz = np.zeros((n.value, 3))
        nrm = np.zeros((n.value, 3))
        self._check(self._lib.kfbim_control_points(self._ctx, comp, ctypes.byref(n),
                                                   _np_ptr(xyz, 3 * n.value, "xyz"),
                                                   _np_ptr(nrm, 3 * n.value, "normal")))
        return xyz, nrm

    def jump_points(self):
        """(n_points, 3) coordinates where f is needed (fpts of solve)."""
        n = c_int64()
        self._check(self._lib.kfbim_jump_points(self._ctx, ctypes.byref(n), None))
        xyz = np.zeros((n.value, 3))
        self._check(self._lib.kfbim_jump_points(self._ctx, ctypes.byref(n), _np_ptr(xyz, 3 * n.value, "xyz")))
        return xyz

    def normals(self):
        """Outward unit normals (n_points, 3) at the control points."""
        nrm = np.zeros((self.n_points, 3))
        self._check(self._lib.kfbim_normals(self._ctx, _np_ptr(nrm, 3 * self.n_points, "normal")))
        return nrm

    def sides(self, c):
        s = np.zeros(self.N ** 3, np.uint8)
        self._check(self._lib.kfbim_sides(self._ctx, c, _np_ptr(s, self.N ** 3, "side", np.uint8)))
        return s.reshape(self.N, self.N, self.N).astype(bool)

    def table_sizes(self):
        a, b, c = c_int64(), c_int64(), c_int64()
        self._check(self._lib.kfbim_table_sizes(self._ctx, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)))
        return a.value, b.value, c.value

    # ----------------------------------------------------------- device ops
    def apply(self, phi, out):
        n = self.n_primary
        self._check(self._lib.kfbim_apply(self._ctx, self._d(phi, n, "phi"), self._d(out, n, "out"),
                                          self._stream()))
        return out

    def solve(self, g, phi, fpts=None, fgrid=None, u=None, p=None):
        n, npt, N3 = self.n_primary, self.n_points, self.N ** 3
        args = (self._d(g, n, "g"), self._d(fpts, 3 * npt, "fpts"), self._d(fgrid, 3 * N3, "fgrid"),
                self._d(phi, n, "phi"), self._d(u, 3 * N3, "u"), self._d(p, N3, "p"))
        st = Stats()
        self._check(self._lib.kfbim_solve(self._ctx, *args, ctypes.byref(st), self._stream()))
        self.last_stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        return phi

    def solve_host(self, g, phi, fpts=None, fgrid=None, u=None, p=None):
        """Host (numpy float64) buffers; copies happen inside the library call."""
        n, npt, N3 = self.n_primary, self.n_points, self.N ** 3
        args = (_np_ptr(g, n, "g"), _np_ptr(fpts, 3 * npt, "fpts"), _np_ptr(fgrid, 3 * N3, "fgrid"),
                _np_ptr(phi, n, "phi"), _np_ptr(u, 3 * N3, "u"), _np_ptr(p, N3, "p"))
        st = Stats()
        self._check(self._lib.kfbim_solve_host(self._ctx, *args, ctypes.byref(st), self._stream()))
        self.last_stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        return phi

    def solve_batch(self, g, phi, fpts=None, fgrid=None, u=None, p=None):
        """B solves in one call: g, phi are (B, n_primary) device tensors, fpts
        (B, 3 n_points), fgrid (B, 3 N^3), u (B, 3 N^3), p (B, N^3); each
        contiguous.  last_stats becomes a list of B dicts."""
        if getattr(g, "dim", lambda: 0)() < 1:
            raise KfbimError(E_INVALID, "g: expected a (B, n_primary) tensor")
        B = int(g.shape[0])
        n, npt, N3 = B * self.n_primary, B * self.n_points, B * self.N ** 3
        args = (self._d(g, n, "g"), self._d(fpts, 3 * npt, "fpts"), self._d(fgrid, 3 * N3, "fgrid"),
                self._d(phi, n, "phi"), self._d(u, 3 * N3, "u"), self._d(p, N3, "p"))
        st = (Stats * max(B, 1))()
        self._check(self._lib.kfbim_solve_batch(self._ctx, B, *args, st, self._stream()))
        self.last_stats = [{k: getattr(st[b], k) for k, _ in Stats._fields_} for b in range(B)]
        return phi

    def apply_adjoint(self, lam, out):
        n = self.n_primary
        self._check(self._lib.kfbim_apply_adjoint(self._ctx, self._d(lam, n, "lam"), self._d(out, n, "out"),
                                                  self._stream()))
        return out

    def solve_adjoint(self, ubar, gbar):
        """gbar = dL/dg for ubar = dL/du (3 N^3 face-grid values)."""
        st = Stats()
        self._check(self._lib.kfbim_solve_adjoint(self._ctx, self._d(ubar, 3 * self.N ** 3, "ubar"),
                                                  self._d(gbar, self.n_primary, "gbar"), ctypes.byref(st),
                                                  self._stream()))
        self.last_stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        return gbar

    def jumps(self, phi, J, fpts=None):
        npt = self.n_points
        self._check(self._lib.kfbim_jumps(self._ctx, self._d(phi, self.n_primary, "phi"),
                                          self._d(fpts, 3 * npt, "fpts"), self._d(J, 12 * npt, "J"),
                                          self._stream()))
        return J

    def interface(self, phi, u, p, fpts=None, fgrid=None):
        N3 = self.N ** 3
        self._check(self._lib.kfbim_interface(self._ctx, self._d(phi, self.n_primary, "phi"),
                                              self._d(fpts, 3 * self.n_points, "fpts"),
                                              self._d(fgrid, 3 * N3, "fgrid"), self._d(u, 3 * N3, "u"),
                                              self._d(p, N3, "p"), self._stream()))
        return u, p

    def pressure_trace(self, p, J, out):
        npt = self.n_points
        self._check(self._lib.kfbim_pressure_trace(self._ctx, self._d(p, self.N ** 3, "p"), self._d(J, 12 * npt, "J"),
                                                   self._d(out, npt, "out"), self._stream()))
        return out

    def trace(self, u, J, out):
        self._check(self._lib.kfbim_trace(self._ctx, self._d(u, 3 * self.N ** 3, "u"),
                                          self._d(J, 12 * self.n_points, "J"),
                                          self._d(out, self.n_primary, "out"), self._stream()))
        return out

    def transform_f32(self, xform, axis, inp, out, backend, wmode=0, wc=0):
        N3 = self.N ** 3
        self._check(self._lib.kfbim_transform_f32(self._ctx, xform, axis, wmode, wc,
                                                  self._d(inp, N3, "inp", "float32"),
                                                  self._d(out, N3, "out", "float32"), backend, self._stream()))
        return out

    def transforms_info(self):
        """{"plain": 0|1, "fused": 0|1 (1 = tensor core), "tune_ms": [4 floats]}."""
        pl, fu = c_int(), c_int()
        ms = (ctypes.c_float * 4)()
        self._check(self._lib.kfbim_transforms_info(self._ctx, ctypes.byref(pl), ctypes.byref(fu), ms))
        return {"plain": pl.value, "fused": fu.value, "tune_ms": [round(float(x), 4) for x in ms]}

    def poisson(self, c, r, u):
        N3 = self.N ** 3
        self._check(self._lib.kfbim_poisson(self._ctx, c, self._d(r, N3, "r"), self._d(u, N3, "u"), self._stream()))
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

    KERNEL_CLASSES = ("transform_fp64", "transform_fp32", "cg_zfwd", "cg_xy", "cg_zinv", "cg_update",
                      "cg_vector", "mac_residual", "jumps")

    def profile_kernels(self):
        """{class: (ms, launches, algorithmic bytes)} since profile(True)."""
        n = len(self.KERNEL_CLASSES)
        ms, bytes_ = (c_double * n)(), (c_double * n)()
        launches = (c_int64 * n)()
        self._check(self._lib.kfbim_profile_kernels(self._ctx, n, ms, launches, bytes_))
        return {k: (ms[i], launches[i], bytes_[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    def schur_apply(self, d, q):
        N3 = self.N ** 3
        self._check(self._lib.kfbim_schur_apply(self._ctx, self._d(d, N3, "d"), self._d(q, N3, "q"),
                                                self._stream()))
        return q

    def schur_apply_f32(self, d, q):
        """FP32 Schur operator of the slab CG (no rank-one term): d, q float32."""
        N3 = self.N ** 3
        self._check(self._lib.kfbim_schur_apply_f32(self._ctx, self._d(d, N3, "d", "float32"),
                                                    self._d(q, N3, "q", "float32"), self._stream()))
        return q
