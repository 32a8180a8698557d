"""Thin ctypes binding of librte.so (include/rte.h): argument marshalling only.

Every function below calls the C entry point of the same name; all arithmetic of the method
runs in the library's CUDA kernels.  There is no Python or CPU fallback: ``load()`` raises
when the library has not been built, and every call raises ``RteError`` on a non-OK status.
"""
import ctypes
import os

import numpy as np

# Hardware work queues of the process's CUDA context, read when the context is created: the
# default 8 makes the streams of batched instances (three each) share queues and serialise.
# Takes effect only when this module is imported before anything initialises CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librte.so")

RTE_OK, RTE_EINVAL, RTE_ENOMEM, RTE_ENOCONV, RTE_ECUDA, RTE_ETIMEOUT, RTE_ESTATE = range(7)
RTE_Q_GL1D, RTE_Q_CL_HEMI, RTE_Q_EXPLICIT = range(3)
RTE_FP64, RTE_FP32, RTE_FP32_BF16F = range(3)
RTE_REL_INF, RTE_ABS_INF = range(2)
RTE_ROM_OFF, RTE_ROM_AUTO, RTE_ROM_MANUAL = range(3)
RTE_ROM_IG, RTE_ROM_PC = range(2)
RTE_SA_DSA, RTE_SA_DMD_ITER = range(2)
RTE_BE, RTE_BDF2 = range(2)
STATUS_NAMES = {0: "RTE_OK", 1: "RTE_EINVAL", 2: "RTE_ENOMEM", 3: "RTE_ENOCONV", 4: "RTE_ECUDA",
                5: "RTE_ETIMEOUT", 6: "RTE_ESTATE"}


class RteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


MAX_PC_LEVELS = 4   # RTE_MAX_PC_LEVELS


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)


class Quadrature(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_gl", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("n_dirs", ctypes.c_int), ("mu", _dp), ("eta", _dp), ("w", _dp)]


class Problem(ctypes.Structure):
    _fields_ = [("mesh", Mesh), ("quad", Quadrature), ("sigma_t", _dp), ("sigma_s", _dp),
                ("source", _dp), ("rho0", _dp), ("c_dt", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("eps_sisa", ctypes.c_double), ("eps_ig", ctypes.c_double),
                ("eps_pc", ctypes.c_double), ("eps_up", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("r_max", ctypes.c_int), ("precision", ctypes.c_int),
                ("rom", ctypes.c_int), ("residual_norm", ctypes.c_int), ("up_rel", ctypes.c_int),
                ("cg_rtol", ctypes.c_double), ("cg_max_iter", ctypes.c_int), ("tune", ctypes.c_int),
                ("sweep_rows", ctypes.c_int), ("sweep_lanes", ctypes.c_int),
                ("sweep_warps", ctypes.c_int), ("sweep_kernel", ctypes.c_int),
                ("lookahead", ctypes.c_int), ("pc_levels", ctypes.c_int),
                ("sa_kind", ctypes.c_int), ("mh_window", ctypes.c_int),
                ("cg_blocks", ctypes.c_int), ("time_scheme", ctypes.c_int),
                ("degree", ctypes.c_int), ("dsa_fp64", ctypes.c_int), ("graph", ctypes.c_int),
                ("dsa_cluster", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("phase", ctypes.c_int), ("last_iterations", ctypes.c_int),
                ("last_cg_iterations", ctypes.c_int), ("total_iterations", ctypes.c_longlong),
                ("total_sweeps", ctypes.c_longlong), ("total_cg_iterations", ctypes.c_longlong),
                ("ig_rank", ctypes.c_int), ("pc_rank", ctypes.c_int), ("ig_updated", ctypes.c_int),
                ("pc_updated", ctypes.c_int), ("last_residual", ctypes.c_double),
                ("last_ig_error", ctypes.c_double), ("last_pc_error", ctypes.c_double),
                ("cell_direction_updates", ctypes.c_longlong), ("time_sweep_ms", ctypes.c_double),
                ("time_dsa_ms", ctypes.c_double), ("time_rom_ms", ctypes.c_double),
                ("time_total_ms", ctypes.c_double), ("si_sweep_launches", ctypes.c_longlong),
                ("si_sweep_kernel_ms", ctypes.c_double), ("f_sweep_launches", ctypes.c_longlong),
                ("f_sweep_kernel_ms", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
                ("sweep_lanes", ctypes.c_int), ("sweep_si_rows", ctypes.c_int),
                ("sweep_si_warps", ctypes.c_int), ("sweep_f_rows", ctypes.c_int),
                ("sweep_f_warps", ctypes.c_int), ("sweep_tuned", ctypes.c_int),
                ("sweep_si_kernel", ctypes.c_int), ("sweep_f_kernel", ctypes.c_int),
                ("pc_level_rank", ctypes.c_int * MAX_PC_LEVELS),
                ("pc_level_updated", ctypes.c_int * MAX_PC_LEVELS),
                ("total_mh_jumps", ctypes.c_longlong)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("pc_level_rank", "pc_level_updated"):
            d[k] = list(d[k])
        return d


_lib = None
_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "rte_default_options": (None, [ctypes.POINTER(Options)]),
    "rte_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(Mesh), ctypes.POINTER(Quadrature),
                                  _dp, _dp, _dp, ctypes.c_double, ctypes.POINTER(Options)]),
    "rte_set_initial": (ctypes.c_int, [_vp, _dp, _dp]),
    "rte_set_inflow": (ctypes.c_int, [_vp, _dp]),
    "rte_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rte_set_stream": (ctypes.c_int, [_vp, _vp]),
    "rte_restart": (ctypes.c_int, [_vp]),
    "rte_rom_update": (ctypes.c_int, [_vp]),
    "rte_get_scalar_flux": (ctypes.c_int, [_vp, _dp]),
    "rte_get_angular_flux": (ctypes.c_int, [_vp, _dp]),
    "rte_get_quadrature": (ctypes.c_int, [_vp, _ip, _dp, _dp, _dp]),
    "rte_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    "rte_last_error": (ctypes.c_char_p, [_vp]),
    "rte_destroy": (None, [_vp]),
    "rte_op_sweep": (ctypes.c_int, [_vp, _dp, _dp]),
    "rte_op_fsweep": (ctypes.c_int, [_vp, _dp, _dp]),
    "rte_op_dsa": (ctypes.c_int, [_vp, _dp, _dp, _ip]),
    "rte_op_rom_append": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, ctypes.c_double, _ip]),
    "rte_op_rom_apply": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp]),
    "rte_op_rom_get": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _dp, _dp, _dp]),
    "rte_op_rom_reset": (ctypes.c_int, [_vp]),
    "rte_quadrature_rule": (ctypes.c_int, [ctypes.POINTER(Quadrature), ctypes.c_int, _ip, _dp, _dp,
                                           _dp]),
    "rte_save_size": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "rte_save": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_size_t]),
    "rte_load": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_size_t]),
    "rte_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(Problem),
                                        ctypes.POINTER(Options)]),
    "rte_batch_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rte_batch_restart": (ctypes.c_int, [_vp]),
    "rte_batch_size": (ctypes.c_int, [_vp]),
    "rte_batch_instance": (_vp, [_vp, ctypes.c_int]),
    "rte_batch_status": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rte_batch_destroy": (None, [_vp]),
    "rte_dsa_solve_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _vp, _vp, _vp, ctypes.c_double,
                                             ctypes.c_int, _vp, _ip, _vp]),
}


def load(path=LIB_PATH):
    """Load librte.so (built by paper_2603_19647_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def default_options(**kw):
    o = Options()
    load().rte_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Handle:
    """One problem instance (an ``rte_handle``).  Methods mirror the C calls one to one.
    Vectors over the degrees of freedom have ndof entries (ncell, or 4 ncell mode-major for the
    Q1 scheme, ``options.degree = 1``)."""

    def __init__(self, ptr, ncell, nv, ndof=None):
        self.ptr = ptr
        self.ncell = ncell
        self.nv = nv
        self.ndof = ncell if ndof is None else ndof

    def _check(self, status):
        if status != RTE_OK:
            msg = load().rte_last_error(self.ptr).decode()
            raise RteError(status, msg)

    # lifecycle -----------------------------------------------------------------------
    def rte_destroy(self):
        if self.ptr and not getattr(self, "_owned_by_batch", False):
            load().rte_destroy(self.ptr)
        self.ptr = None

    destroy = rte_destroy

    def __del__(self):
        try:
            self.rte_destroy()
        except Exception:
            pass

    def rte_set_initial(self, rho0=None, f0=None):
        rho0 = None if rho0 is None else _f64(rho0, self.ndof)
        f0 = None if f0 is None else _f64(f0, self.ndof * self.nv)
        self._check(load().rte_set_initial(self.ptr, _p(rho0), _p(f0)))

    def rte_set_inflow(self, g):
        g = _f64(g, 4)
        self._check(load().rte_set_inflow(self.ptr, _p(g)))

    def rte_set_stream(self, stream_ptr):
        """stream_ptr: an integer cudaStream_t (e.g. torch.cuda.Stream().cuda_stream) or None."""
        self._check(load().rte_set_stream(self.ptr, None if stream_ptr is None else
                                          ctypes.c_void_p(int(stream_ptr))))

    def rte_restart(self):
        self._check(load().rte_restart(self.ptr))

    def rte_step(self, nsteps=1):
        self._check(load().rte_step(self.ptr, int(nsteps)))

    def rte_rom_update(self):
        self._check(load().rte_rom_update(self.ptr))

    def rte_get_scalar_flux(self):
        out = np.empty(self.ndof)
        self._check(load().rte_get_scalar_flux(self.ptr, _p(out)))
        return out

    def rte_get_angular_flux(self):
        out = np.empty((self.nv, self.ndof))
        self._check(load().rte_get_angular_flux(self.ptr, _p(out)))
        return out

    def rte_get_quadrature(self):
        n = ctypes.c_int(0)
        mu, eta, w = np.empty(self.nv), np.empty(self.nv), np.empty(self.nv)
        self._check(load().rte_get_quadrature(self.ptr, ctypes.byref(n), _p(mu), _p(eta), _p(w)))
        return mu, eta, w

    def rte_save(self):
        """rte_save_size + rte_save: the checkpoint as bytes."""
        n = ctypes.c_size_t(0)
        self._check(load().rte_save_size(self.ptr, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(load().rte_save(self.ptr, buf, n))
        return buf.raw

    def rte_load(self, blob):
        blob = bytes(blob)
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(load().rte_load(self.ptr, buf, ctypes.c_size_t(len(blob))))

    def rte_get_stats(self):
        st = Stats()
        self._check(load().rte_get_stats(self.ptr, ctypes.byref(st)))
        return st.as_dict()

    # operator-level calls ------------------------------------------------------------
    def rte_op_sweep(self, rho):
        rho = _f64(rho, self.ndof)
        out = np.empty(self.ndof)
        self._check(load().rte_op_sweep(self.ptr, _p(rho), _p(out)))
        return out

    def rte_op_fsweep(self, rho):
        rho = _f64(rho, self.ndof)
        out = np.empty(self.ndof)
        self._check(load().rte_op_fsweep(self.ptr, _p(rho), _p(out)))
        return out

    def rte_op_dsa(self, residual):
        r = _f64(residual, self.ndof)
        out = np.empty(self.ndof)
        its = ctypes.c_int(0)
        self._check(load().rte_op_dsa(self.ptr, _p(r), _p(out), ctypes.byref(its)))
        return out, its.value

    def rte_op_rom_append(self, which, x, b, trunc_eps=-1.0):
        x = _f64(x, self.ndof)
        b = _f64(b, self.ndof)
        grew = ctypes.c_int(0)
        self._check(load().rte_op_rom_append(self.ptr, int(which), _p(x), _p(b), float(trunc_eps),
                                             ctypes.byref(grew)))
        return bool(grew.value)

    def rte_op_rom_apply(self, which, rhs):
        rhs = _f64(rhs, self.ndof)
        out = np.empty(self.ndof)
        self._check(load().rte_op_rom_apply(self.ptr, int(which), _p(rhs), _p(out)))
        return out

    def rte_op_rom_get(self, which):
        r = ctypes.c_int(0)
        self._check(load().rte_op_rom_get(self.ptr, int(which), ctypes.byref(r), None, None, None))
        r = r.value
        S, U, Ar = np.empty(r), np.empty((r, self.ndof)), np.empty((r, r))
        if r:
            self._check(load().rte_op_rom_get(self.ptr, int(which), None, _p(S), _p(U), _p(Ar)))
        return S, U, Ar

    def rte_op_rom_reset(self):
        self._check(load().rte_op_rom_reset(self.ptr))


def _ndof(n, options):
    return 4 * n if options is not None and options.degree == 1 else n


def as_modes(x, n, nd):
    """A per-cell array as the degrees of freedom of a piecewise-constant field: unchanged for
    Q0; for Q1 the cell values are mode 0 (the cell average) and the other modes are zero."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    if x.size == nd or nd == n:
        return x
    out = np.zeros(nd)
    out[:n] = x
    return out


def rte_create(mesh: Mesh, quad: Quadrature, sigma_t, sigma_s, source, c_dt, options=None):
    """rte_create; returns a Handle.  mesh / quad: ctypes structs (see ``mesh_from`` and
    ``quadrature_from``); sigma_t, sigma_s per cell, x fastest; source per degree of freedom
    (a per-cell source is taken as piecewise constant, see ``as_modes``)."""
    lib = load()
    n = mesh.nx * mesh.ny
    nd = _ndof(n, options)
    st, ss, G = _f64(sigma_t, n), _f64(sigma_s, n), _f64(as_modes(source, n, nd), nd)
    h = _vp()
    opt = ctypes.byref(options) if options is not None else None
    status = lib.rte_create(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), _p(st), _p(ss),
                            _p(G), float(c_dt), opt)
    if status != RTE_OK:
        raise RteError(status, lib.rte_last_error(None).decode())
    nv = ctypes.c_int(0)
    lib.rte_get_quadrature(h, ctypes.byref(nv), None, None, None)
    return Handle(h, n, nv.value, nd)


def rte_dsa_solve_noalloc(dim, nx, ny, x0, x1, y0, y1, c_dt, sigma_t_dev, sigma_s_dev,
                          residual_dev, cg_rtol, cg_max_iter, delta_dev, stream=None):
    """rte_dsa_solve_noalloc with device pointers given as integers (e.g. tensor.data_ptr());
    returns the CG iteration count."""
    its = ctypes.c_int(0)
    lib = load()
    status = lib.rte_dsa_solve_noalloc(int(dim), int(nx), int(ny), float(x0), float(x1), float(y0),
                                       float(y1), float(c_dt), _vp(sigma_t_dev), _vp(sigma_s_dev),
                                       _vp(residual_dev), float(cg_rtol), int(cg_max_iter),
                                       _vp(delta_dev), ctypes.byref(its),
                                       None if stream is None else _vp(int(stream)))
    if status != RTE_OK:
        raise RteError(status, lib.rte_last_error(None).decode())
    return its.value


def rte_quadrature_rule(quad: Quadrature, dim):
    """(mu, eta, w) of the rule `quad` describes, computed by the library on the host."""
    lib = load()
    n = ctypes.c_int(0)
    status = lib.rte_quadrature_rule(ctypes.byref(quad), int(dim), ctypes.byref(n), None, None, None)
    if status != RTE_OK:
        raise RteError(status, lib.rte_last_error(None).decode())
    mu, eta, w = np.empty(n.value), np.empty(n.value), np.empty(n.value)
    status = lib.rte_quadrature_rule(ctypes.byref(quad), int(dim), ctypes.byref(n), _p(mu), _p(eta),
                                     _p(w))
    if status != RTE_OK:
        raise RteError(status, lib.rte_last_error(None).decode())
    return mu, eta, w


def mesh_from(workload):
    x0, x1, y0, y1 = workload.domain
    dim = 1 if workload.quadrature[0] == "gl" else 2
    return Mesh(dim, workload.nx, workload.ny, x0, x1, y0, y1)


def quadrature_from(desc=None, mu=None, eta=None, w=None):
    """A Quadrature struct from a workload descriptor ("gl", n) / ("cl_hemi", n_phi, n_vz), or
    from explicit arrays (kept alive on the returned struct)."""
    if mu is not None:
        mu, w = _f64(mu), _f64(w)
        eta = np.zeros_like(mu) if eta is None else _f64(eta)
        q = Quadrature(RTE_Q_EXPLICIT, 0, 0, mu.size, _p(mu), _p(eta), _p(w))
        q._keep = (mu, eta, w)
        return q
    if desc[0] == "gl":
        return Quadrature(RTE_Q_GL1D, desc[1], 0, 0, None, None, None)
    return Quadrature(RTE_Q_CL_HEMI, desc[2], desc[1], 0, None, None, None)


def create_from_workload(wl, options=None, quad=None):
    """rte_create + rte_set_initial for an inputs.Workload (inflow set when nonzero)."""
    h = rte_create(mesh_from(wl), quad if quad is not None else quadrature_from(wl.quadrature),
                   wl.sigma_t, wl.sigma_s, wl.source, wl.c_dt, options)
    h.rte_set_initial(as_modes(wl.rho0, h.ncell, h.ndof))
    if np.any(wl.inflow):
        h.rte_set_inflow(wl.inflow)
    return h


class Batch:
    """Batched instances (``rte_batch``): independent problems stepped side by side."""

    def __init__(self, ptr, handles, keep):
        self.ptr = ptr
        self.handles = handles
        self._keep = keep

    def rte_batch_step(self, nsteps=1):
        status = load().rte_batch_step(self.ptr, int(nsteps))
        if status != RTE_OK:
            bad = [i for i in range(len(self.handles)) if load().rte_batch_status(self.ptr, i) != RTE_OK]
            msg = load().rte_last_error(self.handles[bad[0]].ptr).decode() if bad else ""
            raise RteError(status, f"instance {bad[0] if bad else '?'}: {msg}")

    def rte_batch_restart(self):
        status = load().rte_batch_restart(self.ptr)
        if status != RTE_OK:
            raise RteError(status, "rte_batch_restart")

    def instance(self, i):
        return self.handles[i]

    def destroy(self):
        if self.ptr:
            load().rte_batch_destroy(self.ptr)
            self.ptr = None
            for h in self.handles:
                h.ptr = None

    def __len__(self):
        return len(self.handles)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def rte_batch_create(workloads, options=None):
    """rte_batch_create for a list of inputs.Workload (isotropic initial flux rho0 each)."""
    lib = load()
    n = len(workloads)
    probs = (Problem * n)()
    keep = []
    for i, wl in enumerate(workloads):
        nc = wl.nx * wl.ny
        nd = _ndof(nc, options)
        arrs = [_f64(wl.sigma_t, nc), _f64(wl.sigma_s, nc), as_modes(wl.source, nc, nd),
                as_modes(wl.rho0, nc, nd)]
        q = quadrature_from(wl.quadrature)
        keep.append((arrs, q))
        probs[i] = Problem(mesh_from(wl), q, _p(arrs[0]), _p(arrs[1]), _p(arrs[2]), _p(arrs[3]),
                           float(wl.c_dt))
    b = _vp()
    opt = ctypes.byref(options) if options is not None else None
    status = lib.rte_batch_create(ctypes.byref(b), n, probs, opt)
    if status != RTE_OK:
        raise RteError(status, lib.rte_last_error(None).decode())
    handles = []
    for i, wl in enumerate(workloads):
        hp = lib.rte_batch_instance(b, i)
        nv = ctypes.c_int(0)
        lib.rte_get_quadrature(hp, ctypes.byref(nv), None, None, None)
        h = Handle(_vp(hp), wl.nx * wl.ny, nv.value, _ndof(wl.nx * wl.ny, options))
        h._owned_by_batch = True
        handles.append(h)
    return Batch(b, handles, keep)
