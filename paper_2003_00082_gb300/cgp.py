"""Python binding of libcgp: the C-ABI entry points under the same names.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device buffers are passed as torch CUDA tensors (torch supplies the
device memory and the stream) or as raw integer device addresses.  The
library must have been built (``paper_2003_00082_gb300.build.build()``); there
is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CGP_OK = 0
CGP_ERR_INVALID_ARG = 1
CGP_ERR_CUDA = 2
CGP_ERR_NOT_CONVERGED = 3
CGP_ERR_BREAKDOWN = 4
CGP_ERR_NONFINITE = 5
CGP_ERR_TIMEOUT = 6
CGP_ERR_OOM = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NOT_CONVERGED", 4: "BREAKDOWN",
                5: "NONFINITE", 6: "TIMEOUT", 7: "OOM"}

CGP_RHS_POTENTIAL = 0
CGP_RHS_PRESSURE = 1
CGP_FP64 = 0
CGP_MIXED = 1
CGP_FP32 = 1          # precision argument of cgp_spmv for the FP32 copy of K

EXPORTS = ("cgp_assemble", "cgp_mesh_query", "cgp_mesh_levels", "cgp_set_far_field", "cgp_far_field_nodes",
           "cgp_mesh_set_ogrid", "cgp_mesh_fine_geometry", "cgp_mesh_matrices",
           "cgp_restrict", "cgp_poisson_solve", "cgp_poisson_solve_async",
           "cgp_poisson_solve_noalloc", "cgp_prolong", "cgp_lorentz", "cgp_velocity_correct", "cgp_spmv",
           "cgp_set_tuning", "cgp_get_tuning", "cgp_autotune", "cgp_last_launch", "cgp_barrier_selftest",
           "cgp_batch_create", "cgp_batch_solve", "cgp_batch_info", "cgp_batch_set_tuning",
           "cgp_batch_autotune", "cgp_batch_query", "cgp_batch_destroy", "cgp_poisson_solve_batched",
           "cgp_gnn_param_count", "cgp_gnn_create", "cgp_gnn_predict", "cgp_gnn_train_step", "cgp_gnn_gradients",
           "cgp_gnn_get_params", "cgp_gnn_set_params", "cgp_gnn_destroy", "cgp_mesh_destroy",
           "cgp_last_error")

CGP_TUNE_SOLVE_FP64 = 0
CGP_TUNE_SOLVE_MIXED = 1
CGP_TUNE_SPMV_FP64 = 2
CGP_TUNE_SPMV_FP32 = 3


class CgpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_it", ctypes.c_int), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("use_x0", ctypes.c_int), ("max_sweeps", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_sweeps", ctypes.c_int),
                ("rel_res_recursive", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libcgp.so (built in-tree) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libcgp.so is not built ({path}); call paper_2003_00082_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), \
        ctypes.c_int, ctypes.c_double
    sig = {
        "cgp_assemble": [dp, i, ip, i, i, ctypes.POINTER(vp)],
        "cgp_mesh_query": [vp, ip, ip, ip, ip, ip, ip],
        "cgp_mesh_fine_geometry": [vp, dp, ip, ip],
        "cgp_mesh_matrices": [vp, ip, ip, dp, dp, dp, dp],
        "cgp_restrict": [vp, i, dp, d, vp, vp, vp, vp, vp, vp],
        "cgp_poisson_solve": [vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp],
        "cgp_poisson_solve_async": [vp, vp, vp, ctypes.POINTER(SolveOpts), vp, vp],
        "cgp_poisson_solve_noalloc": [i, vp, vp, vp, vp, vp, vp, ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(SolveInfo), vp],
        "cgp_prolong": [vp, vp, vp, vp],
        "cgp_mesh_levels": [vp, ip, ip],
        "cgp_set_far_field": [vp, i],
        "cgp_mesh_set_ogrid": [vp, i, i],
        "cgp_far_field_nodes": [vp, ip, ip],
        "cgp_velocity_correct": [vp, vp, vp, vp, d, vp, vp, vp],
        "cgp_lorentz": [vp, vp, vp, vp, dp, d, vp, vp, vp],
        "cgp_spmv": [vp, i, vp, vp, vp],
        "cgp_set_tuning": [vp, i, i, i, i, i],
        "cgp_get_tuning": [vp, i, ip, ip, ip, ip],
        "cgp_last_launch": [vp, i, ip, ip, ip, ip],
        "cgp_autotune": [vp, i, vp, vp, ctypes.c_char_p, vp, dp],
        "cgp_barrier_selftest": [i, i, ctypes.c_longlong, vp],
        "cgp_mesh_destroy": [vp],
        "cgp_batch_create": [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp),
                             ctypes.POINTER(SolveOpts), ctypes.POINTER(vp)],
        "cgp_batch_solve": [vp, vp],
        "cgp_batch_info": [vp, ctypes.POINTER(SolveInfo), dp],
        "cgp_batch_set_tuning": [vp, i, i, i, i],
        "cgp_batch_autotune": [vp, vp, dp],
        "cgp_batch_query": [vp, ip, ip, ip, ip, ip],
        "cgp_batch_destroy": [vp],
        "cgp_poisson_solve_batched": [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp],
        "cgp_gnn_param_count": [],
        "cgp_gnn_create": [vp, i, vp, ctypes.POINTER(vp)],
        "cgp_gnn_predict": [vp, vp, vp, vp, vp, vp],
        "cgp_gnn_train_step": [vp, i, vp, vp, vp, vp, ctypes.c_float, vp, vp],
        "cgp_gnn_gradients": [vp, i, vp, vp, vp, vp, vp, vp, vp, vp],
        "cgp_gnn_get_params": [vp, vp],
        "cgp_gnn_set_params": [vp, vp],
        "cgp_gnn_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.cgp_last_error.argtypes = []
    L.cgp_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(st: int, allow=()):
    if st != CGP_OK and st not in allow:
        msg = load().cgp_last_error().decode(errors="replace")
        raise CgpError(st, msg)
    return st


def _dev(t, dtype_name: str | None = "float64", n: int | None = None):
    """Device address of a torch CUDA tensor (checked) or of a raw integer address."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not getattr(t, "is_cuda", False):
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype_name is not None and str(t.dtype) != "torch." + dtype_name:
        raise ValueError(f"expected dtype {dtype_name}, got {t.dtype}")
    if n is not None and t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} elements, need {n}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dvec3(B):
    return (ctypes.c_double * 3)(*[float(b) for b in B])


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def cgp_assemble(xy_c, tri_c, levels: int = 1):
    """Assemble a mesh pair from host arrays; returns the opaque handle (c_void_p)."""
    xy = np.ascontiguousarray(xy_c, dtype=np.float64)
    tri = np.ascontiguousarray(tri_c, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().cgp_assemble(xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), xy.shape[0],
                               tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), tri.shape[0], levels,
                               ctypes.byref(h)))
    return h


def cgp_mesh_query(mesh):
    vals = [ctypes.c_int() for _ in range(6)]
    _check(load().cgp_mesh_query(mesh, *[ctypes.byref(v) for v in vals]))
    return dict(zip(("n_c", "t_c", "n_e", "n_f", "t_f", "nnz"), [v.value for v in vals]))


def cgp_mesh_levels(mesh):
    """(levels k, node counts of levels 0 .. k)."""
    k = ctypes.c_int()
    _check(load().cgp_mesh_levels(mesh, ctypes.byref(k), None))
    nodes = (ctypes.c_int * (k.value + 1))()
    _check(load().cgp_mesh_levels(mesh, None, nodes))
    return k.value, list(nodes)


def cgp_mesh_set_ogrid(mesh, n_theta, n_r):
    _check(load().cgp_mesh_set_ogrid(mesh, int(n_theta), int(n_r)))


def cgp_set_far_field(mesh, dirichlet):
    _check(load().cgp_set_far_field(mesh, int(dirichlet)))


def cgp_far_field_nodes(mesh):
    cnt = ctypes.c_int()
    _check(load().cgp_far_field_nodes(mesh, ctypes.byref(cnt), None))
    nodes = np.empty(cnt.value, dtype=np.int32)
    _check(load().cgp_far_field_nodes(mesh, None, nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return nodes


def cgp_mesh_fine_geometry(mesh):
    s = cgp_mesh_query(mesh)
    xy = np.empty((s["n_f"], 2), dtype=np.float64)
    tri = np.empty((s["t_f"], 3), dtype=np.int32)
    edges = np.empty((s["n_e"], 2), dtype=np.int32)
    _check(load().cgp_mesh_fine_geometry(mesh, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                         edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return xy, tri, edges


def cgp_mesh_matrices(mesh):
    s = cgp_mesh_query(mesh)
    rowptr = np.empty(s["n_c"] + 1, dtype=np.int32)
    col = np.empty(s["nnz"], dtype=np.int32)
    K, Gx, Gy = (np.empty(s["nnz"]) for _ in range(3))
    dinv = np.empty(s["n_c"])
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))  # noqa: E731
    _check(load().cgp_mesh_matrices(mesh, P(rowptr, ctypes.c_int), P(col, ctypes.c_int), P(K, ctypes.c_double),
                                    P(Gx, ctypes.c_double), P(Gy, ctypes.c_double), P(dinv, ctypes.c_double)))
    return dict(rowptr=rowptr, col=col, K=K, Gx=Gx, Gy=Gy, dinv=dinv)


def cgp_restrict(mesh, kind, B, rho_over_dt, u_f, v_f, b, u_c=None, v_c=None, stream=None):
    _check(load().cgp_restrict(mesh, int(kind), _dvec3(B), float(rho_over_dt), _dev(u_f), _dev(v_f),
                               _dev(u_c), _dev(v_c), _dev(b), _stream(stream)))


def cgp_poisson_solve(mesh, b, x, tol=1e-8, max_it=20000, precision=CGP_FP64, inner_tol=1e-4, use_x0=False,
                      max_sweeps=50, info=True, stream=None, raise_on_status=False):
    """Run one solve; returns the info dict (synchronises) or None when ``info`` is False."""
    opts = SolveOpts(float(tol), int(max_it), int(precision), float(inner_tol), int(bool(use_x0)),
                     int(max_sweeps))
    inf = SolveInfo() if info else None
    st = load().cgp_poisson_solve(mesh, _dev(b), _dev(x), ctypes.byref(opts),
                                  ctypes.byref(inf) if inf is not None else None, _stream(stream))
    solver_states = (CGP_ERR_NOT_CONVERGED, CGP_ERR_BREAKDOWN, CGP_ERR_NONFINITE)
    _check(st, allow=() if raise_on_status else solver_states)
    return inf.as_dict() if inf is not None else None


INFO_BYTES = ctypes.sizeof(SolveInfo)


def cgp_poisson_solve_async(mesh, b, x, tol=1e-8, max_it=20000, precision=CGP_FP64, inner_tol=1e-4,
                            use_x0=False, max_sweeps=50, info_dev=None, stream=None):
    """Launch a solve without host synchronisation; ``info_dev`` is a device address (int) or None."""
    opts = SolveOpts(float(tol), int(max_it), int(precision), float(inner_tol), int(bool(use_x0)),
                     int(max_sweeps))
    _check(load().cgp_poisson_solve_async(mesh, _dev(b), _dev(x), ctypes.byref(opts),
                                          _dev(info_dev, None), _stream(stream)))


CGP_STATIC_MAX_ROWS = 65536


def cgp_poisson_solve_noalloc(n, rowptr, col, K, dinv, b, x, tol=1e-8, max_it=20000, use_x0=False,
                              stream=None):
    """FP64 solve on caller-provided device CSR data; the library allocates nothing (see cgp.h)."""
    opts = SolveOpts(float(tol), int(max_it), CGP_FP64, 1e-4, int(bool(use_x0)), 1)
    inf = SolveInfo()
    st = load().cgp_poisson_solve_noalloc(int(n), _dev(rowptr, "int32"), _dev(col, "int32"), _dev(K), _dev(dinv),
                                          _dev(b), _dev(x), ctypes.byref(opts), ctypes.byref(inf),
                                          _stream(stream))
    _check(st, allow=(CGP_ERR_NOT_CONVERGED, CGP_ERR_BREAKDOWN, CGP_ERR_NONFINITE))
    return inf.as_dict()


def decode_infos(raw: bytes, count: int):
    """Decode ``count`` consecutive cgp_solve_info records copied back from the device."""
    arr = (SolveInfo * count).from_buffer_copy(raw[: count * INFO_BYTES])
    return [a.as_dict() for a in arr]


def cgp_prolong(mesh, x_c, x_f, stream=None):
    _check(load().cgp_prolong(mesh, _dev(x_c), _dev(x_f), _stream(stream)))


def cgp_lorentz(mesh, phi_f, u_f, v_f, B, sigma, grad, force=None, stream=None):
    _check(load().cgp_lorentz(mesh, _dev(phi_f), _dev(u_f), _dev(v_f), _dvec3(B), float(sigma), _dev(grad),
                              _dev(force), _stream(stream)))


def cgp_velocity_correct(mesh, p_f, u_t, v_t, dt_over_rho, u, v, stream=None):
    _check(load().cgp_velocity_correct(mesh, _dev(p_f), _dev(u_t), _dev(v_t), float(dt_over_rho), _dev(u), _dev(v),
                                       _stream(stream)))


def cgp_spmv(mesh, precision, x, y, stream=None):
    dt = "float64" if precision == CGP_FP64 else "float32"
    _check(load().cgp_spmv(mesh, int(precision), _dev(x, dt), _dev(y, dt), _stream(stream)))


def cgp_set_tuning(mesh, what, block=0, lanes=0, blocks=0, flags=0):
    _check(load().cgp_set_tuning(mesh, int(what), int(block), int(lanes), int(blocks), int(flags)))


def cgp_get_tuning(mesh, what):
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().cgp_get_tuning(mesh, int(what), *[ctypes.byref(a) for a in v]))
    return dict(block=v[0].value, lanes=v[1].value, blocks=v[2].value, flags=v[3].value)


def cgp_autotune(mesh, precision, b, x, cache_path=None, stream=None):
    """Time the solver's launch shapes on b and keep the fastest; returns the best time in ms (-1: cache hit)."""
    best = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(load().cgp_autotune(mesh, int(precision), _dev(b), _dev(x), path, _stream(stream), ctypes.byref(best)))
    return best.value


def cgp_last_launch(mesh, precision=CGP_FP64):
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().cgp_last_launch(mesh, int(precision), *[ctypes.byref(a) for a in v]))
    return dict(blocks=v[0].value, block=v[1].value, resident=v[2].value, smem=v[3].value)


def cgp_barrier_selftest(nblk, absent, spin_ns, stream=None):
    """Returns the status (CGP_OK or CGP_ERR_TIMEOUT) without raising for a timeout."""
    return _check(load().cgp_barrier_selftest(int(nblk), int(absent), int(spin_ns), _stream(stream)),
                  allow=(CGP_ERR_TIMEOUT,))


def cgp_mesh_destroy(mesh):
    _check(load().cgp_mesh_destroy(mesh))


def _ptr_array(items, what):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = _dev(t, what).value if t is not None else None
    return arr


class Batch:
    """Many systems solved in one persistent launch (cgp_batch_* calls)."""

    def __init__(self, meshes, b, x, tol=1e-8, max_it=20000, precision=CGP_FP64, inner_tol=1e-4, use_x0=False,
                 max_sweeps=50):
        L = load()
        self.count = len(meshes)
        handles = (ctypes.c_void_p * self.count)(*[m.handle.value if hasattr(m, "handle") else m.value
                                                   for m in meshes])
        opts = SolveOpts(float(tol), int(max_it), int(precision), float(inner_tol), int(bool(use_x0)),
                         int(max_sweeps))
        self.handle = ctypes.c_void_p()
        self._keep = (list(meshes), list(b), list(x))
        _check(L.cgp_batch_create(handles, self.count, _ptr_array(b, "float64"), _ptr_array(x, "float64"),
                                  ctypes.byref(opts), ctypes.byref(self.handle)))

    def solve(self, stream=None):
        _check(load().cgp_batch_solve(self.handle, _stream(stream)))

    def info(self):
        """(list of info dicts, list of per-system seconds); synchronises."""
        infos = (SolveInfo * self.count)()
        secs = (ctypes.c_double * self.count)()
        st = load().cgp_batch_info(self.handle, infos, secs)
        _check(st, allow=(CGP_ERR_NOT_CONVERGED, CGP_ERR_BREAKDOWN, CGP_ERR_NONFINITE))
        return [i.as_dict() for i in infos], list(secs)

    def set_tuning(self, block=0, lanes=0, blocks_per_sm=0, flags=0):
        _check(load().cgp_batch_set_tuning(self.handle, int(block), int(lanes), int(blocks_per_sm), int(flags)))

    def autotune(self, stream=None):
        best = ctypes.c_double()
        _check(load().cgp_batch_autotune(self.handle, _stream(stream), ctypes.byref(best)))
        return best.value

    def query(self):
        v = [ctypes.c_int() for _ in range(4)]
        blocks = (ctypes.c_int * self.count)()
        _check(load().cgp_batch_query(self.handle, *[ctypes.byref(a) for a in v], blocks))
        return dict(grid=v[0].value, block=v[1].value, lanes=v[2].value, resident=v[3].value, blocks=list(blocks))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().cgp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cgp_poisson_solve_batched(meshes, b, x, tol=1e-8, max_it=20000, precision=CGP_FP64, inner_tol=1e-4,
                              use_x0=False, max_sweeps=50, stream=None):
    """One-shot batched solve; returns the list of info dicts."""
    n = len(meshes)
    handles = (ctypes.c_void_p * n)(*[m.handle.value if hasattr(m, "handle") else m.value for m in meshes])
    opts = SolveOpts(float(tol), int(max_it), int(precision), float(inner_tol), int(bool(use_x0)), int(max_sweeps))
    infos = (SolveInfo * n)()
    st = load().cgp_poisson_solve_batched(handles, n, _ptr_array(b, "float64"), _ptr_array(x, "float64"),
                                          ctypes.byref(opts), infos, _stream(stream))
    _check(st, allow=(CGP_ERR_NOT_CONVERGED, CGP_ERR_BREAKDOWN, CGP_ERR_NONFINITE))
    return [i.as_dict() for i in infos]


def cgp_batch_create(*a, **k):
    return Batch(*a, **k)


def cgp_batch_solve(batch, stream=None):
    batch.solve(stream)


def cgp_batch_info(batch):
    return batch.info()


def cgp_batch_set_tuning(batch, *a, **k):
    batch.set_tuning(*a, **k)


def cgp_batch_autotune(batch, stream=None):
    return batch.autotune(stream)


def cgp_batch_query(batch):
    return batch.query()


def cgp_batch_destroy(batch):
    batch.close()


def cgp_gnn_param_count():
    return load().cgp_gnn_param_count()


class GNN:
    """The learned initial-guess network of a mesh (cgp_gnn_* calls)."""

    def __init__(self, mesh, max_batch, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != cgp_gnn_param_count():
            raise ValueError("params has the wrong length")
        self.n = mesh.n_c
        self.handle = ctypes.c_void_p()
        _check(load().cgp_gnn_create(mesh.handle, int(max_batch), p.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(self.handle)))

    def predict(self, b, phi1, phi2, x0, stream=None):
        _check(load().cgp_gnn_predict(self.handle, _dev(b), _dev(phi1), _dev(phi2), _dev(x0), _stream(stream)))

    def train_step(self, batch, b, phi1, phi2, phi_t, lr=1e-3, loss_dev=None, stream=None):
        _check(load().cgp_gnn_train_step(self.handle, int(batch), _dev(b), _dev(phi1), _dev(phi2), _dev(phi_t),
                                         float(lr), _dev(loss_dev, "float32"), _stream(stream)))

    def gradients(self, batch, b, phi1, phi2, phi_t, stream=None):
        """(grads [P], raw outputs [batch, n], loss); synchronous."""
        g = np.empty(cgp_gnn_param_count(), dtype=np.float32)
        out = np.empty((batch, self.n), dtype=np.float32)
        loss = np.empty(1, dtype=np.float32)
        _check(load().cgp_gnn_gradients(self.handle, int(batch), _dev(b), _dev(phi1), _dev(phi2), _dev(phi_t),
                                        g.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                        loss.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return g, out, float(loss[0])

    def get_params(self):
        p = np.empty(cgp_gnn_param_count(), dtype=np.float32)
        _check(load().cgp_gnn_get_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)))
        return p

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().cgp_gnn_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().cgp_gnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cgp_gnn_create(mesh, max_batch, params):
    return GNN(mesh, max_batch, params)


def cgp_gnn_predict(g, b, phi1, phi2, x0, stream=None):
    g.predict(b, phi1, phi2, x0, stream)


def cgp_gnn_train_step(g, *a, **k):
    g.train_step(*a, **k)


def cgp_gnn_gradients(g, *a, **k):
    return g.gradients(*a, **k)


def cgp_gnn_get_params(g):
    return g.get_params()


def cgp_gnn_set_params(g, params):
    g.set_params(params)


def cgp_gnn_destroy(g):
    g.close()


class Mesh:
    """Owning wrapper of a cgp_mesh handle with its sizes."""

    def __init__(self, xy_c, tri_c, levels: int = 1):
        self.handle = cgp_assemble(xy_c, tri_c, levels)
        self.__dict__.update(cgp_mesh_query(self.handle))
        self.levels, self.level_nodes = cgp_mesh_levels(self.handle)

    def fine_geometry(self):
        return cgp_mesh_fine_geometry(self.handle)

    def matrices(self):
        return cgp_mesh_matrices(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            cgp_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
