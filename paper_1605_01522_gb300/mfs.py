"""ctypes binding of libmfs (include/mfs.h): argument marshalling only.

Every computation happens inside libmfs.so.  Vectors may be numpy arrays
(host memory; the library copies them) or CUDA torch tensors (device
pointers passed straight through).  Loading fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_FIELDS = 8
OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_SINGULAR, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_SETUP = 0, -1, -2, -3, -4, -5, -6, -7
BGS_AMG, SIMPLE, AMG_BGS, AMG_SIMPLE, BGS_GS = 0, 1, 2, 3, 4
BWD, FWD, SYM = 0, 1, 2
NS_CONST, NS_RBM, NS_USER = 0, 1, 2
FP64, FP32P = 0, 1
ABSROWSUM, DIAG = 0, 1
CHEBYSHEV, JACOBI, GS = 0, 1, 2
PRED_BGS_AMG, PRED_AMG_BGS = 0, 1

PRECONDS = {"bgs_amg": BGS_AMG, "simple": SIMPLE, "amg_bgs": AMG_BGS, "amg_simple": AMG_SIMPLE, "bgs_gs": BGS_GS}
ORDERS = {"bwd": BWD, "fwd": FWD, "sym": SYM}

# every symbol include/mfs.h declares
EXPORTS = ["mfs_default_params", "mfs_setup", "mfs_solve", "mfs_clone", "mfs_solve_batch", "mfs_apply", "mfs_matvec", "mfs_dot", "mfs_dot_noalloc", "mfs_fp64_rate", "mfs_ndofs", "mfs_device_bytes",
           "mfs_export_csr", "mfs_export_array", "mfs_num_levels", "mfs_kernel_stats", "mfs_kernel_detail", "mfs_profile_filter", "mfs_free",
           "mfs_strerror", "mfs_last_error"]
KERNEL_CLASSES = ["spmv", "smooth", "vector", "coarse_lu", "arnoldi"]
_OTHER = {2: {1: "smooth_first", 2: "fill", 3: "axpy_diag", 4: "axpy", 5: "convert", 6: "scale", 7: "scale_convert", 8: "scale_convert_dev"},
          3: {1: "lu_solve", 2: "coarse_inverse_apply", 3: "vcycle_tail"},
          4: {1: "mdot", 2: "reduce_partials", 3: "cgs_fused", 4: "cgs_update", 5: "gemv_add"}}


def kernel_name(key: int) -> str:
    """Readable name of a mfs_kernel_detail key (class*100000 + signature)."""
    cls, sig = divmod(key, 100000)
    if cls in (0, 1):
        kind, rest = divmod(sig, 1000)
        br, rest = divmod(rest, 100)
        bc, f64 = divmod(rest, 10)
        base = "spmv" if cls == 0 else "smooth"
        layout = {0: "sell", 1: "warp", 2: "rows", 3: "sell4", 4: "gs_sell", 5: "gs_warp",
                  6: "gs_sell4", 7: "cta", 9: "sell8"}.get(kind, str(kind))
        return f"{base}_{layout}<{br}x{bc},{'f64' if f64 else 'f32'}>"
    return _OTHER.get(cls, {}).get(sig, f"class{cls}_id{sig}")


class Block(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("br", C.c_int), ("bc", C.c_int),
                ("nbrows", C.c_int64), ("nbcols", C.c_int64), ("nnzb", C.c_int64),
                ("rowptr", C.POINTER(C.c_int32)), ("colind", C.POINTER(C.c_int32)),
                ("vals", C.POINTER(C.c_double))]


class FieldDesc(C.Structure):
    _fields_ = [("nnodes", C.c_int64), ("dofs_per_node", C.c_int), ("dim", C.c_int),
                ("coords", C.POINTER(C.c_double)), ("nullspace", C.c_int),
                ("strength_theta", C.c_double), ("petrov_galerkin", C.c_int),
                ("ns_user", C.POINTER(C.c_double)), ("ns_dim", C.c_int), ("dirichlet", C.POINTER(C.c_uint8))]


class Params(C.Structure):
    _fields_ = [("precond", C.c_int), ("bgs_order", C.c_int), ("bgs_sweeps", C.c_int),
                ("simple_group", C.c_int * MAX_FIELDS), ("simple_approx", C.c_int),
                ("max_levels", C.c_int), ("coarse_max", C.c_int64), ("smoother", C.c_int),
                ("cheb_degree", C.c_int), ("cheb_ratio", C.c_double), ("cheb_boost", C.c_double),
                ("jacobi_omega", C.c_double), ("jacobi_sweeps", C.c_int), ("restart", C.c_int),
                ("max_iters", C.c_int), ("precision", C.c_int), ("seed", C.c_uint64),
                ("cuda_stream", C.c_void_p), ("verbose", C.c_int), ("setup_only", C.c_int),
                ("profile", C.c_int), ("no_graphs", C.c_int), ("setup_device", C.c_int),
                ("simple_pred", C.c_int), ("gs_sweeps", C.c_int), ("gs_omega", C.c_double),
                ("rows_split", C.c_int), ("layout_tune", C.c_int), ("vcycle_tail", C.c_int),
                ("pdl", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("true_relres", C.c_double), ("est_relres", C.c_double), ("solve_ms", C.c_double),
                ("setup_ms", C.c_double), ("levels", C.c_int * 2)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "levels" else getattr(self, k)) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmfs.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmfs.so not built ({path}); run paper_1605_01522_gb300/build.py")
    lib = C.CDLL(path)
    H = C.c_void_p
    lib.mfs_default_params.argtypes = [C.POINTER(Params)]
    lib.mfs_default_params.restype = None
    lib.mfs_setup.argtypes = [C.POINTER(Block), C.c_int, C.POINTER(FieldDesc), C.c_int, C.POINTER(Params), C.POINTER(H)]
    lib.mfs_setup.restype = C.c_int
    lib.mfs_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(Info)]
    lib.mfs_solve.restype = C.c_int
    lib.mfs_clone.argtypes = [H, C.c_void_p, C.POINTER(H)]
    lib.mfs_clone.restype = C.c_int
    lib.mfs_solve_batch.argtypes = [C.POINTER(H), C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double,
                                    C.POINTER(Info), C.POINTER(C.c_int), C.c_int]
    lib.mfs_solve_batch.restype = C.c_int
    lib.mfs_apply.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.mfs_apply.restype = C.c_int
    lib.mfs_matvec.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.mfs_matvec.restype = C.c_int
    lib.mfs_dot.argtypes = [H, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    lib.mfs_dot.restype = C.c_int
    lib.mfs_dot_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.c_void_p]
    lib.mfs_dot_noalloc.restype = C.c_int
    lib.mfs_fp64_rate.argtypes = [C.POINTER(C.c_double), C.c_void_p]
    lib.mfs_fp64_rate.restype = C.c_int
    lib.mfs_device_bytes.argtypes = [H, C.c_int]
    lib.mfs_device_bytes.restype = C.c_int64
    lib.mfs_ndofs.argtypes = [H]
    lib.mfs_ndofs.restype = C.c_int64
    lib.mfs_export_csr.argtypes = [H, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.c_void_p, C.c_void_p, C.c_void_p]
    lib.mfs_export_csr.restype = C.c_int
    lib.mfs_export_array.argtypes = [H, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                                     C.POINTER(C.c_int64)]
    lib.mfs_export_array.restype = C.c_int
    lib.mfs_num_levels.argtypes = [H, C.c_int]
    lib.mfs_num_levels.restype = C.c_int
    lib.mfs_kernel_stats.argtypes = [H, C.POINTER(C.c_double), C.c_int, C.c_int]
    lib.mfs_kernel_stats.restype = C.c_int
    lib.mfs_kernel_detail.argtypes = [H, C.POINTER(C.c_double), C.c_int]
    lib.mfs_kernel_detail.restype = C.c_int
    lib.mfs_profile_filter.argtypes = [H, C.c_int, C.c_int64]
    lib.mfs_profile_filter.restype = C.c_int
    lib.mfs_free.argtypes = [H]
    lib.mfs_free.restype = None
    lib.mfs_strerror.argtypes = [C.c_int]
    lib.mfs_strerror.restype = C.c_char_p
    lib.mfs_last_error.argtypes = []
    lib.mfs_last_error.restype = C.c_char_p
    _lib = lib
    return lib


DOT_NOALLOC_MAX_N = 1 << 32


def dot_noalloc(x, y, n=None, stream=None):
    """x . y of two device float64 vectors through mfs_dot_noalloc (no device
    allocation; partial sums in the library's static device array)."""
    lib = load()
    out = C.c_double()
    size = lambda a: a.numel() if hasattr(a, "numel") else len(a)
    n = size(x) if n is None else n
    if n > min(size(x), size(y)):
        raise ValueError(f"dot_noalloc: n = {n} exceeds a vector's length ({size(x)}, {size(y)})")
    if hasattr(x, "is_cuda") and hasattr(y, "is_cuda"):  # torch tensors
        import torch
        if x.device != y.device or (x.is_cuda and x.device.index != torch.cuda.current_device()):
            raise ValueError("dot_noalloc: x and y must be on the current CUDA device")
    rc = lib.mfs_dot_noalloc(_ptr(x), _ptr(y), n, C.byref(out), stream)
    if rc != OK:
        raise MfsError(rc, "mfs_dot_noalloc")
    return out.value


def fp64_rate(stream=None):
    """Measured float64 FMA rate of the current device in TFLOP/s (mfs_fp64_rate)."""
    lib = load()
    out = C.c_double()
    rc = lib.mfs_fp64_rate(C.byref(out), stream)
    if rc != OK:
        raise MfsError(rc, "mfs_fp64_rate")
    return out.value


class MfsError(RuntimeError):
    def __init__(self, code, where):
        lib = load(False)
        super().__init__(f"{where}: {lib.mfs_strerror(code).decode()} ({code}): {lib.mfs_last_error().decode()}")
        self.code = code


def default_params(**kw) -> Params:
    lib = load()
    p = Params()
    lib.mfs_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precond" and isinstance(v, str):
            v = PRECONDS[v]
        elif k == "bgs_order" and isinstance(v, str):
            v = ORDERS[v]
        elif k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "fp32p": FP32P}[v]
        elif k == "simple_approx" and isinstance(v, str):
            v = {"absrowsum": ABSROWSUM, "diag": DIAG}[v]
        elif k == "smoother" and isinstance(v, str):
            v = {"chebyshev": CHEBYSHEV, "jacobi": JACOBI, "gs": GS}[v]
        elif k == "simple_pred" and isinstance(v, str):
            v = {"bgs_amg": PRED_BGS_AMG, "amg_bgs": PRED_AMG_BGS}[v]
        if k == "simple_group":
            arr = (C.c_int * MAX_FIELDS)(*([0] * MAX_FIELDS))
            for i, g in enumerate(v):
                arr[i] = g
            v = arr
        setattr(p, k, v)
    return p


def _ptr(a):
    """Device pointer of a CUDA tensor or host pointer of a numpy array."""
    if hasattr(a, "data_ptr"):
        if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
            raise TypeError("vectors must be contiguous float64")
        return C.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("vectors must be contiguous float64")
    return C.c_void_p(a.ctypes.data)


def solve_batch(solvers, rhs, xs=None, tol=1e-8, nthreads=0, check=True):
    """Solve independent systems together (mfs_solve_batch): solvers[k]
    (distinct handles) with rhs[k]; nthreads <= 0 runs the fused executor
    (one multi-system launch per step and group of systems, one CUDA graph
    per iteration; -nthreads groups, 0 = automatic), nthreads > 0 that many
    host threads on per-handle streams; returns (xs, infos, status)."""
    lib = load()
    n = len(solvers)
    if xs is None:
        xs = [np.zeros(s.n) if isinstance(b, np.ndarray) else b.new_zeros(s.n) for s, b in zip(solvers, rhs)]
    hs = (C.c_void_p * n)(*[s.h.value if isinstance(s.h, C.c_void_p) else s.h for s in solvers])
    rp = (C.c_void_p * n)(*[_ptr(b).value for b in rhs])
    xp = (C.c_void_p * n)(*[_ptr(x).value for x in xs])
    infos = (Info * n)()
    status = (C.c_int * n)()
    rc = lib.mfs_solve_batch(hs, n, rp, xp, tol, infos, status, nthreads)
    if check and rc not in (OK, ERR_NOT_CONVERGED):
        raise MfsError(rc, "mfs_solve_batch")
    return xs, [i.as_dict() for i in infos], list(status)


class Solver:
    """Owns one mfs_handle built from an inputs.BlockSystem."""

    def __init__(self, system, params: Params | None = None, **kw):
        lib = load()
        self.lib = lib
        prm = params if params is not None else default_params(**kw)
        keep = []
        blocks = (Block * len(system.blocks))()
        for k, ((i, j), b) in enumerate(sorted(system.blocks.items())):
            rp = np.ascontiguousarray(b.rowptr, np.int32)
            ci = np.ascontiguousarray(b.colind, np.int32)
            vv = np.ascontiguousarray(b.vals, np.float64)
            keep += [rp, ci, vv]
            blocks[k] = Block(i, j, b.br, b.bc, b.nbrows, b.nbcols, b.nnzb,
                              rp.ctypes.data_as(C.POINTER(C.c_int32)), ci.ctypes.data_as(C.POINTER(C.c_int32)),
                              vv.ctypes.data_as(C.POINTER(C.c_double)))
        fields = (FieldDesc * system.nfields)()
        for i, f in enumerate(system.fields):
            co = np.ascontiguousarray(f.coords, np.float64)
            keep.append(co)
            kind = {"rbm": NS_RBM, "user": NS_USER}.get(f.nullspace, NS_CONST)
            nsu, nsd = None, 0
            if kind == NS_USER:
                nsu = np.ascontiguousarray(f.ns_user, np.float64)
                nsd = int(nsu.shape[1])
                keep.append(nsu)
            dm = getattr(f, "dirichlet_dofs", None)
            if dm is not None:
                dm = np.ascontiguousarray(dm, np.uint8)
                keep.append(dm)
            fields[i] = FieldDesc(f.nnodes, f.b, f.dim, co.ctypes.data_as(C.POINTER(C.c_double)), kind, f.theta,
                                  1 if getattr(f, "petrov_galerkin", False) else 0,
                                  nsu.ctypes.data_as(C.POINTER(C.c_double)) if nsu is not None else None, nsd,
                                  dm.ctypes.data_as(C.POINTER(C.c_uint8)) if dm is not None else None)
        h = C.c_void_p()
        rc = lib.mfs_setup(blocks, len(system.blocks), fields, system.nfields, C.byref(prm), C.byref(h))
        if rc != OK:
            raise MfsError(rc, "mfs_setup")
        self.h = h
        self.params = prm
        self.n = lib.mfs_ndofs(h)
        self.nfields = system.nfields

    def solve(self, rhs, x=None, tol=1e-8, check=True):
        """Solve A x = rhs; x (host or device float64) is overwritten; returns (x, info dict, rc)."""
        if x is None:
            x = np.zeros(self.n) if isinstance(rhs, np.ndarray) else rhs.new_zeros(self.n)
        info = Info()
        rc = self.lib.mfs_solve(self.h, _ptr(rhs), _ptr(x), tol, C.byref(info))
        if check and rc not in (OK, ERR_NOT_CONVERGED):
            raise MfsError(rc, "mfs_solve")
        return x, info.as_dict(), rc

    def apply(self, v, z=None):
        if z is None:
            z = np.zeros(self.n) if isinstance(v, np.ndarray) else v.new_zeros(self.n)
        rc = self.lib.mfs_apply(self.h, _ptr(v), _ptr(z))
        if rc != OK:
            raise MfsError(rc, "mfs_apply")
        return z

    def matvec(self, x, y=None):
        if y is None:
            y = np.zeros(self.n) if isinstance(x, np.ndarray) else x.new_zeros(self.n)
        rc = self.lib.mfs_matvec(self.h, _ptr(x), _ptr(y))
        if rc != OK:
            raise MfsError(rc, "mfs_matvec")
        return y

    def dot(self, x, y):
        """x . y (device float64 vectors of length n) with the solver's reduction."""
        out = C.c_double()
        rc = self.lib.mfs_dot(self.h, _ptr(x), _ptr(y), C.byref(out))
        if rc != OK:
            raise MfsError(rc, "mfs_dot")
        return out.value

    def clone(self, stream=None):
        """A Solver sharing this one's device hierarchy, with its own workspace and stream."""
        h = C.c_void_p()
        rc = self.lib.mfs_clone(self.h, stream, C.byref(h))
        if rc != OK:
            raise MfsError(rc, "mfs_clone")
        other = Solver.__new__(Solver)
        other.lib, other.h, other.params, other.n, other.nfields = self.lib, h, self.params, self.n, self.nfields
        return other

    def device_bytes(self, shared=True):
        """Device bytes of the shared hierarchy (shared=True) or of this handle's workspace."""
        return int(self.lib.mfs_device_bytes(self.h, 1 if shared else 0))

    def num_levels(self, group=0):
        return self.lib.mfs_num_levels(self.h, group)

    def export_csr(self, what, group, level, i, j=0):
        """what: 'A', 'P' or 'R'; returns a scipy CSR matrix."""
        import scipy.sparse as sp
        w = {"A": 0, "P": 1, "R": 2}[what]
        nr, nc, nnz = C.c_int64(), C.c_int64(), C.c_int64()
        rc = self.lib.mfs_export_csr(self.h, w, group, level, i, j, C.byref(nr), C.byref(nc), C.byref(nnz),
                                     None, None, None)
        if rc != OK:
            raise MfsError(rc, "mfs_export_csr")
        rp = np.zeros(nr.value + 1, np.int32)
        ci = np.zeros(nnz.value, np.int32)
        vv = np.zeros(nnz.value, np.float64)
        rc = self.lib.mfs_export_csr(self.h, w, group, level, i, j, C.byref(nr), C.byref(nc), C.byref(nnz),
                                     rp.ctypes.data, ci.ctypes.data, vv.ctypes.data)
        if rc != OK:
            raise MfsError(rc, "mfs_export_csr")
        return sp.csr_matrix((vv, ci, rp), shape=(nr.value, nc.value))

    def export_array(self, what, group, level, i):
        """what: 'agg' (int32 per node), 'lambda' (float), 'dtilde' (float64),
        'colors' (int32 per node, Gauss-Seidel smoother)."""
        w = {"agg": 0, "lambda": 1, "dtilde": 2, "colors": 3}[what]
        cnt = C.c_int64()
        rc = self.lib.mfs_export_array(self.h, w, group, level, i, None, 0, C.byref(cnt))
        if rc != OK:
            raise MfsError(rc, "mfs_export_array")
        buf = np.zeros(cnt.value, np.int32 if w in (0, 3) else np.float64)
        rc = self.lib.mfs_export_array(self.h, w, group, level, i, buf.ctypes.data, cnt.value, C.byref(cnt))
        if rc != OK:
            raise MfsError(rc, "mfs_export_array")
        return float(buf[0]) if w == 1 else buf

    def kernel_stats(self, reset=True):
        """{class: (launches, ms, algorithmic bytes)} of the profiled solves."""
        out = (C.c_double * 15)()
        k = self.lib.mfs_kernel_stats(self.h, out, 15, 1 if reset else 0)
        if k < 0:
            raise MfsError(k, "mfs_kernel_stats")
        return {KERNEL_CLASSES[c]: (int(out[3 * c]), out[3 * c + 1], out[3 * c + 2]) for c in range(k)}

    def kernel_detail(self):
        """Per-kernel rows (name, rows, launches, ms, algorithmic bytes, key, flops), slowest first.
        Call before kernel_stats(reset=True)."""
        cap = 6 * 512
        out = (C.c_double * cap)()
        k = self.lib.mfs_kernel_detail(self.h, out, cap)
        if k < 0:
            raise MfsError(k, "mfs_kernel_detail")
        rows = []
        for r in range(k):
            key, nrows, launches, ms, nbytes, flops = (out[6 * r + q] for q in range(6))
            rows.append((kernel_name(int(key)), int(nrows), int(launches), ms, nbytes, int(key), flops))
        return rows

    def profile_filter(self, key=0, rows=0):
        """Time only the kernel with this detail key (0 = all kernels)."""
        rc = self.lib.mfs_profile_filter(self.h, key, rows)
        if rc != OK:
            raise MfsError(rc, "mfs_profile_filter")

    def close(self):
        if getattr(self, "h", None):
            self.lib.mfs_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
