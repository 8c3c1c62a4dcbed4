"""GB300 hybrid DH^2 compression of the Helmholtz single layer operator.

Thin ctypes binding of ``libdh2.so`` (C ABI in ``include/dh2.h``).  Every step
of the construction and of the matvec runs in the library's CUDA kernels; this
module only marshals arguments.  Importing it does not need a GPU; calling into
the library does, and a missing library raises ``RuntimeError`` (there is no
fallback path).

The functions keep the C names (``dh2_build_tree``, ``dh2_build_dh2``,
``dh2_matvec`` ...).  ``Tree`` and ``Matrix`` are small owning wrappers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdh2.so")

DH2_OK, DH2_EINVAL, DH2_ENOMEM, DH2_ECUDA, DH2_ETIMEOUT, DH2_ENUMERIC, DH2_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
DH2_FP64, DH2_MIXED = 0, 1
DH2_C64, DH2_C128 = 1, 2
DH2_RANK_BLOCKREL, DH2_RANK_GLOBAL, DH2_RANK_SPECTRAL = 0, 1, 2
DH2_FAULT_NONE, DH2_FAULT_TIMEOUT, DH2_FAULT_NONFINITE, DH2_FAULT_ALLOC = 0, 1, 2, 3
DH2_SINGLE_LAYER, DH2_DOUBLE_LAYER = 0, 1
(DH2_X_R, DH2_X_ZROW, DH2_X_ZCOL, DH2_X_SROW, DH2_X_SCOL, DH2_X_QROW, DH2_X_QCOL,
 DH2_X_CROW, DH2_X_CCOL, DH2_X_P, DH2_X_RW, DH2_X_PW) = range(12)
DH2_MLP_IN, DH2_MLP_HIDDEN, DH2_MLP_OUT, DH2_MLP_NPARAMS, DH2_PROBE_ORDERS = 8, 128, 2, 17922, 6
# the trained weights of the learned order/rank model (FP32, little endian, packed order of dh2.h)
LEARNED_WEIGHTS = os.path.join(HERE, "learned_order_rank.f32")

_STATUS = {DH2_EINVAL: "EINVAL", DH2_ENOMEM: "ENOMEM", DH2_ECUDA: "ECUDA", DH2_ETIMEOUT: "ETIMEOUT",
           DH2_ENUMERIC: "ENUMERIC", DH2_EUNSUPPORTED: "EUNSUPPORTED"}


class dh2_options(C.Structure):
    _fields_ = [("eta1", C.c_double), ("leaf_max", C.c_int32), ("precision", C.c_int32),
                ("rank_rule", C.c_int32), ("qr_fp64", C.c_int32), ("qr_group_rows", C.c_int32),
                ("workspace_bytes", C.c_int64), ("tensor_cores", C.c_int32), ("kb_store", C.c_int32),
                ("learned", C.c_int32), ("svd_fp64", C.c_int32), ("model", C.c_void_p),
                ("qr_tpc", C.c_int32 * 3), ("fault", C.c_int32), ("symmetry", C.c_int32), ("direct", C.c_int32),
                ("layer", C.c_int32), ("gram_tc", C.c_int32)]


class dh2_tree_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nclusters", C.c_int32), ("depth", C.c_int32)]


class dh2_matrix_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("depth", C.c_int32), ("m", C.c_int32), ("k", C.c_int32),
                ("nadm", C.c_int64), ("nnear", C.c_int64), ("npairs", C.c_int64), ("nactive", C.c_int64),
                ("near_entries", C.c_int64), ("coupling_entries", C.c_int64), ("basis_entries", C.c_int64),
                ("matvec_bytes", C.c_int64), ("max_rank_row", C.c_int32), ("max_rank_col", C.c_int32),
                ("mean_rank_row", C.c_double), ("mean_rank_col", C.c_double),
                ("stage_ms", C.c_double * 16), ("kernel_ms", C.c_double * 16),
                ("kernel_launches", C.c_int64 * 16), ("kernel_work", C.c_double * 16),
                ("kernel_work_kind", C.c_int32 * 16), ("learned_m", C.c_int32), ("rank_cap_retries", C.c_int32),
                ("truncation_bytes", C.c_int64), ("symmetric", C.c_int32), ("direct", C.c_int32),
                ("peak_pool_bytes", C.c_int64)]


class DH2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = C.c_void_p
_SIGS = {
    "dh2_options_default": (C.c_int, [C.POINTER(dh2_options)]),
    "dh2_build_tree": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.POINTER(dh2_options), _P, C.POINTER(_P)]),
    "dh2_build_dh2": (C.c_int, [_P, C.c_double, C.c_int32, C.c_double, C.c_double, C.POINTER(dh2_options), _P,
                                C.POINTER(_P)]),
    "dh2_build_dh2_batch": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_double, C.c_double,
                                      C.POINTER(dh2_options), C.c_int32, _P]),
    "dh2_matvec": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "dh2_matvec_batch": (C.c_int, [_P, C.c_int32, _P, _P, C.c_int32, _P]),
    "dh2_matvec_noalloc": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "dh2_matvec_host": (C.c_int, [_P, _P, _P, _P]),
    "dh2_set_timing": (C.c_int, [_P, C.c_int32]),
    "dh2_sync": (C.c_int, [_P]),
    "dh2_release_cached": (C.c_int, []),
    "dh2_tree_get_info": (C.c_int, [_P, C.POINTER(dh2_tree_info)]),
    "dh2_tree_export": (C.c_int, [_P] + [_P] * 9),
    "dh2_matrix_get_info": (C.c_int, [_P, C.POINTER(dh2_matrix_info)]),
    "dh2_export_directions": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "dh2_export_blocks": (C.c_int, [_P, _P, _P, _P]),
    "dh2_export_pair": (C.c_int, [_P, C.c_int32, C.c_int64, _P, C.c_int64, _P, _P]),
    "dh2_export_ranks": (C.c_int, [_P, _P, _P]),
    "dh2_stage_name": (C.c_char_p, [C.c_int32]),
    "dh2_kernel_name": (C.c_char_p, [C.c_int32]),
    "dh2_free_tree": (None, [_P]),
    "dh2_free_matrix": (None, [_P]),
    "dh2_last_error": (C.c_char_p, []),
    "dh2_kernel_launches": (C.c_int64, []),
    "dh2_model_create": (C.c_int, [_P, _P, C.POINTER(_P)]),
    "dh2_model_get_params": (C.c_int, [_P, _P]),
    "dh2_model_forward": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "dh2_model_grad": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "dh2_model_train_step": (C.c_int, [_P, _P, _P, C.c_int64, C.c_float, _P, _P]),
    "dh2_free_model": (None, [_P]),
    "dh2_dense_rows": (C.c_int, [_P, C.c_double, _P, C.c_int32, _P, _P, _P]),
    "dh2_gram": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int64, C.c_int32, _P, _P]),
    "dh2_autotune": (C.c_int, [_P, C.c_double, C.c_int32, C.c_double, C.c_double, C.POINTER(dh2_options), C.c_int32,
                               _P, C.POINTER(dh2_options), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dh2_learned_features": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(dh2_options), _P, _P, C.c_int64,
                                       C.POINTER(C.c_int64), _P]),
    "dh2_learned_probe": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(dh2_options), _P, _P, C.c_int64,
                                    C.POINTER(C.c_int64)]),
}


def lib():
    """Loads libdh2.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdh2.so not built ({LIB_PATH}); run paper_1809_04384_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status):
    if status != DH2_OK:
        raise DH2Error(status, lib().dh2_last_error().decode())


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def options(**kw) -> dh2_options:
    o = dh2_options()
    _check(lib().dh2_options_default(C.byref(o)))
    for k, v in kw.items():
        if k == "qr_tpc":
            for i, t in enumerate(v):
                o.qr_tpc[i] = int(t)
        else:
            setattr(o, k, v)
    return o


def dh2_autotune(tree, kappa, m, eta, eps, base=None, reps=2, stream=None):
    """(tuned options, QR ms per build tuned, QR ms per build of base): the weight-QR tile
    shapes and row-group size that build this workload fastest (timed builds)."""
    tuned = dh2_options()
    t_ms, b_ms = C.c_double(), C.c_double()
    _check(lib().dh2_autotune(tree, float(kappa), int(m), float(eta), float(eps), C.byref(base or options()),
                              int(reps), _stream(stream), C.byref(tuned), C.byref(t_ms), C.byref(b_ms)))
    return tuned, t_ms.value, b_ms.value


# ----------------------------------------------------------------------------- C names

def dh2_build_tree(vertices, triangles=None, opts=None, stream=None):
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = None if triangles is None else np.ascontiguousarray(triangles, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().dh2_build_tree(_ptr(v), len(v), _ptr(t), 0 if t is None else len(t),
                                C.byref(opts or options()), _stream(stream), C.byref(h)))
    return h


def dh2_build_dh2(tree, kappa, m, eta, eps, opts=None, stream=None):
    h = C.c_void_p()
    _check(lib().dh2_build_dh2(tree, float(kappa), int(m), float(eta), float(eps), C.byref(opts or options()),
                               _stream(stream), C.byref(h)))
    return h


def dh2_build_dh2_batch(trees, kappas, m, eta, eps, opts=None, nstreams=0):
    """Concurrent builds of len(trees) matrices; returns their handles in order."""
    count = len(trees)
    th = (C.c_void_p * max(count, 1))(*[t for t in trees])
    ka = np.ascontiguousarray(kappas, dtype=np.float64)
    if len(ka) != count:
        raise ValueError("one kappa per tree")
    out = (C.c_void_p * max(count, 1))()
    _check(lib().dh2_build_dh2_batch(C.cast(th, C.c_void_p), count, _ptr(ka), int(m), float(eta), float(eps),
                                     C.byref(opts or options()), int(nstreams), C.cast(out, C.c_void_p)))
    return [C.c_void_p(out[i]) for i in range(count)]


def _vec_dtype(xs, ys):
    import torch
    dts = {x.dtype for x in xs} | {y.dtype for y in ys}
    if len(dts) != 1 or next(iter(dts)) not in (torch.complex64, torch.complex128):
        raise TypeError("all vectors must share one dtype, complex64 or complex128")
    for v in list(xs) + list(ys):
        if not (v.is_cuda and v.is_contiguous()):
            raise TypeError("vectors must be contiguous CUDA tensors")
    return DH2_C64 if next(iter(dts)) == torch.complex64 else DH2_C128


def dh2_matvec_batch(mats, xs, ys, stream=None):
    """ys[i] = G~_i xs[i] for distinct matrices (CUDA tensors, one dtype)."""
    import torch
    count = len(mats)
    if len(xs) != count or len(ys) != count:
        raise ValueError("one x and one y per matrix")
    if count == 0:
        return ys
    dtype = _vec_dtype(xs, ys)
    if stream is None:
        stream = torch.cuda.current_stream(xs[0].device)
    mh = (C.c_void_p * count)(*[m for m in mats])
    xp = (C.c_void_p * count)(*[x.data_ptr() for x in xs])
    yp = (C.c_void_p * count)(*[y.data_ptr() for y in ys])
    _check(lib().dh2_matvec_batch(C.cast(mh, C.c_void_p), count, C.cast(xp, C.c_void_p), C.cast(yp, C.c_void_p),
                                  dtype, _stream(stream)))
    return ys


def dh2_matvec(mat, x, y, stream=None):
    """y = G~ x for CUDA tensors x, y (complex64 or complex128, same dtype)."""
    import torch
    if x.dtype != y.dtype or x.dtype not in (torch.complex64, torch.complex128):
        raise TypeError("x and y must both be complex64 or complex128")
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise TypeError("x and y must be contiguous CUDA tensors")
    dtype = DH2_C64 if x.dtype == torch.complex64 else DH2_C128
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    _check(lib().dh2_matvec(mat, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), dtype, _stream(stream)))
    return y


def dh2_matvec_noalloc(mat, x, y, stream=None):
    """dh2_matvec with its scratch in the library's fixed device array (no allocation)."""
    import torch
    if x.dtype != y.dtype or x.dtype not in (torch.complex64, torch.complex128):
        raise TypeError("x and y must both be complex64 or complex128")
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise TypeError("x and y must be contiguous CUDA tensors")
    dtype = DH2_C64 if x.dtype == torch.complex64 else DH2_C128
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    _check(lib().dh2_matvec_noalloc(mat, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), dtype,
                                    _stream(stream)))
    return y


def dh2_matvec_host(mat, x, stream=None):
    """End-to-end matvec on host arrays (complex128, original order)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(x)
    _check(lib().dh2_matvec_host(mat, _ptr(x), _ptr(y), _stream(stream)))
    return y


def dh2_dense_rows(tree, kappa, rows, x, stream=None):
    """(G x)[rows] in FP64 on the GPU (reference rows for the product's error); x: complex128
    CUDA tensor in original element order, rows: original element ids."""
    import torch
    if not (x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous()):
        raise TypeError("x must be a contiguous complex128 CUDA tensor")
    r = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty(len(r), dtype=np.complex128)
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    _check(lib().dh2_dense_rows(tree, float(kappa), _ptr(r), len(r), C.c_void_p(x.data_ptr()), _ptr(out),
                                _stream(stream)))
    return out


def dh2_gram(z, gram_tc=1, stream=None):
    """G = Z^* Z in FP64 (complex128 CUDA tensor) of a complex64 CUDA matrix z (rows x cols,
    row pitch z.stride(0)), as the weight factorisations form it."""
    import torch
    if not (z.is_cuda and z.dtype == torch.complex64 and z.dim() == 2 and z.stride(1) == 1):
        raise TypeError("z must be a complex64 CUDA matrix with unit column stride")
    rows, cols = z.shape
    g = torch.empty((cols, cols), dtype=torch.complex128, device=z.device)
    if stream is None:
        stream = torch.cuda.current_stream(z.device)
    _check(lib().dh2_gram(C.c_void_p(z.data_ptr()), rows, cols, z.stride(0), int(gram_tc), C.c_void_p(g.data_ptr()),
                          _stream(stream)))
    return g


def dh2_release_cached():
    """Hands the freed device memory the library's pool keeps back to the driver."""
    _check(lib().dh2_release_cached())


def dh2_free_tree(tree):
    lib().dh2_free_tree(tree)


def dh2_free_matrix(mat):
    lib().dh2_free_matrix(mat)


# ----------------------------------------------------------------------------- wrappers

class Tree:
    """Cluster tree and bounding boxes on the GPU (owning handle)."""

    def __init__(self, vertices, triangles=None, leaf_max=32, stream=None):
        self.handle = dh2_build_tree(vertices, triangles, options(leaf_max=leaf_max), stream)
        info = dh2_tree_info()
        _check(lib().dh2_tree_get_info(self.handle, C.byref(info)))
        self.n, self.nclusters, self.depth = info.n, info.nclusters, info.depth

    def export(self):
        nc, n = self.nclusters, self.n
        out = {k: np.empty(nc, dtype=np.int32) for k in ("offset", "size", "parent", "son0", "son1", "level")}
        perm = np.empty(n, dtype=np.int32)
        lo = np.empty((nc, 3))
        hi = np.empty((nc, 3))
        _check(lib().dh2_tree_export(self.handle, _ptr(perm), _ptr(out["offset"]), _ptr(out["size"]),
                                     _ptr(out["parent"]), _ptr(out["son0"]), _ptr(out["son1"]),
                                     _ptr(out["level"]), _ptr(lo), _ptr(hi)))
        out.update(perm=perm, lo=lo, hi=hi)
        return out

    def close(self):
        if getattr(self, "handle", None):
            dh2_free_tree(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """Recompressed DH^2 matrix on the GPU (owning handle).  With ``model`` (a ``Model``) the
    build chooses the order and sizes the truncation by the learned model (m is ignored)."""

    def __init__(self, tree: Tree, kappa, m, eta, eps, precision=DH2_MIXED, eta1=10.0, rank_rule=DH2_RANK_BLOCKREL,
                 qr_fp64=1, svd_fp64=1, workspace_bytes=0, qr_group_rows=0, tensor_cores=1, kb_store=0, model=None,
                 qr_tpc=(0, 0, 0), fault=DH2_FAULT_NONE, symmetry=1, direct=0, layer=DH2_SINGLE_LAYER, gram_tc=1,
                 stream=None):
        opts = options(eta1=eta1, leaf_max=32, precision=precision, rank_rule=rank_rule, qr_fp64=qr_fp64,
                       svd_fp64=svd_fp64, qr_group_rows=qr_group_rows, workspace_bytes=workspace_bytes,
                       tensor_cores=tensor_cores, kb_store=kb_store, qr_tpc=qr_tpc, fault=fault, symmetry=symmetry,
                       direct=direct, layer=layer, gram_tc=gram_tc)
        if model is not None:
            opts.learned = 1
            opts.model = model.handle
        self.precision = precision
        self.handle = dh2_build_dh2(tree.handle, kappa, m, eta, eps, opts, stream)
        self.info = self.get_info()
        self.n = self.info.n

    @classmethod
    def from_handle(cls, handle, precision):
        """Takes ownership of a dh2_matrix handle (e.g. one of dh2_build_dh2_batch)."""
        self = cls.__new__(cls)
        self.precision = precision
        self.handle = handle
        self.info = self.get_info()
        self.n = self.info.n
        return self

    def get_info(self):
        info = dh2_matrix_info()
        _check(lib().dh2_matrix_get_info(self.handle, C.byref(info)))
        return info

    def stage_ms(self):
        info = self.get_info()
        out = {}
        for i in range(16):
            name = lib().dh2_stage_name(i)
            if name is None:
                break
            out[name.decode()] = info.stage_ms[i]
        return out

    def kernel_times(self):
        """{kernel name: (summed ms, launches)} from the library's CUDA events."""
        info = self.get_info()
        out = {}
        for i in range(16):
            name = lib().dh2_kernel_name(i)
            if name is None:
                break
            out[name.decode()] = (info.kernel_ms[i], info.kernel_launches[i])
        return out

    def kernel_work(self):
        """{kernel name: (kind, amount)}: kind 'flop32' | 'flop64' | 'byte' | 'tc_bf16'."""
        info = self.get_info()
        kinds = {1: "flop32", 2: "flop64", 3: "byte", 4: "tc_bf16"}
        out = {}
        for i in range(16):
            name = lib().dh2_kernel_name(i)
            if name is None:
                break
            if info.kernel_work_kind[i] in kinds:
                out[name.decode()] = (kinds[info.kernel_work_kind[i]], info.kernel_work[i])
        return out

    def matvec(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        return dh2_matvec(self.handle, x, y, stream)

    def matvec_host(self, x, stream=None):
        return dh2_matvec_host(self.handle, x, stream)

    def set_timing(self, on):
        _check(lib().dh2_set_timing(self.handle, 1 if on else 0))

    def directions(self, level):
        cnt = C.c_int32()
        ms = C.c_int32()
        _check(lib().dh2_export_directions(self.handle, level, C.byref(cnt), C.byref(ms), None, None))
        dirs = np.empty((cnt.value, 3))
        sd = np.empty(cnt.value, dtype=np.int32)
        _check(lib().dh2_export_directions(self.handle, level, C.byref(cnt), C.byref(ms), _ptr(dirs), _ptr(sd)))
        return ms.value, dirs, sd

    def blocks(self):
        info = self.info
        adm = np.empty((info.nadm, 3), dtype=np.int32)
        near = np.empty((info.nnear, 2), dtype=np.int32)
        active = np.empty(info.npairs, dtype=np.int8)
        _check(lib().dh2_export_blocks(self.handle, _ptr(adm), _ptr(near), _ptr(active)))
        return adm, near, active.astype(bool)

    def pair(self, which, tc):
        k = self.info.k
        cap = max(4 * k * k, 1)
        buf = np.empty(2 * cap)
        r = C.c_int32()
        c = C.c_int32()
        _check(lib().dh2_export_pair(self.handle, which, int(tc), _ptr(buf), cap, C.byref(r), C.byref(c)))
        return buf[: 2 * r.value * c.value].view(np.complex128).reshape(r.value, c.value)

    def ranks(self):
        rr = np.empty(self.info.npairs, dtype=np.int32)
        rc = np.empty(self.info.npairs, dtype=np.int32)
        _check(lib().dh2_export_ranks(self.handle, _ptr(rr), _ptr(rc)))
        return rr, rc

    def close(self):
        if getattr(self, "handle", None):
            dh2_free_matrix(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_batch(trees, kappas, m, eta, eps, precision=DH2_MIXED, eta1=10.0, rank_rule=DH2_RANK_BLOCKREL,
                nstreams=0, model=None, qr_tpc=(0, 0, 0), qr_group_rows=0, qr_fp64=1, svd_fp64=1, symmetry=1,
                gram_tc=1):
    """Concurrent builds (dh2_build_dh2_batch) wrapped as Matrix objects, in order."""
    opts = options(eta1=eta1, leaf_max=32, precision=precision, rank_rule=rank_rule, qr_tpc=qr_tpc,
                   qr_group_rows=qr_group_rows, qr_fp64=qr_fp64, svd_fp64=svd_fp64, symmetry=symmetry,
                   gram_tc=gram_tc)
    if model is not None:
        opts.learned = 1
        opts.model = model.handle
    handles = dh2_build_dh2_batch([t.handle for t in trees], kappas, m, eta, eps, opts, nstreams)
    return [Matrix.from_handle(h, precision) for h in handles]


def matvec_batch(mats, xs, ys=None, stream=None):
    """Overlapped products ys[i] = mats[i] xs[i] (dh2_matvec_batch)."""
    import torch
    if ys is None:
        ys = [torch.empty_like(x) for x in xs]
    return dh2_matvec_batch([m.handle for m in mats], xs, ys, stream)


# ----------------------------------------------------------------------------- learned order and rank

def _f32_cuda(a, cols):
    import torch
    if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
            and a.dim() == 2 and a.shape[1] == cols):
        raise TypeError(f"expected a contiguous CUDA float32 tensor of shape (n, {cols})")
    return a


class Model:
    """The learned order/rank MLP on the current GPU (owning handle, dh2_model_*)."""

    def __init__(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (DH2_MLP_NPARAMS,):
            raise ValueError(f"expected {DH2_MLP_NPARAMS} parameters")
        self.handle = C.c_void_p()
        _check(lib().dh2_model_create(_ptr(p), _stream(stream), C.byref(self.handle)))

    @classmethod
    def load(cls, path=None, stream=None):
        """The trained model shipped with the package (or the FP32 file at ``path``)."""
        return cls(np.fromfile(path or LEARNED_WEIGHTS, dtype="<f4"), stream)

    def params(self):
        out = np.empty(DH2_MLP_NPARAMS, dtype=np.float32)
        _check(lib().dh2_model_get_params(self.handle, _ptr(out)))
        return out

    def save(self, path):
        self.params().astype("<f4").tofile(path)

    def forward(self, X, stream=None):
        import torch
        X = _f32_cuda(X, DH2_MLP_IN)
        Y = torch.empty((X.shape[0], DH2_MLP_OUT), dtype=torch.float32, device=X.device)
        s = stream or torch.cuda.current_stream(X.device)
        _check(lib().dh2_model_forward(self.handle, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr()),
                                       _stream(s)))
        return Y

    def grad(self, X, T, stream=None):
        """(gradient [NPARAMS], loss [1]) as CUDA tensors."""
        import torch
        X, T = _f32_cuda(X, DH2_MLP_IN), _f32_cuda(T, DH2_MLP_OUT)
        g = torch.empty(DH2_MLP_NPARAMS, dtype=torch.float32, device=X.device)
        L = torch.empty(1, dtype=torch.float32, device=X.device)
        s = stream or torch.cuda.current_stream(X.device)
        _check(lib().dh2_model_grad(self.handle, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), X.shape[0],
                                    C.c_void_p(g.data_ptr()), C.c_void_p(L.data_ptr()), _stream(s)))
        return g, L

    def train_step(self, X, T, lr, loss=None, stream=None):
        """One Adam step on the batch; the batch loss (before the step) goes to ``loss`` if given."""
        import torch
        X, T = _f32_cuda(X, DH2_MLP_IN), _f32_cuda(T, DH2_MLP_OUT)
        s = stream or torch.cuda.current_stream(X.device)
        _check(lib().dh2_model_train_step(self.handle, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                          X.shape[0], float(lr), None if loss is None else C.c_void_p(loss.data_ptr()),
                                          _stream(s)))
        return loss

    def close(self):
        if getattr(self, "handle", None):
            lib().dh2_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def learned_features(tree: Tree, kappa, eta, eta1=10.0, stream=None):
    """(features [npairs, 8] CUDA float32 tensor, active [npairs] bool) for the block structure."""
    import torch
    opts = options(eta1=eta1)
    n = C.c_int64()
    _check(lib().dh2_learned_features(tree.handle, float(kappa), float(eta), C.byref(opts), _stream(stream), None, 0,
                                      C.byref(n), None))
    F = torch.empty((max(n.value, 1), DH2_MLP_IN), dtype=torch.float32, device="cuda")
    act = np.zeros(max(n.value, 1), dtype=np.int8)
    _check(lib().dh2_learned_features(tree.handle, float(kappa), float(eta), C.byref(opts), _stream(stream),
                                      C.c_void_p(F.data_ptr()), F.shape[0], C.byref(n), _ptr(act)))
    return F[: n.value], act[: n.value].astype(bool)


def learned_probe(tree: Tree, kappa, eta, eta1=10.0, stream=None):
    """Interpolation error [npairs, 6] of every pair at m = 3..8 (dh2_learned_probe)."""
    opts = options(eta1=eta1)
    n = C.c_int64()
    _check(lib().dh2_learned_probe(tree.handle, float(kappa), float(eta), C.byref(opts), _stream(stream), None, 0,
                                   C.byref(n)))
    err = np.zeros((max(n.value, 1), DH2_PROBE_ORDERS))
    _check(lib().dh2_learned_probe(tree.handle, float(kappa), float(eta), C.byref(opts), _stream(stream), _ptr(err),
                                   err.shape[0], C.byref(n)))
    return err[: n.value]
