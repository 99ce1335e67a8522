"""ctypes binding of the C ABI in include/xtc.h (argument marshalling only).

Every step of the xTC build runs inside ``libxtc.so``.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); they are passed to the library as plain pointers.  Loading
fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxtc.so")

PREC_FP64, PREC_FP16X2, PREC_BF16X3 = 0, 1, 2
PRECISIONS = {"fp64": PREC_FP64, "fp16x2": PREC_FP16X2, "bf16x3": PREC_BF16X3}
KERNEL_NAMES = ("prep", "vfield", "fields", "assemble", "final", "grad", "aux")

EXPORTED = ("xtc_default_params", "xtc_create", "xtc_destroy", "xtc_strerror", "xtc_last_error_detail",
            "xtc_set_jastrow", "xtc_set_outer_range", "xtc_build_1b2b", "xtc_jastrow_grad", "xtc_vfield",
            "xtc_get_timings", "xtc_vfield_noalloc", "xtc_build_1b2b_batched", "xtc_build_1b2b_rohf",
            "xtc_three_body_L", "xtc_autotune_chunk", "xtc_selftest_wait_timeout", "xtc_engine_revision",
            "xtc_selftest_reciprocals", "xtc_frozen_core_fold", "xtc_two_body_K")


class XtcParams(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("grid_chunk", ctypes.c_int64), ("split_k", ctypes.c_int), ("timing", ctypes.c_int),
                ("range_stages", ctypes.c_int), ("alloc", ctypes.c_void_p), ("release", ctypes.c_void_p),
                ("alloc_user", ctypes.c_void_p)]


# xtc_params.alloc / xtc_params.release
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class XtcInstance(ctypes.Structure):
    _fields_ = [("n_grid", ctypes.c_int64), ("n_orb", ctypes.c_int), ("grid_xyz", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("n_nuc", ctypes.c_int), ("nuc_xyz", ctypes.c_void_p), ("nuc_set", ctypes.c_void_p),
                ("n_sets", ctypes.c_int), ("n_terms", ctypes.c_int), ("mno", ctypes.c_void_p),
                ("coef", ctypes.c_void_p), ("dU", ctypes.c_void_p), ("dU_f32", ctypes.c_void_p),
                ("dh", ctypes.c_void_p), ("e0", ctypes.c_void_p), ("status", ctypes.c_int)]


class XtcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"xtc status {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Loads libxtc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    lib.xtc_default_params.argtypes = [ctypes.POINTER(XtcParams)]
    lib.xtc_default_params.restype = None
    lib.xtc_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(XtcParams)]
    lib.xtc_destroy.argtypes = [P]
    lib.xtc_strerror.argtypes = [I]
    lib.xtc_strerror.restype = ctypes.c_char_p
    lib.xtc_last_error_detail.argtypes = [P]
    lib.xtc_last_error_detail.restype = ctypes.c_char_p
    lib.xtc_set_jastrow.argtypes = [P, I, D, D, I, I, D, D]
    lib.xtc_set_outer_range.argtypes = [P, I64, I64]
    lib.xtc_build_1b2b.argtypes = [P, I64, I, D, D, D, D, D, D, D, D]
    lib.xtc_jastrow_grad.argtypes = [P, I64, D, D, D]
    lib.xtc_vfield.argtypes = [P, I64, I, D, D, D, I64, I64, D]
    lib.xtc_vfield_noalloc.argtypes = [P, I64, I, D, D, D, I64, I64, D]
    lib.xtc_get_timings.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), I]
    lib.xtc_build_1b2b_batched.argtypes = [P, I, ctypes.POINTER(XtcInstance), I]
    lib.xtc_build_1b2b_rohf.argtypes = [P, I64, I, D, D, D, D, D, D, D, D, D, D, D]
    lib.xtc_three_body_L.argtypes = [P, I64, I, D, D, D, D]
    lib.xtc_two_body_K.argtypes = [P, I64, I, D, D, D, D, D]
    lib.xtc_autotune_chunk.argtypes = [P, I64, I, D, D, D, D, ctypes.POINTER(ctypes.c_int64)]
    lib.xtc_selftest_wait_timeout.argtypes = [P, I]
    lib.xtc_engine_revision.argtypes = []
    lib.xtc_selftest_reciprocals.argtypes = [P, I64, D, D, D]
    lib.xtc_frozen_core_fold.argtypes = [P, I, D, D, I, ctypes.POINTER(ctypes.c_int), D, D, D]
    for name in ("xtc_create", "xtc_destroy", "xtc_set_jastrow", "xtc_set_outer_range", "xtc_build_1b2b",
                 "xtc_jastrow_grad", "xtc_vfield", "xtc_get_timings", "xtc_vfield_noalloc",
                 "xtc_build_1b2b_batched", "xtc_build_1b2b_rohf", "xtc_three_body_L", "xtc_autotune_chunk",
                 "xtc_selftest_wait_timeout", "xtc_engine_revision", "xtc_selftest_reciprocals",
                 "xtc_frozen_core_fold", "xtc_two_body_K"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def engine_revision() -> int:
    """Revision of the tensor-core GEMM engine (xtc_engine_revision)."""
    return int(load().xtc_engine_revision())


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _size(a):
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _need(a, n, name, dtype="float64"):
    """Checks that a (numpy array or tensor, or None) holds at least n elements of dtype: the
    library reads and writes exactly the sizes its arguments imply, so a short or mistyped buffer
    would be overrun in host or device memory."""
    if a is None:
        return None
    kind = str(a.dtype).replace("torch.", "")
    if kind != dtype:
        raise TypeError(f"{name} must be {dtype}, not {kind}")
    if _size(a) < n:
        raise ValueError(f"{name} holds {_size(a)} elements, {n} needed")
    return a


def _grid_inputs(grid, weights, phi):
    """n_grid, n_orb from phi ([n_grid][n_orb]) and the size checks of grid and weights."""
    if len(phi.shape) != 2:
        raise ValueError("phi must be [n_grid][n_orb]")
    n_grid, n_orb = int(phi.shape[0]), int(phi.shape[1])
    _need(grid, 3 * n_grid, "grid_xyz")
    _need(weights, n_grid, "weights")
    return n_grid, n_orb


def _f64(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    if hasattr(a, "dtype") and str(a.dtype) != "torch.float64":
        raise TypeError("float64 tensors are required")
    return a


class Context:
    """One library context (one device, one stream, one precision)."""

    def __init__(self, precision="fp16x2", device=0, stream=None, grid_chunk=0, split_k=0, timing=False,
                 range_stages=0, allocator=None):
        """allocator: optional pair (alloc, release) of Python callables, alloc(nbytes) -> device
        address (int, 0 when it cannot) and release(address), that supply the device workspace
        (for instance from torch's caching allocator); default cudaMalloc / cudaFree."""
        lib = load()
        self._lib = lib
        p = XtcParams()
        lib.xtc_default_params(ctypes.byref(p))
        p.device = device
        p.stream = stream
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.grid_chunk = grid_chunk
        p.split_k = split_k
        p.timing = 1 if timing else 0
        p.range_stages = range_stages
        self._alloc_cbs = None
        if allocator is not None:
            alloc_py, release_py = allocator
            self._alloc_cbs = (ALLOC_FN(lambda n, user: alloc_py(int(n)) or None),
                               RELEASE_FN(lambda ptr, user: release_py(int(ptr))))
            p.alloc = ctypes.cast(self._alloc_cbs[0], ctypes.c_void_p)
            p.release = ctypes.cast(self._alloc_cbs[1], ctypes.c_void_p)
        h = ctypes.c_void_p()
        rc = lib.xtc_create(ctypes.byref(h), ctypes.byref(p))
        if rc != 0:
            raise XtcError(rc, lib.xtc_strerror(rc).decode())
        self._h = h
        self.precision = precision
        self.device = int(device)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.xtc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc != 0:
            detail = self._lib.xtc_last_error_detail(self._h).decode()
            raise XtcError(rc, f"{self._lib.xtc_strerror(rc).decode()} ({detail})")

    def set_jastrow(self, nuc_xyz, nuc_set, terms, coef):
        nuc = np.ascontiguousarray(nuc_xyz, dtype=np.float64)
        ns = np.ascontiguousarray(nuc_set, dtype=np.int32)
        tm = np.ascontiguousarray(terms, dtype=np.int32)
        cf = np.ascontiguousarray(coef, dtype=np.float64)
        if nuc.ndim != 2 or nuc.shape[1] != 3 or ns.shape != (nuc.shape[0],):
            raise ValueError("nuc_xyz must be [n_nuc][3] and nuc_set [n_nuc]")
        if tm.ndim != 2 or tm.shape[1] != 3 or cf.ndim != 2 or cf.shape[1] != tm.shape[0]:
            raise ValueError("terms must be [n_terms][3] and coef [n_sets][n_terms]")
        self._check(self._lib.xtc_set_jastrow(self._h, nuc.shape[0], _ptr(nuc), _ptr(ns), cf.shape[0],
                                              tm.shape[0], _ptr(tm), _ptr(cf)))

    def set_outer_range(self, begin=0, end=-1):
        self._check(self._lib.xtc_set_outer_range(self._h, int(begin), int(end)))

    def build(self, grid, weights, phi, gamma, dU=None, dU_f32=None, dh=None, e0=None, want_dU=True):
        """Runs the build.  With numpy inputs and no outputs given, returns numpy outputs."""
        grid, weights, phi, gamma = _f64(grid), _f64(weights), _f64(phi), _f64(gamma)
        n_grid, n_orb = _grid_inputs(grid, weights, phi)
        _need(gamma, n_orb ** 2, "gamma")
        if dU is None and dU_f32 is None and want_dU:
            dU = np.empty((n_orb,) * 4)
        if dh is None:
            dh = np.empty((n_orb, n_orb))
        if e0 is None:
            e0 = np.empty(1)
        _need(dU, n_orb ** 4, "dU")
        _need(dU_f32, n_orb ** 4, "dU_f32", "float32")
        _need(dh, n_orb ** 2, "dh")
        _need(e0, 1, "e0")
        self._check(self._lib.xtc_build_1b2b(self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi),
                                             _ptr(gamma), _ptr(dU), _ptr(dU_f32), _ptr(dh), _ptr(e0)))
        return {"dU": dU if dU is not None else dU_f32, "dh": dh, "e0": e0}

    def build_rohf(self, grid, weights, phi, gamma_a, gamma_b, want_dU=True, **out):
        """The build for separate alpha and beta densities (xtc_build_1b2b_rohf).  Outputs may be
        given as keyword arguments dU_aa, dU_ab, dU_bb, dh_a, dh_b, e0 (numpy arrays or float64
        tensors); missing ones are allocated as numpy arrays (the Delta U blocks only with
        want_dU).  Returns them in a dict."""
        grid, weights, phi = _f64(grid), _f64(weights), _f64(phi)
        gamma_a, gamma_b = _f64(gamma_a), _f64(gamma_b)
        n_grid, n_orb = _grid_inputs(grid, weights, phi)
        _need(gamma_a, n_orb ** 2, "gamma_a")
        _need(gamma_b, n_orb ** 2, "gamma_b")
        res = {}
        for k in ("dU_aa", "dU_ab", "dU_bb"):
            res[k] = out.get(k)
            if res[k] is None and want_dU:
                res[k] = np.empty((n_orb,) * 4)
        for k in ("dh_a", "dh_b"):
            res[k] = out.get(k) if out.get(k) is not None else np.empty((n_orb, n_orb))
        res["e0"] = out.get("e0") if out.get("e0") is not None else np.empty(1)
        for k in ("dU_aa", "dU_ab", "dU_bb"):
            _need(res[k], n_orb ** 4, k)
        _need(res["dh_a"], n_orb ** 2, "dh_a")
        _need(res["dh_b"], n_orb ** 2, "dh_b")
        _need(res["e0"], 1, "e0")
        self._check(self._lib.xtc_build_1b2b_rohf(
            self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi), _ptr(gamma_a), _ptr(gamma_b),
            _ptr(res["dU_aa"]), _ptr(res["dU_ab"]), _ptr(res["dU_bb"]), _ptr(res["dh_a"]), _ptr(res["dh_b"]),
            _ptr(res["e0"])))
        return res

    def frozen_core_fold(self, dU, dh, core, dh_fc=None, dU_act=None, e_core=None, want_dU=False):
        """xTC-FC folding of (dU, dh) over the core orbital list ``core`` (xtc_frozen_core_fold):
        returns dh_fc [n_act][n_act], e_core [1] and, with want_dU or a given dU_act, the active
        block dU_act [n_act]^4.  Missing outputs are allocated as numpy arrays."""
        dU, dh = _f64(dU), _f64(dh)
        n_orb = int(dh.shape[0])
        _need(dU, n_orb ** 4, "dU")
        _need(dh, n_orb ** 2, "dh")
        idx = np.ascontiguousarray(np.asarray(core, dtype=np.int32).reshape(-1))
        n_act = n_orb - int(idx.size)
        if dh_fc is None:
            dh_fc = np.empty((max(n_act, 0),) * 2)
        if e_core is None:
            e_core = np.empty(1)
        if dU_act is None and want_dU:
            dU_act = np.empty((max(n_act, 0),) * 4)
        _need(dh_fc, max(n_act, 0) ** 2, "dh_fc")
        _need(dU_act, max(n_act, 0) ** 4, "dU_act")
        _need(e_core, 1, "e_core")
        core_ptr = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if idx.size else None
        self._check(self._lib.xtc_frozen_core_fold(self._h, n_orb, _ptr(dU), _ptr(dh), int(idx.size), core_ptr,
                                                   _ptr(dh_fc) if n_act > 0 else None, _ptr(dU_act),
                                                   _ptr(e_core)))
        return {"dh_fc": dh_fc, "dU_act": dU_act, "e_core": e_core}

    def selftest_reciprocals(self, x):
        """The refined 1/sqrt(x) and 1/x of the step (a) kernel on float32 x (xtc_selftest_reciprocals)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        ys, yr = np.empty_like(x), np.empty_like(x)
        self._check(self._lib.xtc_selftest_reciprocals(self._h, int(x.size), _ptr(x), _ptr(ys), _ptr(yr)))
        return ys, yr

    def selftest_wait_timeout(self, limit_ms=50):
        """Runs one bounded device wait that must time out; returns the status (XTC_ERR_TIMEOUT)."""
        return int(self._lib.xtc_selftest_wait_timeout(self._h, int(limit_ms)))

    def autotune_chunk(self, grid, weights, phi, gamma):
        """Times a few grid-chunk lengths on this problem and keeps the fastest for later builds
        (xtc_autotune_chunk); returns it."""
        grid, weights, phi, gamma = _f64(grid), _f64(weights), _f64(phi), _f64(gamma)
        n_grid, n_orb = _grid_inputs(grid, weights, phi)
        _need(gamma, n_orb ** 2, "gamma")
        c = ctypes.c_int64(0)
        self._check(self._lib.xtc_autotune_chunk(self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi),
                                                 _ptr(gamma), ctypes.byref(c)))
        return int(c.value)

    def three_body_L(self, grid, weights, phi, out=None):
        """The explicit three-body tensor of eq. Ldecomp (xtc_three_body_L): out[p, r, t, q, s, u] =
        L_prt^qsu over the context's outer range; a numpy array unless out is given."""
        grid, weights, phi = _f64(grid), _f64(weights), _f64(phi)
        n_grid, n_orb = _grid_inputs(grid, weights, phi)
        if out is None:
            out = np.empty((n_orb,) * 6)
        _need(out, n_orb ** 6, "L")
        self._check(self._lib.xtc_three_body_L(self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi),
                                               _ptr(out)))
        return out

    def two_body_K(self, grid, weights, phi, dphi, out=None):
        """The two-body integrals K of the similarity-transformed Hamiltonian (xtc_two_body_K):
        out[p, q, r, s] = K_pr^qs over the context's outer range, from the orbitals phi
        (n_grid, n_orb) and their gradients dphi (n_grid, n_orb, 3); a numpy array unless out is
        given."""
        grid, weights, phi, dphi = _f64(grid), _f64(weights), _f64(phi), _f64(dphi)
        n_grid, n_orb = _grid_inputs(grid, weights, phi)
        _need(dphi, n_grid * n_orb * 3, "dphi")
        if out is None:
            out = np.empty((n_orb,) * 4)
        _need(out, n_orb ** 4, "K")
        self._check(self._lib.xtc_two_body_K(self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi),
                                             _ptr(dphi), _ptr(out)))
        return out

    def jastrow_grad(self, r1, r2, out=None):
        r1, r2 = _f64(r1), _f64(r2)
        n = int(r1.shape[0])
        _need(r1, 3 * n, "r1")
        _need(r2, 3 * n, "r2")
        if out is None:
            out = np.empty((n, 3))
        _need(out, 3 * n, "out")
        self._check(self._lib.xtc_jastrow_grad(self._h, n, _ptr(r1), _ptr(r2), _ptr(out)))
        return out

    def vfield(self, grid, weights, phi, outer_begin, outer_end, out=None):
        grid, weights, phi = _f64(grid), _f64(weights), _f64(phi)
        n_grid, n_orb = _grid_inputs(grid, weights, phi)
        n_pair = n_orb * (n_orb + 1) // 2
        if out is None:
            out = np.empty((max(outer_end - outer_begin, 0), 3, n_pair))
        _need(out, max(outer_end - outer_begin, 0) * 3 * n_pair, "V")
        self._check(self._lib.xtc_vfield(self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi),
                                         int(outer_begin), int(outer_end), _ptr(out)))
        return out

    def vfield_noalloc(self, grid, weights, phi, outer_begin, outer_end, out):
        """xtc_vfield without device allocation: every argument must be a CUDA tensor (float64);
        workspace comes from the library's fixed scratch array (small problems only)."""
        for name, a in (("grid", grid), ("weights", weights), ("phi", phi), ("V", out)):
            dev = getattr(a, "device", None)
            if getattr(dev, "type", None) == "cuda" and dev.index is not None and dev.index != self.device:
                raise ValueError(f"{name} is on cuda:{dev.index}, the context on cuda:{self.device}")
        n_grid, n_orb = _grid_inputs(grid, _need(weights, 0, "weights"), _need(phi, 0, "phi"))
        _need(out, max(outer_end - outer_begin, 0) * 3 * (n_orb * (n_orb + 1) // 2), "V")
        self._check(self._lib.xtc_vfield_noalloc(self._h, n_grid, n_orb, _ptr(grid), _ptr(weights), _ptr(phi),
                                                 int(outer_begin), int(outer_end), _ptr(out)))
        return out

    def build_batched(self, instances, n_lanes=0, want_dU=True):
        """Batched build.  instances: list of dicts with keys nuc_xyz, nuc_set, terms, coef, grid,
        weights, phi, gamma (numpy arrays or float64 tensors) and optional outputs dU / dU_f32 / dh /
        e0; returns the list of output dicts {"dU", "dh", "e0"} in instance order."""
        n = len(instances)
        arr = (XtcInstance * max(n, 1))()
        keep, outs = [], []
        for k, d in enumerate(instances):
            grid, w, phi, gamma = _f64(d["grid"]), _f64(d["weights"]), _f64(d["phi"]), _f64(d["gamma"])
            nuc = np.ascontiguousarray(d["nuc_xyz"], dtype=np.float64)
            ns = np.ascontiguousarray(d["nuc_set"], dtype=np.int32)
            tm = np.ascontiguousarray(d["terms"], dtype=np.int32)
            cf = np.ascontiguousarray(d["coef"], dtype=np.float64)
            n_grid, n_orb = _grid_inputs(grid, w, phi)
            _need(gamma, n_orb ** 2, f"instance {k} gamma")
            if nuc.ndim != 2 or nuc.shape[1] != 3 or ns.shape != (nuc.shape[0],) or tm.ndim != 2 \
                    or tm.shape[1] != 3 or cf.ndim != 2 or cf.shape[1] != tm.shape[0]:
                raise ValueError(f"instance {k}: Jastrow arrays of inconsistent shapes")
            dU, dU32 = d.get("dU"), d.get("dU_f32")
            if dU is None and dU32 is None and want_dU:
                dU = np.empty((n_orb,) * 4)
            dh = d.get("dh") if d.get("dh") is not None else np.empty((n_orb, n_orb))
            e0 = d.get("e0") if d.get("e0") is not None else np.empty(1)
            _need(dU, n_orb ** 4, f"instance {k} dU")
            _need(dU32, n_orb ** 4, f"instance {k} dU_f32", "float32")
            _need(dh, n_orb ** 2, f"instance {k} dh")
            _need(e0, 1, f"instance {k} e0")
            keep += [grid, w, phi, gamma, nuc, ns, tm, cf, dU, dU32, dh, e0]
            it = arr[k]
            it.n_grid, it.n_orb = n_grid, n_orb
            it.grid_xyz, it.weights, it.phi, it.gamma = _ptr(grid), _ptr(w), _ptr(phi), _ptr(gamma)
            it.n_nuc, it.nuc_xyz, it.nuc_set = nuc.shape[0], _ptr(nuc), _ptr(ns)
            it.n_sets, it.n_terms, it.mno, it.coef = cf.shape[0], tm.shape[0], _ptr(tm), _ptr(cf)
            it.dU, it.dU_f32, it.dh, it.e0 = _ptr(dU), _ptr(dU32), _ptr(dh), _ptr(e0)
            outs.append({"dU": dU if dU is not None else dU32, "dh": dh, "e0": e0})
        self._check(self._lib.xtc_build_1b2b_batched(self._h, n, arr, int(n_lanes)))
        return outs

    def timings(self):
        n = len(KERNEL_NAMES)
        ms = (ctypes.c_double * n)()
        ln = (ctypes.c_int64 * n)()
        self._check(self._lib.xtc_get_timings(self._h, ms, ln, n))
        return {k: (ms[i], ln[i]) for i, k in enumerate(KERNEL_NAMES)}


def pair_index(n_orb):
    """(p, q) of every packed pair index, p <= q, row-major upper triangle."""
    p, q = np.triu_indices(n_orb)
    return p, q


def unpack_pairs(Vp, n_orb):
    """[..., n_pair] -> [..., n_orb, n_orb] symmetric."""
    p, q = pair_index(n_orb)
    out = np.zeros(Vp.shape[:-1] + (n_orb, n_orb))
    out[..., p, q] = Vp
    out[..., q, p] = Vp
    return out
