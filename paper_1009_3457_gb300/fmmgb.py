"""Thin ctypes binding of libfmmgb (include/fmmgb.h), with the C entry points' names.

Argument marshalling only: torch tensors are passed by device pointer, the
stream is the caller's current torch stream.  Every step of the translation
path runs in the library's CUDA kernels; there is no fallback.  If the library
is missing, or there is no GPU, calls raise ``FmmError``.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmmgb.so")

FMM_OK = 0
FMM_EINVAL = -1
FMM_ENOMEM = -2
FMM_ECUDA = -3
FMM_ETIMEOUT = -4
FMM_EUNSUPPORTED = -5
FMM_EDEVICE = -6

FMM_FP32 = 0
FMM_TC_BF16X3 = 1
FMM_TC_BF16 = 2
FMM_TC_TF32X3 = 3

FMM_ACCUMULATE = 1
FMM_CONJ = 2
FMM_TREE_PERIODIC = 1
FMM_MAX_LEVEL = 14
FMM_BATCH_AUTOTUNE = 4
FMM_HOST_CONTIGUOUS = 8
FMM_P2P_SHARE_SM = 16

STATUS_NAMES = {0: "FMM_OK", -1: "FMM_EINVAL", -2: "FMM_ENOMEM", -3: "FMM_ECUDA", -4: "FMM_ETIMEOUT",
                -5: "FMM_EUNSUPPORTED", -6: "FMM_EDEVICE"}


class FmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class fmm_level_info(ctypes.Structure):
    _fields_ = [
        ("nbox", ctypes.c_int64),
        ("side", ctypes.c_int32),
        ("list_stride", ctypes.c_int32),
        ("ntranslations", ctypes.c_int64),
        ("list_host", ctypes.POINTER(ctypes.c_int32)),
        ("offcode_host", ctypes.POINTER(ctypes.c_int8)),
        ("list_dev", ctypes.c_void_p),
        ("offcode_dev", ctypes.c_void_p),
        ("nexist", ctypes.c_int64),
        ("exists_host", ctypes.POINTER(ctypes.c_uint8)),
    ]


class fmm_batch_info_t(ctypes.Structure):
    _fields_ = [
        ("items", ctypes.c_int64),
        ("translations", ctypes.c_int64),
        ("grid", ctypes.c_int32),
        ("chunk", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("tuned", ctypes.c_int32),
        ("tuned_ms", ctypes.c_float),
        ("variant", ctypes.c_int32),
        ("form", ctypes.c_int32),
        ("loads", ctypes.c_int32),
        ("from_cache", ctypes.c_int32),
    ]


class fmm_host_stream_info_t(ctypes.Structure):
    _fields_ = [
        ("entries", ctypes.c_int64),
        ("bytes_in", ctypes.c_int64),
        ("bytes_out", ctypes.c_int64),
        ("steps", ctypes.c_int64),
        ("depth", ctypes.c_int32),
        ("lmin", ctypes.c_int32),
        ("lmax", ctypes.c_int32),
        ("p", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("h2d_stream", ctypes.c_void_p),
        ("compute_stream", ctypes.c_void_p),
        ("d2h_stream", ctypes.c_void_p),
    ]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_d = ctypes.c_double
_f = ctypes.c_float

# name -> (restype, argtypes); the list of exported entry points of include/fmmgb.h
SIGNATURES = {
    "fmm_build_lists": (ctypes.c_int, [_vp, _i64, _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    "fmm_tree_level_info": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(fmm_level_info)]),
    "fmm_tree_translations": (ctypes.c_int64, [_vp, _i32]),
    "fmm_tree_destroy": (None, [_vp]),
    "fmm_prepare": (ctypes.c_int, [_i32, _i32]),
    "fmm_m2l": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp]),
    "fmm_m2l_adjoint": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp]),
    "fmm_m2l_levels": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                      _i32, _vp]),
    "fmm_m2l_adjoint_levels": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, ctypes.POINTER(_vp),
                                              ctypes.POINTER(_vp), _i32, _vp]),
    "fmm_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_i32), _i32, ctypes.POINTER(_vp),
                                        ctypes.POINTER(_vp), _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "fmm_batch_run": (ctypes.c_int, [_vp, _vp]),
    "fmm_batch_info": (ctypes.c_int, [_vp, ctypes.POINTER(fmm_batch_info_t)]),
    "fmm_batch_destroy": (None, [_vp, _vp]),
    "fmm_m2l_batched": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_i32), _i32, ctypes.POINTER(_vp),
                                       ctypes.POINTER(_vp), _i32, _i32, _vp]),
    "fmm_host_stream_create": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, _i32, ctypes.POINTER(_vp)]),
    "fmm_host_stream_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32]),
    "fmm_host_stream_sync": (ctypes.c_int, [_vp]),
    "fmm_host_stream_info": (ctypes.c_int, [_vp, ctypes.POINTER(fmm_host_stream_info_t)]),
    "fmm_host_stream_destroy": (None, [_vp]),
    "fmm_m2m_adjoint": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _vp]),
    "fmm_l2l": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _vp]),
    "fmm_l2l_adjoint": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _vp]),
    "fmm_leaf_boxes": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "fmm_l2p": (ctypes.c_int, [_i32, _i64, _vp, _vp, _vp, ctypes.POINTER(_vp), _i32, _vp, _i32, _vp]),
    "fmm_l2p_adjoint": (ctypes.c_int, [_i32, _i64, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp), _i32, _vp]),
    "fmm_p2m_adjoint": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i64, _vp, _vp, _i32, _vp]),
    "fmm_p2m": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i64, _vp, _i32, _vp]),
    "fmm_m2m": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _vp]),
    "fgt_h2t": (ctypes.c_int, [_i32, _i32, _i32, _i32, _d, _vp, _vp, _vp, _i32, _vp]),
    "fgt_h2t_noalloc": (ctypes.c_int, [_i32, _i32, _i32, _d, _vp, _vp, _i32, _vp]),
    "fgt_t2p": (ctypes.c_int, [_i32, _i32, _d, _vp, _vp, _i64, _vp, _i32, _vp]),
    "fgt_p2h": (ctypes.c_int, [_i32, _i32, _d, _vp, _vp, _i64, _vp, _i32, _vp]),
    "fgt_bin_points": (ctypes.c_int, [_i32, _vp, _i64, _vp, _vp, _vp, _vp]),
    "fmm_bin_points": (ctypes.c_int, [_i32, _vp, _i64, _vp, _vp, _vp, _vp]),
    "fmm_m2l_paper_design": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _i32, _vp]),
    "fmm_p2m_binned": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _vp]),
    "fmm_l2p_binned": (ctypes.c_int, [_i32, _i32, _vp, _i64, _vp, _vp, _vp, _vp, _i32, _vp]),
    "fgt_t2p_binned": (ctypes.c_int, [_i32, _i32, ctypes.c_double, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _vp]),
    "fmm_p2p": (ctypes.c_int, [_i32, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _vp]),
    "fgt_p2h_binned": (ctypes.c_int, [_i32, _i32, _d, _vp, _vp, _i64, _vp, _vp, _i32, _vp]),
    "fgt_h2p": (ctypes.c_int, [_i32, _i32, _i32, _i32, _d, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _vp]),
    "fmm_wait_probe": (ctypes.c_int, [_i32, _i32, _vp]),
    "fmm_sync_status": (ctypes.c_int, [_vp]),
    "fmm_last_error": (ctypes.c_char_p, []),
    "fmm_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfmmgb.so (raises FmmError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FmmError(FMM_EUNSUPPORTED, f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            if not hasattr(lib, name):
                continue
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != FMM_OK:
        raise FmmError(rc, load().fmm_last_error().decode())


def _ptr(t) -> int:
    """Device pointer of a CUDA tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise FmmError(FMM_EINVAL, "tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise FmmError(FMM_EINVAL, "tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Tree:
    """Owning wrapper of an ``fmm_tree*`` handle."""

    def __init__(self, handle: int, max_level: int, periodic: bool, leaf_cap: int = 0):
        self.handle = handle
        self.max_level = max_level
        self.periodic = periodic
        self.leaf_cap = leaf_cap
        self.adaptive = leaf_cap > 0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.fmm_tree_destroy(h)
            self.handle = None

    def translations(self, level: int) -> int:
        return int(load().fmm_tree_translations(self.handle, level))

    def level_info(self, level: int) -> fmm_level_info:
        info = fmm_level_info()
        _check(load().fmm_tree_level_info(self.handle, level, ctypes.byref(info)))
        return info

    def exists(self, level: int):
        """Box existence of a level, numpy bool [4^level] (all True on a uniform tree)."""
        import numpy as np

        info = self.level_info(level)
        if not info.exists_host:
            return np.ones(info.nbox, dtype=bool)
        return np.ctypeslib.as_array(info.exists_host, shape=(info.nbox,)).astype(bool)

    def lists(self, level: int):
        """Host copies of the level's lists: (list [nbox, 27] int32, offset codes [nbox, 27] int8)."""
        import numpy as np

        info = self.level_info(level)
        n = info.nbox * info.list_stride
        lst = np.ctypeslib.as_array(info.list_host, shape=(n,)).reshape(info.nbox, info.list_stride).copy()
        code = np.ctypeslib.as_array(info.offcode_host, shape=(n,)).reshape(info.nbox, info.list_stride).copy()
        return lst, code


def fmm_build_lists(xy=None, max_level: int = 2, leaf_cap: int = 0, periodic: bool = False) -> Tree:
    import numpy as np

    lib = load()
    h = _vp()
    if xy is not None:
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        n = xy.shape[0]
        xp = xy.ctypes.data
    else:
        n, xp = 0, None
    _check(lib.fmm_build_lists(xp, n, max_level, leaf_cap, FMM_TREE_PERIODIC if periodic else 0, ctypes.byref(h)))
    return Tree(h.value, max_level, periodic, leaf_cap)


def fmm_prepare(p: int, prec: int = FMM_FP32):
    _check(load().fmm_prepare(p, prec))


def fmm_m2l(tree: Tree, level: int, p: int, M, L, prec: int = FMM_FP32, accumulate: bool = False, stream=None):
    _check(load().fmm_m2l(tree.handle, level, p, prec, _ptr(M), _ptr(L), FMM_ACCUMULATE if accumulate else 0,
                          _stream(stream)))


def fmm_m2l_adjoint(tree: Tree, level: int, p: int, W, G, prec: int = FMM_FP32, accumulate: bool = False,
                    conj: bool = False, stream=None):
    flags = (FMM_ACCUMULATE if accumulate else 0) | (FMM_CONJ if conj else 0)
    _check(load().fmm_m2l_adjoint(tree.handle, level, p, prec, _ptr(W), _ptr(G), flags, _stream(stream)))


def _ptr_array(ts):
    return (_vp * len(ts))(*[_ptr(t) for t in ts])


def fmm_m2l_levels(tree: Tree, lmin: int, p: int, Ms, Ls, prec: int = FMM_FP32, accumulate: bool = False,
                   stream=None):
    """One launch over levels lmin .. lmin + len(Ms) - 1; Ms[i], Ls[i] belong to level lmin + i."""
    assert len(Ms) == len(Ls) and len(Ms) > 0
    _check(load().fmm_m2l_levels(tree.handle, lmin, lmin + len(Ms) - 1, p, prec, _ptr_array(Ms), _ptr_array(Ls),
                                 FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_m2l_adjoint_levels(tree: Tree, lmin: int, p: int, Ws, Gs, prec: int = FMM_FP32, accumulate: bool = False,
                           conj: bool = False, stream=None):
    assert len(Ws) == len(Gs) and len(Ws) > 0
    flags = (FMM_ACCUMULATE if accumulate else 0) | (FMM_CONJ if conj else 0)
    _check(load().fmm_m2l_adjoint_levels(tree.handle, lmin, lmin + len(Ws) - 1, p, prec, _ptr_array(Ws),
                                         _ptr_array(Gs), flags, _stream(stream)))


def _batch_args(trees, ps, Ms, Ls):
    """Marshal a batch: Ms[i], Ls[i] are problem i's level lists (levels 2..trees[i].max_level)."""
    n = len(trees)
    assert len(ps) == n and len(Ms) == n and len(Ls) == n and n > 0
    flatM, flatL = [], []
    for t, m, l in zip(trees, Ms, Ls):
        if len(m) != t.max_level - 1 or len(l) != t.max_level - 1:
            raise FmmError(FMM_EINVAL, "each problem needs one M and one L per level 2..max_level")
        flatM += list(m)
        flatL += list(l)
    return ((_vp * n)(*[t.handle for t in trees]), (_i32 * n)(*[int(p) for p in ps]), n, _ptr_array(flatM),
            _ptr_array(flatL))


class Batch:
    """Owning wrapper of an ``fmm_batch*`` plan (fmm_batch_create / run / info / destroy)."""

    def __init__(self, handle: int, keep, stream):
        self.handle = handle
        self._keep = keep  # the trees and coefficient tensors the plan points into
        self._stream = stream  # the plan's device arrays are freed in order on the last stream used

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.fmm_batch_destroy(h, self._stream)
            self.handle = None

    def run(self, stream=None):
        self._stream = _stream(stream)
        _check(load().fmm_batch_run(self.handle, self._stream))

    def info(self) -> dict:
        inf = fmm_batch_info_t()
        _check(load().fmm_batch_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in fmm_batch_info_t._fields_}


def fmm_batch_create(trees, ps, Ms, Ls, prec: int = FMM_FP32, accumulate: bool = False, autotune: bool = False,
                     stream=None) -> Batch:
    tr, pa, n, mp, lp = _batch_args(trees, ps, Ms, Ls)
    flags = (FMM_ACCUMULATE if accumulate else 0) | (FMM_BATCH_AUTOTUNE if autotune else 0)
    h = _vp()
    st = _stream(stream)
    _check(load().fmm_batch_create(tr, pa, n, mp, lp, prec, flags, st, ctypes.byref(h)))
    return Batch(h.value, (list(trees), [list(m) for m in Ms], [list(l) for l in Ls]), st)


def fmm_m2l_batched(trees, ps, Ms, Ls, prec: int = FMM_FP32, accumulate: bool = False, stream=None):
    tr, pa, n, mp, lp = _batch_args(trees, ps, Ms, Ls)
    _check(load().fmm_m2l_batched(tr, pa, n, mp, lp, prec, FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def _host_ptr(t) -> int:
    """Host address of a CPU tensor (or an int address)."""
    if isinstance(t, int):
        return t
    if t.is_cuda:
        raise FmmError(FMM_EINVAL, "tensor must live in host memory")
    if not t.is_contiguous():
        raise FmmError(FMM_EINVAL, "tensor must be contiguous")
    return t.data_ptr()


class HostStream:
    """Owning wrapper of an ``fmm_host_stream*`` (fmm_host_stream_create / submit / sync / info / destroy)."""

    def __init__(self, handle: int, tree: Tree, nlev: int, entries: int):
        self.handle = handle
        self._tree = tree  # the pipeline points into the tree's lists
        self.nlev = nlev
        self.entries = entries

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.fmm_host_stream_destroy(h)
            self.handle = None

    def submit(self, M_host, L_host):
        """One step.  M_host, L_host: per-level lists of host tensors (levels lmin..lmax; one copy
        per level), or one complex64 host tensor each holding every level back to back (one copy
        per direction, FMM_HOST_CONTIGUOUS)."""
        if isinstance(M_host, list) and isinstance(L_host, list):
            if len(M_host) != self.nlev or len(L_host) != self.nlev:
                raise FmmError(FMM_EINVAL, f"one M and one L per level ({self.nlev} levels)")
            mp = (_vp * self.nlev)(*[_host_ptr(t) for t in M_host])
            lp = (_vp * self.nlev)(*[_host_ptr(t) for t in L_host])
            flags = 0
        else:
            for t in (M_host, L_host):
                if isinstance(t, list) or t.numel() != self.entries:
                    raise FmmError(FMM_EINVAL, f"a flat buffer holds all {self.entries} entries")
            mp, lp = (_vp * 1)(_host_ptr(M_host)), (_vp * 1)(_host_ptr(L_host))
            flags = FMM_HOST_CONTIGUOUS
        _check(load().fmm_host_stream_submit(self.handle, mp, lp, flags))

    def sync(self):
        _check(load().fmm_host_stream_sync(self.handle))

    def info(self) -> dict:
        inf = fmm_host_stream_info_t()
        _check(load().fmm_host_stream_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in fmm_host_stream_info_t._fields_}


def fmm_host_stream_create(tree: Tree, lmin: int, lmax: int, p: int, prec: int = FMM_FP32,
                           depth: int = 2) -> HostStream:
    h = _vp()
    _check(load().fmm_host_stream_create(tree.handle, lmin, lmax, p, prec, depth, ctypes.byref(h)))
    return HostStream(h.value, tree, lmax - lmin + 1, p * sum(4 ** l for l in range(lmin, lmax + 1)))


def fmm_p2m(level: int, p: int, xy, c, M, accumulate: bool = False, stream=None):
    n = 0 if c is None else c.numel()
    _check(load().fmm_p2m(level, p, _ptr(xy), _ptr(c), n, _ptr(M), FMM_ACCUMULATE if accumulate else 0,
                          _stream(stream)))


def fmm_p2m_binned(level: int, p: int, xy, c, perm, box_start, M, accumulate: bool = False, stream=None):
    """fmm_p2m for points binned by fmm_bin_points at `level` (deterministic, no atomics)."""
    n = 0 if c is None else c.numel()
    _check(load().fmm_p2m_binned(level, p, _ptr(xy), _ptr(c), n, _ptr(perm), _ptr(box_start), _ptr(M),
                                 FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_m2m(child_level: int, p: int, Mc, Mp, accumulate: bool = False, stream=None):
    _check(load().fmm_m2m(child_level, p, _ptr(Mc), _ptr(Mp), FMM_ACCUMULATE if accumulate else 0,
                          _stream(stream)))


def fmm_m2m_adjoint(child_level: int, p: int, Wp, Wc, accumulate: bool = False, stream=None):
    _check(load().fmm_m2m_adjoint(child_level, p, _ptr(Wp), _ptr(Wc), FMM_ACCUMULATE if accumulate else 0,
                                  _stream(stream)))


def fmm_l2l(child_level: int, p: int, Lp, Lc, accumulate: bool = False, stream=None):
    _check(load().fmm_l2l(child_level, p, _ptr(Lp), _ptr(Lc), FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_l2l_adjoint(child_level: int, p: int, Wc, Wp, accumulate: bool = False, stream=None):
    _check(load().fmm_l2l_adjoint(child_level, p, _ptr(Wc), _ptr(Wp), FMM_ACCUMULATE if accumulate else 0,
                                  _stream(stream)))


def _level_table(arrays, max_level):
    """Host array of max_level + 1 device pointers from {level: tensor} (NULL where absent)."""
    return (_vp * (max_level + 1))(*[_ptr(arrays[l]) if l in arrays else None for l in range(max_level + 1)])


def fmm_leaf_boxes(tree, xy, level, box, stream=None):
    """Deepest existing box of `tree` holding each point: level (int32 [n]), box (int64 [n])."""
    n = 0 if level is None else level.numel()
    _check(load().fmm_leaf_boxes(tree.handle, _ptr(xy), n, _ptr(level), _ptr(box), _stream(stream)))


def fmm_l2p(p: int, z, lev, box, L_levels: dict, max_level: int, phi, accumulate: bool = False, stream=None):
    """phi (complex64 [n]) from the LEs of each point's (lev, box); L_levels: {level: [4^l, p] complex64}."""
    n = 0 if lev is None else lev.numel()
    _check(load().fmm_l2p(p, n, _ptr(z), _ptr(lev), _ptr(box), _level_table(L_levels, max_level), max_level,
                          _ptr(phi), FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_l2p_binned(level: int, p: int, z, perm, box_start, L, phi, accumulate: bool = False, stream=None):
    """fmm_l2p at the points z of level `level`, binned by fmm_bin_points (one block per box)."""
    n = 0 if perm is None else perm.numel()
    _check(load().fmm_l2p_binned(level, p, _ptr(z), n, _ptr(perm), _ptr(box_start), _ptr(L), _ptr(phi),
                                 FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_l2p_adjoint(p: int, z, lev, box, cot, G_levels: dict, max_level: int, stream=None):
    n = 0 if lev is None else lev.numel()
    _check(load().fmm_l2p_adjoint(p, n, _ptr(z), _ptr(lev), _ptr(box), _ptr(cot), _level_table(G_levels, max_level),
                                  max_level, _stream(stream)))


def fmm_p2m_adjoint(level: int, p: int, xy, c, G, grad, accumulate: bool = False, stream=None):
    n = 0 if c is None else c.numel()
    _check(load().fmm_p2m_adjoint(level, p, _ptr(xy), _ptr(c), n, _ptr(G), _ptr(grad),
                                  FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_h2t(grid_log2: int, n_cut: int, p: int, sigma: float, A, C, work=None, accumulate: bool = False,
            stream=None, prec: int = FMM_FP32):
    _check(load().fgt_h2t(grid_log2, n_cut, p, prec, float(sigma), _ptr(A), _ptr(C), _ptr(work),
                          FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_h2t_noalloc(grid_log2: int, n_cut: int, p: int, sigma: float, A, C, accumulate: bool = False,
                    stream=None):
    """fgt_h2t with its intermediate in the library's built-in scratch array (no device allocation)."""
    _check(load().fgt_h2t_noalloc(grid_log2, n_cut, p, float(sigma), _ptr(A), _ptr(C),
                                  FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_p2h(grid_log2: int, p: int, sigma: float, x, q, A, accumulate: bool = False, stream=None):
    n = 0 if q is None else q.numel()
    _check(load().fgt_p2h(grid_log2, p, float(sigma), _ptr(x), _ptr(q), n, _ptr(A),
                          FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_t2p(grid_log2: int, p: int, sigma: float, C, y, G, accumulate: bool = False, stream=None):
    """G (float32 [n]) at the targets y (float64 [n, 2]) from the Taylor coefficients C of their boxes."""
    n = 0 if G is None else G.numel()
    _check(load().fgt_t2p(grid_log2, p, float(sigma), _ptr(C), _ptr(y), n, _ptr(G),
                          FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_t2p_binned(grid_log2: int, p: int, sigma: float, C, y, perm, box_start, G, accumulate: bool = False,
                   stream=None):
    """fgt_t2p at targets binned by fgt_bin_points (one block per box, coefficients in shared memory)."""
    n = 0 if perm is None else perm.numel()
    _check(load().fgt_t2p_binned(grid_log2, p, float(sigma), _ptr(C), _ptr(y), n, _ptr(perm), _ptr(box_start),
                                 _ptr(G), FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_bin_points(grid_log2: int, y, perm, box_start, work, stream=None):
    """Counting sort of the points y (float64 [n, 2]) by box of the 2^g grid: perm (int32 [n])
    lists the points box by box, box_start (int32 [4^g + 1]) where each box's run begins;
    work: int32 [4^g] scratch."""
    n = 0 if y is None else y.shape[0]
    _check(load().fgt_bin_points(grid_log2, _ptr(y), n, _ptr(perm), _ptr(box_start), _ptr(work),
                                 _stream(stream)))


def fmm_m2l_paper_design(tree: Tree, level: int, p: int, M, L, work, accumulate: bool = False, stream=None):
    """The paper's two-kernel M2L (per-translation LEs in `work`, then a reduction); for comparison."""
    _check(load().fmm_m2l_paper_design(tree.handle, level, p, _ptr(M), _ptr(L), _ptr(work),
                                       FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_bin_points(level: int, y, perm, box_start, work, stream=None):
    """fgt_bin_points on the boxes of quadtree level `level`."""
    n = 0 if y is None else y.shape[0]
    _check(load().fmm_bin_points(level, _ptr(y), n, _ptr(perm), _ptr(box_start), _ptr(work), _stream(stream)))


def fmm_p2p(level: int, xy, c, src_perm, src_start, z, tgt_perm, tgt_start, phi, accumulate: bool = False,
            stream=None, share_sm: bool = False):
    """Near field at the finest level of a uniform tree: phi (complex64 [nz]) at the targets z
    (float64 [nz, 2]) from the sources xy, c in the own and adjacent boxes; both sets binned
    by fmm_bin_points at `level`.  share_sm: leave room on every SM for kernels of other
    streams (FMM_P2P_SHARE_SM)."""
    n = 0 if c is None else c.numel()
    nz = 0 if z is None else z.shape[0]
    flags = (FMM_ACCUMULATE if accumulate else 0) | (FMM_P2P_SHARE_SM if share_sm else 0)
    _check(load().fmm_p2p(level, _ptr(xy), _ptr(c), n, _ptr(src_perm), _ptr(src_start), _ptr(z), nz,
                          _ptr(tgt_perm), _ptr(tgt_start), _ptr(phi), flags, _stream(stream)))


def fgt_p2h_binned(grid_log2: int, p: int, sigma: float, x, q, perm, A, accumulate: bool = False, stream=None):
    """fgt_p2h for sources binned by fgt_bin_points (perm)."""
    n = 0 if q is None else q.numel()
    _check(load().fgt_p2h_binned(grid_log2, p, float(sigma), _ptr(x), _ptr(q), n, _ptr(perm), _ptr(A),
                                 FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fgt_h2p(grid_log2: int, n_cut: int, p: int, sigma: float, A, y, perm, box_start, G, accumulate: bool = False,
            prec: int = FMM_FP32, stream=None):
    """G (float32 [n]) at the targets y (float64 [n, 2], binned by fgt_bin_points into perm and
    box_start) from the Hermite coefficients A of every box within n_cut of each target's box.
    prec: FMM_FP32 (CUDA cores), FMM_TC_BF16X3 or FMM_TC_BF16 (tensor cores, p = 16)."""
    n = 0 if G is None else G.numel()
    _check(load().fgt_h2p(grid_log2, n_cut, p, prec, float(sigma), _ptr(A), _ptr(y), n, _ptr(perm),
                          _ptr(box_start), _ptr(G), FMM_ACCUMULATE if accumulate else 0, _stream(stream)))


def fmm_wait_probe(polls: int, arrive: bool, stream=None):
    """Launch the bounded-wait probe (see include/fmmgb.h); read the outcome with fmm_sync_status."""
    _check(load().fmm_wait_probe(int(polls), 1 if arrive else 0, _stream(stream)))


def fmm_sync_status(stream=None):
    _check(load().fmm_sync_status(_stream(stream)))


def fmm_last_error() -> str:
    return load().fmm_last_error().decode()


def fmm_version() -> str:
    return load().fmm_version().decode()
