"""ctypes declarations of the libmglma C ABI (include/mglma.h)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MGLMA_FP64, MGLMA_FP32, MGLMA_BF16, MGLMA_FP16 = 0, 1, 2, 3
MGLMA_OP_D, MGLMA_OP_DDAG, MGLMA_OP_Q, MGLMA_OP_DDAGD = 0, 1, 2, 3
_STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "RANK", 5: "NOT_CONVERGED", 6: "NUMERIC",
           7: "TIMEOUT", 8: "REJECTED"}


class MglmaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"MGLMA_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    path = _build.LIB
    if _build.stale():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libmglma.so is missing and could not be built")
    return C.CDLL(path)


lib = _load()


class mglma_lattice(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("t_bc", C.c_int)]


_vp = C.c_void_p
_i64 = C.c_int64


def _sig(name, res, *args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("mglma_create", C.c_int, C.c_int, C.POINTER(_vp))
_sig("mglma_destroy", None, _vp)
_sig("mglma_last_error", C.c_char_p)
_sig("mglma_version", C.c_char_p)
_sig("mglma_profile", C.c_int, _vp, C.c_int, C.c_int)
_sig("mglma_profile_get", C.c_int, _vp, C.c_char_p, C.POINTER(C.c_longlong), C.POINTER(C.c_double))
_sig("mglma_gauge_load", C.c_int, _vp, C.POINTER(mglma_lattice), _vp, _i64, _i64, C.c_double, C.c_double,
     C.POINTER(_vp))
_sig("mglma_gauge_free", None, _vp)
_sig("mglma_gauge_info", C.c_int, _vp, C.POINTER(C.c_int), C.POINTER(_i64))
_sig("mglma_dirac_apply", C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_debug_tables", C.c_int, _vp, C.POINTER(C.c_int), _vp, _vp)


def _check(st: int):
    if st != 0:
        raise MglmaError(st, lib.mglma_last_error().decode())


def ptr(x):
    """Address of a numpy array (host) or a torch tensor (device or host)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def mglma_version() -> str:
    return lib.mglma_version().decode()


def mglma_last_error() -> str:
    return lib.mglma_last_error().decode()


def mglma_create(device: int = 0):
    h = _vp()
    _check(lib.mglma_create(device, C.byref(h)))
    return h


def mglma_destroy(ctx):
    lib.mglma_destroy(ctx)


class Context:
    """Owns an mglma context (stream + memory pool on one device)."""

    def __init__(self, device: int = 0):
        self.handle = mglma_create(device)
        self.device = device

    def close(self):
        if self.handle:
            mglma_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _h(x):
    return x.handle if hasattr(x, "handle") else x


def mglma_profile(ctx, enable: bool, reset: bool = False):
    _check(lib.mglma_profile(_h(ctx), int(enable), int(reset)))


def mglma_profile_get(ctx, name: str):
    n = C.c_longlong()
    ms = C.c_double()
    _check(lib.mglma_profile_get(_h(ctx), name.encode(), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def mglma_gauge_load(ctx, L, links, kappa, csw, t_bc=-1, t_begin=0, t_count=None, gauge=None):
    lat = mglma_lattice((C.c_int * 4)(*[int(v) for v in L]), int(t_bc))
    h = _vp(gauge) if gauge is not None else _vp()
    if t_count is None:
        t_count = int(L[0]) - t_begin
    _check(lib.mglma_gauge_load(_h(ctx), C.byref(lat), ptr(links), int(t_begin), int(t_count), float(kappa),
                                float(csw), C.byref(h)))
    return h.value


def mglma_gauge_free(g):
    lib.mglma_gauge_free(g)


def mglma_gauge_info(g):
    L = (C.c_int * 4)()
    V = _i64()
    _check(lib.mglma_gauge_info(g, L, C.byref(V)))
    return tuple(L), V.value


def mglma_dirac_apply(ctx, g, op, nrhs, inp, out, compute=MGLMA_FP64, stream=None):
    _check(lib.mglma_dirac_apply(_h(ctx), g, int(op), int(nrhs), ptr(inp), ptr(out), int(compute),
                                 _stream_ptr(stream)))


def mglma_debug_tables(g, block, nbr, block_of_site=None):
    b = (C.c_int * 4)(*block) if block is not None else None
    _check(lib.mglma_debug_tables(g, b, ptr(nbr), ptr(block_of_site)))
