"""ctypes declarations of the libmglma C ABI (include/mglma.h)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MGLMA_FP64, MGLMA_FP32, MGLMA_BF16, MGLMA_FP16 = 0, 1, 2, 3
MGLMA_OP_D, MGLMA_OP_DDAG, MGLMA_OP_Q, MGLMA_OP_DDAGD, MGLMA_OP_SCHUR, MGLMA_OP_SCHUR_Q = 0, 1, 2, 3, 4, 5
MGLMA_COARSE_GCR, MGLMA_COARSE_MINRES, MGLMA_COARSE_MINRES_EO = 0, 1, 2
MGLMA_SOLVER_CGNE, MGLMA_SOLVER_MG, MGLMA_SOLVER_CGNE_EO = 0, 1, 2
MGLMA_SOURCE_Z2, MGLMA_SOURCE_Z4, MGLMA_SOURCE_POINT = 0, 1, 2
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
_sig("mglma_profile_get", C.c_int, _vp, C.c_char_p, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
     C.POINTER(C.c_double), C.POINTER(C.c_double))
_sig("mglma_gauge_load", C.c_int, _vp, C.POINTER(mglma_lattice), _vp, _i64, _i64, C.c_double, C.c_double,
     C.POINTER(_vp))
_sig("mglma_gauge_random", C.c_int, _vp, C.POINTER(mglma_lattice), C.c_double, C.c_uint64, C.c_double, C.c_double,
     C.POINTER(_vp))
_sig("mglma_gauge_free", None, _vp)
_sig("mglma_gauge_info", C.c_int, _vp, C.POINTER(C.c_int), C.POINTER(_i64))
_sig("mglma_dirac_apply", C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_debug_tables", C.c_int, _vp, C.POINTER(C.c_int), _vp, _vp)
_sig("mglma_dirac_apply_noalloc", C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_subspace_build", C.c_int, _vp, _vp, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_uint64, C.c_int,
     C.POINTER(_vp))
class mglma_subspace_params(C.Structure):
    _fields_ = [("block", C.c_int * 4), ("nv", C.c_int), ("n_smooth", C.c_int), ("n_cg", C.c_int),
                ("cg_prec", C.c_int), ("seed", C.c_uint64), ("store", C.c_int), ("lean_group", C.c_int)]


_sig("mglma_subspace_create", C.c_int, _vp, _vp, C.POINTER(mglma_subspace_params), C.POINTER(_vp))
_sig("mglma_subspace_load", C.c_int, _vp, _vp, C.POINTER(C.c_int), C.c_int, _vp, C.c_int, C.POINTER(_vp))
_sig("mglma_subspace_free", None, _vp)
_sig("mglma_subspace_info", C.c_int, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_i64))
_sig("mglma_subspace_export", C.c_int, _vp, _vp)
_sig("mglma_restrict", C.c_int, _vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_prolong", C.c_int, _vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_coarse_build", C.c_int, _vp, _vp, _vp, C.c_int, C.POINTER(_vp))
_sig("mglma_coarse_free", None, _vp)
_sig("mglma_coarse_release_fp64", C.c_int, _vp)
_sig("mglma_coarse_info", C.c_int, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_i64))
_sig("mglma_coarse_export", C.c_int, _vp, _vp)
_sig("mglma_coarse_apply", C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_coarse_build_next", C.c_int, _vp, _vp, C.POINTER(C.c_int), C.c_int, C.POINTER(_vp))
_sig("mglma_coarse_restrict", C.c_int, _vp, _vp, C.c_int, _vp, _vp, _vp)
_sig("mglma_coarse_prolong", C.c_int, _vp, _vp, C.c_int, _vp, _vp, _vp)
_sig("mglma_pieces", C.c_int, _vp, _vp, C.POINTER(_vp), C.c_int, C.c_int, _vp, _vp, C.c_double, _vp)
_sig("mglma_coarse_gamma5_gamma", C.c_int, _vp, _vp, C.c_int, _vp)
_sig("mglma_coarse_dense_inverse", C.c_int, _vp, _vp, _vp)
_sig("mglma_exact_correlator", C.c_int, _vp, _vp, _vp, _vp)


class mglma_solve_params(C.Structure):
    _fields_ = [("method", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("gcr_m", C.c_int),
                ("nu", C.c_int), ("inner_tol", C.c_double), ("coarse_tol", C.c_double),
                ("coarse_max_iter", C.c_int), ("check_every", C.c_int), ("max_batch", C.c_int),
                ("coarse_solver", C.c_int), ("autotune", C.c_int), ("graph", C.c_int)]


class mglma_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("coarse_iterations", C.c_longlong),
                ("residual", C.c_double), ("converged", C.c_int), ("batch", C.c_int)]


_sig("mglma_sources", C.c_int, _vp, C.POINTER(mglma_lattice), C.c_int, C.c_int, C.c_uint64, _i64,
     C.POINTER(_i64), C.POINTER(C.c_int), C.c_int, _vp, _vp)
_sig("mglma_autotune", C.c_int, _vp, _vp, _vp, C.c_int)
_sig("mglma_autotune_get", C.c_int, _vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double))
_sig("mglma_contract", C.c_int, _vp, C.POINTER(mglma_lattice), C.c_int, _vp, _vp, _vp, _vp)
_sig("mglma_gamma5_gamma", C.c_int, _vp, C.POINTER(mglma_lattice), C.c_int, C.c_int, _vp, _vp, _vp)
_sig("mglma_autotune_set", C.c_int, _vp, C.c_int, C.c_int, C.c_int)
_sig("mglma_autotune_save", C.c_int, _vp, C.c_char_p)
_sig("mglma_autotune_load", C.c_int, _vp, C.c_char_p)
_sig("mglma_solve_params_default", None, C.POINTER(mglma_solve_params), C.c_int)
_sig("mglma_solve_batch", C.c_int, _vp, _vp, _vp, C.POINTER(mglma_solve_params), C.c_int, C.POINTER(C.c_int), _vp,
     _vp, _vp, C.POINTER(mglma_solve_stats), _vp)


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
    """(launches, milliseconds, algorithmic bytes, algorithmic flops) of a kernel class."""
    n = C.c_longlong()
    ms, by, fl = C.c_double(), C.c_double(), C.c_double()
    _check(lib.mglma_profile_get(_h(ctx), name.encode(), C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
    return n.value, ms.value, by.value, fl.value


def mglma_gauge_load(ctx, L, links, kappa, csw, t_bc=-1, t_begin=0, t_count=None, gauge=None):
    lat = mglma_lattice((C.c_int * 4)(*[int(v) for v in L]), int(t_bc))
    h = _vp(gauge) if gauge is not None else _vp()
    if t_count is None:
        t_count = int(L[0]) - t_begin
    _check(lib.mglma_gauge_load(_h(ctx), C.byref(lat), ptr(links), int(t_begin), int(t_count), float(kappa),
                                float(csw), C.byref(h)))
    return h.value


def mglma_gauge_random(ctx, L, eps, seed, kappa, csw, t_bc=-1):
    """Gauge field from the seeded link recipe, generated on the device."""
    lat = mglma_lattice((C.c_int * 4)(*[int(v) for v in L]), int(t_bc))
    h = _vp()
    _check(lib.mglma_gauge_random(_h(ctx), C.byref(lat), float(eps), int(seed), float(kappa), float(csw),
                                  C.byref(h)))
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


def mglma_dirac_apply_noalloc(ctx, g, op, nrhs, inp, out, compute=MGLMA_FP64, stream=None):
    """Allocation-free mglma_dirac_apply: device buffers only, nrhs x V
    bounded by the library's 32 MiB scratch array (see include/mglma.h)."""
    _check(lib.mglma_dirac_apply_noalloc(_h(ctx), g, int(op), int(nrhs), ptr(inp), ptr(out), int(compute),
                                         _stream_ptr(stream)))


def mglma_debug_tables(g, block, nbr, block_of_site=None):
    b = (C.c_int * 4)(*block) if block is not None else None
    _check(lib.mglma_debug_tables(g, b, ptr(nbr), ptr(block_of_site)))


def _block(b):
    return (C.c_int * 4)(*[int(v) for v in b])


def mglma_subspace_build(ctx, g, block, nv, n_smooth, seed, store=MGLMA_FP32):
    h = _vp()
    _check(lib.mglma_subspace_build(_h(ctx), g, _block(block), int(nv), int(n_smooth), int(seed), int(store),
                                    C.byref(h)))
    return h.value


def mglma_subspace_create(ctx, g, block, nv, n_smooth, seed, store=MGLMA_FP32, n_cg=0, cg_prec=MGLMA_FP64,
                          lean_group=0):
    p = mglma_subspace_params(_block(block), int(nv), int(n_smooth), int(n_cg), int(cg_prec), int(seed), int(store),
                              int(lean_group))
    h = _vp()
    _check(lib.mglma_subspace_create(_h(ctx), g, C.byref(p), C.byref(h)))
    return h.value


def mglma_subspace_load(ctx, g, block, nv, vecs, store=MGLMA_FP32):
    h = _vp()
    _check(lib.mglma_subspace_load(_h(ctx), g, _block(block), int(nv), ptr(vecs), int(store), C.byref(h)))
    return h.value


def mglma_subspace_free(sub):
    lib.mglma_subspace_free(sub)


def mglma_subspace_info(sub):
    nv = C.c_int()
    Lb = (C.c_int * 4)()
    V1 = _i64()
    _check(lib.mglma_subspace_info(sub, C.byref(nv), Lb, C.byref(V1)))
    return nv.value, tuple(Lb), V1.value


def mglma_subspace_export(sub, phi):
    _check(lib.mglma_subspace_export(sub, ptr(phi)))


def mglma_restrict(ctx, sub, nrhs, inp, out, compute=MGLMA_FP64, stream=None):
    _check(lib.mglma_restrict(_h(ctx), sub, int(nrhs), ptr(inp), ptr(out), int(compute), _stream_ptr(stream)))


def mglma_prolong(ctx, sub, nrhs, inp, out, compute=MGLMA_FP64, stream=None):
    _check(lib.mglma_prolong(_h(ctx), sub, int(nrhs), ptr(inp), ptr(out), int(compute), _stream_ptr(stream)))


def mglma_coarse_build(ctx, g, sub, store=MGLMA_BF16):
    h = _vp()
    _check(lib.mglma_coarse_build(_h(ctx), g, sub, int(store), C.byref(h)))
    return h.value


def mglma_coarse_free(c):
    lib.mglma_coarse_free(c)


def mglma_coarse_info(c):
    nv = C.c_int()
    Lb = (C.c_int * 4)()
    V1 = _i64()
    _check(lib.mglma_coarse_info(c, C.byref(nv), Lb, C.byref(V1)))
    return nv.value, tuple(Lb), V1.value


def mglma_coarse_release_fp64(c):
    _check(lib.mglma_coarse_release_fp64(c))


def mglma_coarse_export(c, dhat):
    _check(lib.mglma_coarse_export(c, ptr(dhat)))


def mglma_coarse_apply(ctx, c, nrhs, inp, out, compute=MGLMA_FP64, stream=None, op=MGLMA_OP_D):
    _check(lib.mglma_coarse_apply(_h(ctx), c, int(op), int(nrhs), ptr(inp), ptr(out), int(compute),
                                  _stream_ptr(stream)))


def mglma_coarse_build_next(ctx, parent, block, store=MGLMA_BF16):
    """D_{l+1} = R_l D_l T_l on the grid of the parent's coarse sites blocked by `block`."""
    out = _vp()
    _check(lib.mglma_coarse_build_next(_h(ctx), parent, _block(block), int(store), C.byref(out)))
    return out.value


def mglma_coarse_restrict(ctx, level, nrhs, inp, out, stream=None):
    _check(lib.mglma_coarse_restrict(_h(ctx), level, int(nrhs), ptr(inp), ptr(out), _stream_ptr(stream)))


def mglma_coarse_prolong(ctx, level, nrhs, inp, out, stream=None):
    _check(lib.mglma_coarse_prolong(_h(ctx), level, int(nrhs), ptr(inp), ptr(out), _stream_ptr(stream)))


def mglma_pieces(ctx, g, levels, nrhs, b, psi, tol=1e-10, stream=None):
    """psi[l-1] = calT_l D_l^-1 calR_l b for the chain of coarse levels."""
    arr = (_vp * len(levels))(*levels)
    _check(lib.mglma_pieces(_h(ctx), g, arr, len(levels), int(nrhs), ptr(b), ptr(psi), float(tol),
                            _stream_ptr(stream)))


def mglma_coarse_gamma5_gamma(ctx, level, k, out):
    """Gam_k(x0) of the level, complex128 [L0][V_c][2nv][2nv]."""
    _check(lib.mglma_coarse_gamma5_gamma(_h(ctx), level, int(k), ptr(out)))


def mglma_coarse_dense_inverse(ctx, level, out):
    """Q_c^-1 of the level, complex128 [n][n]."""
    _check(lib.mglma_coarse_dense_inverse(_h(ctx), level, ptr(out)))


def mglma_exact_correlator(ctx, level, corr=None, G=None):
    """corr[x0][y0] and G[t] of the exact estimator on the level (complex128)."""
    _check(lib.mglma_exact_correlator(_h(ctx), level, ptr(corr), ptr(G)))


def mglma_solve_params_default(method=MGLMA_SOLVER_MG, **overrides):
    p = mglma_solve_params()
    lib.mglma_solve_params_default(C.byref(p), int(method))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def mglma_solve_batch(ctx, g, coarse, params, group_nrhs, b, x, x_coarse=None, stream=None, raise_on_error=True):
    """Returns (status, stats list of dicts)."""
    groups = [int(v) for v in group_nrhs]
    arr = (C.c_int * len(groups))(*groups)
    st = (mglma_solve_stats * max(1, sum(groups)))()
    status = lib.mglma_solve_batch(_h(ctx), g, coarse, C.byref(params), len(groups), arr, ptr(b), ptr(x),
                                   ptr(x_coarse), st, _stream_ptr(stream))
    if status != 0 and raise_on_error:
        _check(status)
    out = [dict(iterations=s.iterations, outer=s.outer, coarse_iterations=s.coarse_iterations,
                residual=s.residual, converged=bool(s.converged), batch=s.batch) for s in st[:sum(groups)]]
    return status, out


def mglma_sources(ctx, L, kind, nrhs, seed, out, first=0, point_sites=None, point_sc=None, t_slice=-1, stream=None):
    lat = mglma_lattice((C.c_int * 4)(*[int(v) for v in L]), -1)
    ps = (_i64 * nrhs)(*[int(v) for v in point_sites]) if point_sites is not None else None
    pc = (C.c_int * nrhs)(*[int(v) for v in point_sc]) if point_sc is not None else None
    _check(lib.mglma_sources(_h(ctx), C.byref(lat), int(kind), int(nrhs), int(seed), int(first), ps, pc,
                             int(t_slice), ptr(out), _stream_ptr(stream)))


def mglma_contract(ctx, L, nrhs, a, b, out, stream=None):
    """out[r][x0] = -(1/(3 L^3)) sum_k sum_{x in x0} <a[r][k-1](x), gamma5 gamma_k b[r](x)> (Eq. C_stoch2)."""
    lat = mglma_lattice((C.c_int * 4)(*[int(v) for v in L]), -1)
    _check(lib.mglma_contract(_h(ctx), C.byref(lat), int(nrhs), ptr(a), ptr(b), ptr(out), _stream_ptr(stream)))


def mglma_gamma5_gamma(ctx, L, k, nrhs, inp, out, stream=None):
    lat = mglma_lattice((C.c_int * 4)(*[int(v) for v in L]), -1)
    _check(lib.mglma_gamma5_gamma(_h(ctx), C.byref(lat), int(k), int(nrhs), ptr(inp), ptr(out), _stream_ptr(stream)))


def mglma_autotune(ctx, g=None, coarse=None, nrhs=1):
    _check(lib.mglma_autotune(_h(ctx), g, coarse, int(nrhs)))


def mglma_autotune_get(ctx, kernel, nrhs):
    c = C.c_int()
    ms = C.c_double()
    _check(lib.mglma_autotune_get(_h(ctx), int(kernel), int(nrhs), C.byref(c), C.byref(ms)))
    return c.value, ms.value


def mglma_autotune_set(ctx, kernel, nrhs, choice):
    _check(lib.mglma_autotune_set(_h(ctx), int(kernel), int(nrhs), int(choice)))


def dslash32_tile_code(nr, rw):
    """Tile code of the FP32 stencil: NR RHS per thread, RW RHS tiles per CTA."""
    return int(nr) + 16 * (int(rw) - 1)


def dslash32_staged_code(nrt):
    """Tile code of the FP32 staged-tile stencil: 32 sites x nrt (4, 8, 16) RHS per CTA."""
    return 64 + int(nrt)


def mglma_autotune_save(ctx, path):
    _check(lib.mglma_autotune_save(_h(ctx), str(path).encode()))


def mglma_autotune_load(ctx, path):
    _check(lib.mglma_autotune_load(_h(ctx), str(path).encode()))


class mglma_serve_lattice(C.Structure):
    _fields_ = [("gauge", _vp), ("coarse", _vp)]


class mglma_request(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nrhs", C.c_int), ("b", _vp), ("x", _vp), ("arrival", C.c_double),
                ("id", C.c_int64)]


class mglma_serve_config(C.Structure):
    _fields_ = [("nlattices", C.c_int), ("lattices", C.POINTER(mglma_serve_lattice)), ("max_slots", C.c_int),
                ("hbm_fraction", C.c_double), ("params", mglma_solve_params)]


class mglma_serve_stats(C.Structure):
    _fields_ = [("requests", C.c_longlong), ("rhs", C.c_longlong), ("rejected", C.c_longlong),
                ("wall_s", C.c_double), ("solves_per_s", C.c_double), ("p50_s", C.c_double),
                ("p99_s", C.c_double), ("mean_s", C.c_double), ("max_s", C.c_double), ("slots", C.c_int * 8),
                ("slot_bytes", C.c_double * 8)]


_REQ_FN = C.CFUNCTYPE(C.c_int, _vp, C.c_double, C.POINTER(mglma_request))
_DONE_FN = C.CFUNCTYPE(None, _vp, C.POINTER(mglma_request), C.c_int, C.c_double, C.POINTER(mglma_solve_stats))
_sig("mglma_serve", C.c_int, _vp, C.POINTER(mglma_serve_config), _REQ_FN, _DONE_FN, _vp,
     C.POINTER(mglma_serve_stats))


def mglma_serve(ctx, lattices, requests, params=None, max_slots=16, hbm_fraction=0.8):
    """Serves `requests` (dicts with lattice, b, x, arrival in seconds, sorted
    by arrival; b and x numpy arrays or device tensors).  The request
    callback hands each request to the server once the serving clock passes
    its arrival.  Returns (stats dict, per-request list of dicts with status,
    latency and per-RHS stats)."""
    lat = (mglma_serve_lattice * len(lattices))(*[mglma_serve_lattice(g, c) for g, c in lattices])
    cfg = mglma_serve_config(len(lattices), lat, int(max_slots), float(hbm_fraction),
                             params if params is not None else mglma_solve_params_default(MGLMA_SOLVER_MG))
    order = sorted(range(len(requests)), key=lambda i: requests[i]["arrival"])
    state = {"next": 0}
    results = [None] * len(requests)

    def next_fn(user, now, out):
        k = state["next"]
        if k >= len(order):
            return -1
        i = order[k]
        rq = requests[i]
        if rq["arrival"] > now:
            return 0
        nrhs = rq["b"].shape[0]
        out[0] = mglma_request(int(rq["lattice"]), int(nrhs), ptr(rq["b"]), ptr(rq["x"]), float(rq["arrival"]), i)
        state["next"] = k + 1
        return 1

    def done_fn(user, req, status, latency, per_rhs):
        r = req[0]
        results[r.id] = dict(status=status, latency=latency,
                             stats=[dict(iterations=per_rhs[j].iterations, outer=per_rhs[j].outer,
                                         residual=per_rhs[j].residual, converged=bool(per_rhs[j].converged))
                                    for j in range(r.nrhs)])

    cb_next, cb_done = _REQ_FN(next_fn), _DONE_FN(done_fn)
    st = mglma_serve_stats()
    _check(lib.mglma_serve(_h(ctx), C.byref(cfg), cb_next, cb_done, None, C.byref(st)))
    stats = dict(requests=st.requests, rhs=st.rhs, rejected=st.rejected, wall_s=st.wall_s,
                 solves_per_s=st.solves_per_s, p50_s=st.p50_s, p99_s=st.p99_s, mean_s=st.mean_s, max_s=st.max_s,
                 slots=list(st.slots[:len(lattices)]), slot_bytes=list(st.slot_bytes[:len(lattices)]))
    return stats, results
