"""ctypes binding of ``librsfd.so`` (argument marshalling only).

Host inputs are numpy arrays; device buffers are torch CUDA tensors whose
``data_ptr()`` is passed through.  Matrices follow the C ABI's column-major
convention per energy: a torch tensor ``G`` of shape ``(K, ncols, nb)`` holds
column ``c`` of energy ``k`` in ``G[k, c, :]`` (so ``G[k].T`` is the matrix).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

RSFD_OK = 0
RSFD_ERR_ARG = 1
RSFD_ERR_ALLOC = 2
RSFD_ERR_CUDA = 3
RSFD_ERR_NOT_CONVERGED = 4
RSFD_ERR_BREAKDOWN = 5
RSFD_ERR_TIMEOUT = 6
RSFD_ERR_UNSUPPORTED = 7
RSFD_FP64 = 0
RSFD_MIXED = 1
RSFD_DF64 = 2
RSFD_SEED_MID = 0
RSFD_SEED_FIRST = 1
RSFD_SEED_INDEX = 2
RSFD_SEED_AUX = 3
RSFD_PASS_AUTO = 0
RSFD_PASS_RECOMPUTE = 1
RSFD_PASS_STORED = 2
RSFD_PASS_SPLIT = 3
RSFD_PASS_SPLIT_BFP = 4
RSFD_DYSON_AUTO = 0
RSFD_DYSON_FP64 = 1
RSFD_DYSON_TC = 2

_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_ALLOC", 3: "ERR_CUDA", 4: "ERR_NOT_CONVERGED", 5: "ERR_BREAKDOWN",
           6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}


class RsfdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class rsfd_projectors(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("ptr", ctypes.POINTER(ctypes.c_int64)),
                ("idx", ctypes.POINTER(ctypes.c_int64)), ("val", ctypes.POINTER(ctypes.c_double)),
                ("E", ctypes.POINTER(ctypes.c_double))]


class rsfd_col_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("switches", ctypes.c_int32), ("status", ctypes.c_int32),
                ("final_seed", ctypes.c_int32)]


class rsfd_solve_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("iters_per_sync", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("z_chunk", ctypes.c_int32), ("use_graphs", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("pass_kind", ctypes.c_int32), ("prefetch", ctypes.c_int32), ("rows_per_thread", ctypes.c_int32),
                ("dyson_kind", ctypes.c_int32), ("dyson_refine", ctypes.c_int32), ("reg_budget", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("wait_cap", ctypes.c_int32), ("dyson_cols", ctypes.c_int32),
                ("breakdown_tol", ctypes.c_double)]


class rsfd_region_solve(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("cols", ctypes.POINTER(ctypes.c_int64)), ("ncols", ctypes.c_int32),
                ("energies", ctypes.POINTER(ctypes.c_double)), ("K", ctypes.c_int32), ("eta", ctypes.c_double),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("seed_kind", ctypes.c_int32),
                ("seed_index", ctypes.c_int32), ("G0_bb", ctypes.c_void_p),
                ("info", ctypes.POINTER(rsfd_col_info)), ("final_res", ctypes.POINTER(ctypes.c_double)),
                ("status", ctypes.c_int)]


class rsfd_stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_pass", ctypes.c_double), ("ms_shift", ctypes.c_double),
                ("n_pass", ctypes.c_int64), ("n_shift", ctypes.c_int64), ("n_other", ctypes.c_int64),
                ("slot_iterations", ctypes.c_int64), ("shift_updates", ctypes.c_int64),
                ("shift_slot_chunks", ctypes.c_int64),
                ("slots", ctypes.c_int32), ("iters_per_sync", ctypes.c_int32), ("ms_combine", ctypes.c_double)]


# every symbol declared in include/rsfd.h, with (restype, argtypes)
_P = ctypes.c_void_p
_SIGNATURES = {
    "rsfd_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int32), ctypes.c_double,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(rsfd_projectors), ctypes.c_int32, _P]),
    "rsfd_boundary_rows": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    "rsfd_set_tracked_planes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "rsfd_tracked_rows": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    "rsfd_set_solve_options": (ctypes.c_int, [_P, ctypes.POINTER(rsfd_solve_opts)]),
    "rsfd_shifted_cocg": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                         ctypes.POINTER(rsfd_col_info), ctypes.POINTER(ctypes.c_double)]),
    "rsfd_shifted_cocg_aux": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                             ctypes.POINTER(rsfd_col_info), ctypes.POINTER(ctypes.c_double)]),
    "rsfd_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(rsfd_stats)]),
    "rsfd_lead_sigma_decimation": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                                  ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "rsfd_shifted_cocg_sweep": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_char_p, _P, ctypes.POINTER(rsfd_col_info),
                                               ctypes.POINTER(ctypes.c_int32)]),
    "rsfd_sweep_load_energies": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32, _P]),
    "rsfd_shifted_cocg_regions": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(rsfd_region_solve)]),
    "rsfd_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(rsfd_solve_opts),
                                     ctypes.POINTER(ctypes.c_double)]),
    "rsfd_dyson_boundary": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_double)]),
    "rsfd_dyson_tracked": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_double)]),
    "rsfd_cgemm_tf32x3": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_double), _P, ctypes.c_int32, ctypes.c_int64, _P,
                                         ctypes.c_int32, ctypes.c_int64, ctypes.c_double, _P, ctypes.c_int32,
                                         ctypes.c_int64, _P]),
    "rsfd_transmission": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "rsfd_lead_sigma_uniform": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "rsfd_dyson_boundary_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                                                   ctypes.POINTER(ctypes.c_double), _P]),
    "rsfd_last_error": (ctypes.c_char_p, [_P]),
    "rsfd_destroy": (None, [_P]),
}

_LIB = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "librsfd.so")


def load_library():
    """Load librsfd.so (raises if it has not been built; there is no fallback)."""
    global _LIB
    if _LIB is None:
        p = lib_path()
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with paper_1502_00081_gb300.build_lib.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return ctypes.c_void_p(int(stream))


def _check(h, status, allow=()):
    if status != RSFD_OK and status not in allow:
        raise RsfdError(status, rsfd_last_error(h))
    return status


def _dev_ptr(t, dtypes, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def rsfd_last_error(h=None) -> str:
    return load_library().rsfd_last_error(h).decode()


def rsfd_create(grid, h, fd_order, V_loc, n_face=0, proj=None, precision=RSFD_FP64, stream=None):
    lib = load_library()
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    V, Vp = _f64(np.asarray(V_loc).ravel())
    keep = []
    pp = None
    if proj is not None:
        ptr, ptrp = _i64(proj.ptr)
        idx, idxp = _i64(proj.idx)
        val, valp = _f64(proj.val)
        E, Ep = _f64(proj.E)
        keep += [ptr, idx, val, E]
        pp = ctypes.byref(rsfd_projectors(int(proj.n_atoms), ptrp, idxp, valp, Ep))
    out = ctypes.c_void_p()
    st = lib.rsfd_create(ctypes.byref(out), g, float(h), int(fd_order), int(n_face), Vp, pp, int(precision),
                         _stream_ptr(stream))
    _check(None, st)
    return out


def rsfd_set_tracked_planes(h, planes):
    lib = load_library()
    z = np.ascontiguousarray(np.asarray(planes, dtype=np.int32).ravel())
    _check(h, lib.rsfd_set_tracked_planes(h, int(z.size), z.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
                                          if z.size else None))


def rsfd_tracked_rows(h):
    lib = load_library()
    nr = ctypes.c_int32()
    _check(h, lib.rsfd_tracked_rows(h, ctypes.byref(nr), None))
    rows = np.zeros(nr.value, np.int64)
    _check(h, lib.rsfd_tracked_rows(h, ctypes.byref(nr), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return rows


def rsfd_dyson_tracked(h, G0, Sigma_L, Sigma_R, G):
    """Dyson step on the recorded rows (G0, G: [K][nr][nr] column-major); returns refinement residuals."""
    import torch
    lib = load_library()
    K = int(G0.shape[0])
    p0 = _dev_ptr(G0, (torch.complex64, torch.complex128), name="G0")
    pl = _dev_ptr(Sigma_L, (torch.complex128,), name="Sigma_L")
    pr = _dev_ptr(Sigma_R, (torch.complex128,), name="Sigma_R")
    pg = _dev_ptr(G, (G0.dtype,), tuple(G0.shape), name="G")
    ref = np.zeros(K, np.float64)
    _check(h, lib.rsfd_dyson_tracked(h, p0, pl, pr, K, pg, ref.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return ref


def rsfd_boundary_rows(h):
    lib = load_library()
    nb = ctypes.c_int32()
    _check(h, lib.rsfd_boundary_rows(h, ctypes.byref(nb), None))
    rows = np.zeros(nb.value, np.int64)
    _check(h, lib.rsfd_boundary_rows(h, ctypes.byref(nb), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return rows


def rsfd_set_solve_options(h, slots=0, iters_per_sync=0, tile_y=0, z_chunk=0, use_graphs=0, profile=0,
                           pass_kind=0, prefetch=0, rows_per_thread=0, dyson_kind=0, dyson_refine=0, reg_budget=0,
                           tile_x=0, wait_cap=0, dyson_cols=0, breakdown_tol=0.0):
    lib = load_library()
    o = rsfd_solve_opts(int(slots), int(iters_per_sync), int(tile_y), int(z_chunk), int(use_graphs), int(profile),
                        int(pass_kind), int(prefetch), int(rows_per_thread), int(dyson_kind), int(dyson_refine),
                        int(reg_budget), int(tile_x), int(wait_cap), int(dyson_cols), float(breakdown_tol))
    _check(h, lib.rsfd_set_solve_options(h, ctypes.byref(o)))


def rsfd_shifted_cocg(h, cols, energies, eta, tol, maxit, G0_bb, seed_kind=RSFD_SEED_MID, seed_index=0,
                      aux_energies=None):
    """Returns (status, info [ncols] structured array, final_res [ncols, K]).  With aux_energies the
    call goes to rsfd_shifted_cocg_aux (seed candidates outside the set)."""
    import torch
    lib = load_library()
    c, cp = _i64(cols)
    e, ep = _f64(energies)
    ptr = _dev_ptr(G0_bb, (torch.complex64, torch.complex128), name="G0_bb")
    info = (rsfd_col_info * c.size)()
    res = np.zeros((c.size, e.size), np.float64)
    if aux_energies is None:
        st = lib.rsfd_shifted_cocg(h, cp, int(c.size), ep, int(e.size), float(eta), float(tol), int(maxit),
                                   int(seed_kind), int(seed_index), ptr, info,
                                   res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    else:
        a, apt = _f64(aux_energies)
        st = lib.rsfd_shifted_cocg_aux(h, cp, int(c.size), ep, int(e.size), apt, int(a.size), float(eta), float(tol),
                                       int(maxit), int(seed_kind), int(seed_index), ptr, info,
                                       res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(h, st, allow=(RSFD_ERR_NOT_CONVERGED, RSFD_ERR_BREAKDOWN))
    arr = np.array([(i.iters, i.switches, i.status, i.final_seed) for i in info],
                   dtype=[("iters", np.int32), ("switches", np.int32), ("status", np.int32),
                          ("final_seed", np.int32)])
    return st, arr, res


def rsfd_lead_sigma_decimation(h, energies, eta, V_left=None, V_right=None, maxit=200, ns=None):
    """Lead self-energies by decimation on the GPU; returns (Sigma_L, Sigma_R) as complex128 CUDA
    tensors [K, ns, ns] and the number of decimation steps used."""
    import torch
    lib = load_library()
    e, ep = _f64(energies)
    if ns is None:
        ns = int(rsfd_boundary_rows(h).size) // 2
    SL = torch.empty((e.size, ns, ns), dtype=torch.complex128, device="cuda")
    SR = torch.empty_like(SL)
    keep = []
    ptrs = []
    for V in (V_left, V_right):
        if V is None:
            ptrs.append(None)
        else:
            v, vp = _f64(np.asarray(V, dtype=np.float64).ravel())
            keep.append(v)
            ptrs.append(vp)
    it = ctypes.c_int32(0)
    _check(h, lib.rsfd_lead_sigma_decimation(h, ptrs[0], ptrs[1], ep, int(e.size), float(eta), int(maxit),
                                             SL.data_ptr(), SR.data_ptr(), ctypes.byref(it)))
    return SL, SR, int(it.value)


def rsfd_shifted_cocg_sweep(h, cols, energies, eta, tol, maxit, G0_bb, block, directory, seed_kind=RSFD_SEED_MID,
                            seed_index=0):
    """Checkpointed column sweep; returns (status, info structured array, blocks resumed from files)."""
    import torch
    lib = load_library()
    c, cp = _i64(cols)
    e, ep = _f64(energies)
    ptr = None if G0_bb is None else _dev_ptr(G0_bb, (torch.complex64, torch.complex128), name="G0_bb")
    info = (rsfd_col_info * c.size)()
    resumed = ctypes.c_int32(0)
    st = lib.rsfd_shifted_cocg_sweep(h, cp, int(c.size), ep, int(e.size), float(eta), float(tol), int(maxit),
                                     int(seed_kind), int(seed_index), int(block), str(directory).encode(), ptr, info,
                                     ctypes.byref(resumed))
    _check(h, st, allow=(RSFD_ERR_NOT_CONVERGED, RSFD_ERR_BREAKDOWN))
    arr = np.array([(i.iters, i.switches, i.status, i.final_seed) for i in info],
                   dtype=[("iters", np.int32), ("switches", np.int32), ("status", np.int32),
                          ("final_seed", np.int32)])
    return st, arr, int(resumed.value)


def rsfd_sweep_load_energies(h, cols, energies, eta, tol, maxit, block, directory, k0, kcount, G0_part,
                             seed_kind=RSFD_SEED_MID, seed_index=0):
    """Energies k0 .. k0+kcount-1 of a completed checkpointed sweep into G0_part [kcount, ncols, nb]."""
    import torch
    lib = load_library()
    c, cp = _i64(cols)
    e, ep = _f64(energies)
    ptr = _dev_ptr(G0_part, (torch.complex64, torch.complex128), name="G0_part")
    _check(h, lib.rsfd_sweep_load_energies(h, cp, int(c.size), ep, int(e.size), float(eta), float(tol), int(maxit),
                                           int(seed_kind), int(seed_index), int(block), str(directory).encode(),
                                           int(k0), int(kcount), ptr))


def rsfd_shifted_cocg_regions(jobs):
    """Several regions in one call.  jobs: list of dicts with keys h (handle pointer), cols, energies,
    eta, tol, maxit, G0_bb (device tensor) and optionally seed_kind, seed_index.  Returns
    (worst status, [(status, info, final_res) per job])."""
    import torch
    lib = load_library()
    n = len(jobs)
    arr = (rsfd_region_solve * n)()
    keep = []
    for i, j in enumerate(jobs):
        c, cp = _i64(j["cols"])
        e, ep = _f64(j["energies"])
        info = (rsfd_col_info * c.size)()
        res = np.zeros((c.size, e.size), np.float64)
        ptr = _dev_ptr(j["G0_bb"], (torch.complex64, torch.complex128), name="G0_bb")
        keep.append((c, e, info, res))
        arr[i] = rsfd_region_solve(j["h"], cp, int(c.size), ep, int(e.size), float(j["eta"]), float(j["tol"]),
                                   int(j["maxit"]), int(j.get("seed_kind", RSFD_SEED_MID)), int(j.get("seed_index", 0)),
                                   ptr, info, res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    st = lib.rsfd_shifted_cocg_regions(n, arr)
    _check(None, st, allow=(RSFD_ERR_NOT_CONVERGED, RSFD_ERR_BREAKDOWN))
    out = []
    for i, (c, e, info, res) in enumerate(keep):
        inf = np.array([(x.iters, x.switches, x.status, x.final_seed) for x in info],
                       dtype=[("iters", np.int32), ("switches", np.int32), ("status", np.int32),
                              ("final_seed", np.int32)])
        out.append((int(arr[i].status), inf, res))
    return st, out


def rsfd_autotune(h, energies, eta, slots, iters=128):
    """Tune the handle's launch options on short solves; returns (options dict, us per slot-iteration)."""
    lib = load_library()
    e, ep = _f64(energies)
    o = rsfd_solve_opts()
    us = ctypes.c_double(0.0)
    _check(h, lib.rsfd_autotune(h, ep, int(e.size), float(eta), int(slots), int(iters), ctypes.byref(o),
                                ctypes.byref(us)))
    return {k: getattr(o, k) for k, _ in rsfd_solve_opts._fields_}, float(us.value)


def rsfd_get_stats(h) -> dict:
    lib = load_library()
    s = rsfd_stats()
    _check(h, lib.rsfd_get_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in rsfd_stats._fields_}


def rsfd_dyson_boundary(h, G0_bb, Sigma_L, Sigma_R, G_bb):
    import torch
    lib = load_library()
    K = int(G0_bb.shape[0])
    p0 = _dev_ptr(G0_bb, (torch.complex64, torch.complex128), name="G0_bb")
    pl = _dev_ptr(Sigma_L, (torch.complex128,), name="Sigma_L")
    pr = _dev_ptr(Sigma_R, (torch.complex128,), name="Sigma_R")
    pg = _dev_ptr(G_bb, (G0_bb.dtype,), tuple(G0_bb.shape), name="G_bb")
    ref = np.zeros(K, np.float64)
    _check(h, lib.rsfd_dyson_boundary(h, p0, pl, pr, K, pg, ref.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return ref


def rsfd_cgemm_tf32x3(A, B, C, alpha=1.0, beta=0.0, stream=None):
    """C[b] = alpha A[b] B[b] + beta C[b] on the tensor cores (3xTF32).  A, B, C: complex64 CUDA tensors of
    shape [batch, cols, rows] holding column-major matrices (rows fastest); C is written in place."""
    import torch
    lib = load_library()
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        if t.dtype != torch.complex64 or not t.is_cuda or t.dim() != 3 or not t.is_contiguous():
            raise RsfdError(RSFD_ERR_ARG, f"{nm}: contiguous complex64 CUDA tensor [batch, cols, rows] expected")
    batch, k, m = A.shape
    n = B.shape[1]
    if B.shape[0] != batch or B.shape[2] != k or tuple(C.shape) != (batch, n, m):
        raise RsfdError(RSFD_ERR_ARG, "shape mismatch")
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.rsfd_cgemm_tf32x3(int(batch), int(m), int(n), int(k), al, A.data_ptr(), int(m), int(m * k),
                               B.data_ptr(), int(k), int(k * n), float(beta), C.data_ptr(), int(m), int(m * n),
                               ctypes.c_void_p(stream))
    _check(None, st)


def rsfd_dyson_boundary_noalloc(G0_bb, Sigma_L, Sigma_R, G_bb, stream=None):
    """Allocation-free Dyson step (c128 data, no handle); returns the refinement residuals."""
    import torch
    lib = load_library()
    K, nb = int(G0_bb.shape[0]), int(G0_bb.shape[-1])
    p0 = _dev_ptr(G0_bb, (torch.complex128,), name="G0_bb")
    pl = _dev_ptr(Sigma_L, (torch.complex128,), name="Sigma_L")
    pr = _dev_ptr(Sigma_R, (torch.complex128,), name="Sigma_R")
    pg = _dev_ptr(G_bb, (torch.complex128,), tuple(G0_bb.shape), name="G_bb")
    ref = np.zeros(K, np.float64)
    st = lib.rsfd_dyson_boundary_noalloc(nb, K, p0, pl, pr, pg, ref.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         _stream_ptr(stream))
    _check(None, st)
    return ref


def rsfd_transmission(h, G_bb, Sigma_L, Sigma_R):
    import torch
    lib = load_library()
    K = int(G_bb.shape[0])
    pg = _dev_ptr(G_bb, (torch.complex64, torch.complex128), name="G_bb")
    pl = _dev_ptr(Sigma_L, (torch.complex128,), name="Sigma_L")
    pr = _dev_ptr(Sigma_R, (torch.complex128,), name="Sigma_R")
    T = np.zeros(K, np.float64)
    _check(h, lib.rsfd_transmission(h, pg, pl, pr, K, T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return T


def rsfd_lead_sigma_uniform(Nx, Ny, h, fd_order, energies, eta):
    """Host helper: returns (Sigma_L, Sigma_R) as complex128 arrays [K][ns][ns] in the ABI's
    column-major layout (element (k, a, c) at [k, c, a]); Sigma is complex symmetric."""
    lib = load_library()
    e, ep = _f64(energies)
    ns = (fd_order // 2) * Nx * Ny
    SL = np.zeros((e.size, ns, ns), np.complex128)
    SR = np.zeros((e.size, ns, ns), np.complex128)
    st = lib.rsfd_lead_sigma_uniform(int(Nx), int(Ny), float(h), int(fd_order), ep, float(eta), int(e.size),
                                     SL.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     SR.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(None, st)
    return SL, SR


def rsfd_destroy(h):
    if h is not None and h.value:
        load_library().rsfd_destroy(h)


class Handle:
    """Owns one rsfd handle; ``with Handle(...) as h:`` destroys it on exit."""

    def __init__(self, grid, h, fd_order, V_loc, n_face=0, proj=None, precision=RSFD_FP64, stream=None):
        self.grid, self.h, self.fd_order = tuple(grid), float(h), int(fd_order)
        self.precision = precision
        self.ptr = rsfd_create(grid, h, fd_order, V_loc, n_face, proj, precision, stream)
        self.rows = rsfd_boundary_rows(self.ptr)
        self.nb = int(self.rows.size)

    @property
    def complex_dtype(self):
        import torch
        return torch.complex64 if self.precision == RSFD_MIXED else torch.complex128

    def close(self):
        rsfd_destroy(self.ptr)
        self.ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
