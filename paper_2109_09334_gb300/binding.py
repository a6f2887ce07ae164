"""Thin ctypes binding of ``libsfft.so`` (include/sfft.h).

Argument marshalling only: every step of the subtraction runs in the CUDA
library.  Functions keep the C names; pointers may be given as integers or as
objects with ``data_ptr()`` (torch tensors), streams as integers or
``torch.cuda.Stream``.  A negative status raises :class:`SfftError`.
"""
from __future__ import annotations

import ctypes
import os
import re

from .build import LIB

SFFT_OK = 0
SFFT_ERR_INVALID = -1
SFFT_ERR_OOM = -2
SFFT_ERR_CUDA = -3
SFFT_ERR_SINGULAR = -4
SFFT_ERR_NOT_CONVERGED = -5
SFFT_ERR_TIMEOUT = -6
SFFT_ERR_BUSY = -7
SFFT_ERR_UNSUPPORTED = -8

SFFT_F32, SFFT_F64 = 0, 1
SFFT_STAGE_ROWS, SFFT_STAGE_COLS, SFFT_STAGE_GATHER, SFFT_STAGE_LAGS, SFFT_STAGE_SOLVE, SFFT_STAGE_SUBTRACT = range(6)
STAGE_NAMES = ["rows", "cols", "gather", "lags", "solve", "subtract"]
SFFT_PREC_FP64, SFFT_PREC_MIXED = 0, 1
SFFT_SOLVE_STATIC_MAX_N = 1024
SFFT_REQ_DEVICE, SFFT_REQ_HOST = 0, 1

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sfft.h")


class sfft_config(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in
                ("n0", "n1", "w0", "w1", "dk", "db", "const_phot_ratio", "dtype", "precision", "basis",
                 "kdeg", "kint", "bdeg", "bint")]


class sfft_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("min_pivot", ctypes.c_double)]


class sfft_request(ctypes.Structure):
    _fields_ = [("memory", ctypes.c_int32), ("ref", ctypes.c_void_p), ("sci", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("x", ctypes.c_void_p), ("info", ctypes.c_void_p),
                ("diff", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class sfft_ticket(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_uint64)]


class sfft_pool_ticket(ctypes.Structure):
    _fields_ = [("lane", ctypes.c_uint64), ("seq", ctypes.c_uint64)]


class SfftError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


_lib = None


def library():
    """Load libsfft.so; fails loudly if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libsfft.so not built ({LIB}); run paper_2109_09334_gb300.build.build()")
        lib = ctypes.CDLL(LIB)
        vp, i32, cfgp = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(sfft_config)
        lib.sfft_status_string.restype = ctypes.c_char_p
        lib.sfft_status_string.argtypes = [ctypes.c_int]
        lib.sfft_num_unknowns.argtypes = [cfgp, ctypes.POINTER(i32)]
        lib.sfft_plan_create.argtypes = [cfgp, vp, ctypes.POINTER(vp)]
        lib.sfft_plan_destroy.argtypes = [vp]
        lib.sfft_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.sfft_plan_set_solve_panel.argtypes = [vp, ctypes.c_int32]
        lib.sfft_plan_solve_panel.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
        lib.sfft_build_system.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.sfft_solve.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.sfft_solve_batch.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        lib.sfft_solve_static.argtypes = [vp, vp, i32, i32, vp, vp, vp]
        dbl = ctypes.c_double
        lib.sfft_decorrelate.argtypes = [vp, vp, dbl, dbl, dbl, dbl, vp, vp, vp]
        lib.sfft_subtract.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.sfft_run_pair.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.sfft_run_pair_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        lib.sfft_run_pairs.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
        lib.sfft_batch_create.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, i32, ctypes.POINTER(vp)]
        lib.sfft_batch_launch.argtypes = [vp, vp]
        lib.sfft_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
        lib.sfft_batch_destroy.argtypes = [vp]
        reqp, tkp = ctypes.POINTER(sfft_request), ctypes.POINTER(sfft_ticket)
        lib.sfft_server_create.argtypes = [cfgp, i32, i32, ctypes.POINTER(vp)]
        lib.sfft_flush.argtypes = [vp]
        lib.sfft_server_destroy.argtypes = [vp]
        lib.sfft_server_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.sfft_submit.argtypes = [vp, reqp, tkp]
        lib.sfft_poll.argtypes = [vp, tkp]
        lib.sfft_wait.argtypes = [vp, tkp, ctypes.c_int64]
        lib.sfft_stream_wait_ticket.argtypes = [vp, tkp, vp]
        lib.sfft_server_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.sfft_server_debug_fail_queries.argtypes = [vp, i32]
        lib.sfft_server_set_eager.argtypes = [vp, i32]
        lib.sfft_pool_set_eager.argtypes = [vp, i32]
        ptk = ctypes.POINTER(sfft_pool_ticket)
        lib.sfft_pool_create.argtypes = [ctypes.c_uint64, i32, i32, ctypes.POINTER(vp)]
        lib.sfft_pool_destroy.argtypes = [vp]
        lib.sfft_pool_submit.argtypes = [vp, cfgp, reqp, ptk]
        lib.sfft_pool_poll.argtypes = [vp, ptk]
        lib.sfft_pool_wait.argtypes = [vp, ptk, ctypes.c_int64]
        lib.sfft_pool_usage.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i32)]
        lib.sfft_plan_autotune.argtypes = [vp, vp, vp, vp, vp]
        dbl = ctypes.c_double
        lib.sfft_decorrelate_coadd.argtypes = [vp, vp, dbl, dbl, i32, vp, vp, i32, vp, vp, i32, i32, vp, vp, vp]
        lib.sfft_plan_tuning.argtypes = [vp, ctypes.POINTER(i32)]
        lib.sfft_saturation_mask.argtypes = [i32, i32, i32, vp, vp, dbl, dbl, i32, vp, vp, vp]
        lib.sfft_plan_set_tuning.argtypes = [vp, ctypes.POINTER(i32)]
        lib.sfft_plan_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.sfft_replay_stage.argtypes = [vp, ctypes.c_int, vp]
        _lib = lib
    return _lib


def declared_functions():
    """Names of the functions include/sfft.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sfft_\w+)\s*\(", text, re.M)))


def _p(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    if isinstance(x, ctypes.Structure):
        return ctypes.addressof(x)
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _s(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc, where):
    if rc != SFFT_OK:
        raise SfftError(rc, where)


def status_string(status):
    return library().sfft_status_string(status).decode()


SFFT_BASIS_POLY, SFFT_BASIS_BSPLINE = 0, 1


def make_config(n0, n1, w0, w1, dk, db, const_phot_ratio, dtype="float32", precision="mixed", spline=None):
    """spline: None (polynomial basis) or (kdeg, kint, bdeg, bint) for the B-spline basis (dk = db = 0)."""
    dt = {"float32": SFFT_F32, "f32": SFFT_F32, "float64": SFFT_F64, "f64": SFFT_F64}[str(dtype)]
    pr = {"fp64": SFFT_PREC_FP64, "mixed": SFFT_PREC_MIXED}[precision]
    if spline is None:
        return sfft_config(n0, n1, w0, w1, dk, db, int(bool(const_phot_ratio)), dt, pr, SFFT_BASIS_POLY, 0, 0, 0, 0)
    kdeg, kint, bdeg, bint = spline
    return sfft_config(n0, n1, w0, w1, dk, db, int(bool(const_phot_ratio)), dt, pr, SFFT_BASIS_BSPLINE,
                       kdeg, kint, bdeg, bint)


def sfft_num_unknowns(cfg):
    n = ctypes.c_int32()
    _check(library().sfft_num_unknowns(ctypes.byref(cfg), ctypes.byref(n)), "sfft_num_unknowns")
    return n.value


def sfft_plan_create(cfg, stream=None):
    h = ctypes.c_void_p()
    _check(library().sfft_plan_create(ctypes.byref(cfg), _s(stream), ctypes.byref(h)), "sfft_plan_create")
    return h.value


def sfft_plan_destroy(plan):
    _check(library().sfft_plan_destroy(plan), "sfft_plan_destroy")


def sfft_plan_set_solve_panel(plan, width):
    _check(library().sfft_plan_set_solve_panel(plan, int(width)), "sfft_plan_set_solve_panel")


def sfft_plan_solve_panel(plan):
    w = ctypes.c_int32()
    _check(library().sfft_plan_solve_panel(plan, ctypes.byref(w)), "sfft_plan_solve_panel")
    return w.value


def sfft_plan_workspace_bytes(plan):
    b = ctypes.c_uint64()
    _check(library().sfft_plan_workspace_bytes(plan, ctypes.byref(b)), "sfft_plan_workspace_bytes")
    return b.value


def sfft_build_system(plan, d_ref, d_sci, d_mask, d_M, d_rhs, stream=None):
    _check(library().sfft_build_system(plan, _p(d_ref), _p(d_sci), _p(d_mask), _p(d_M), _p(d_rhs), _s(stream)),
           "sfft_build_system")


def sfft_solve(plan, d_M, d_rhs, d_x, d_info=None, stream=None):
    _check(library().sfft_solve(plan, _p(d_M), _p(d_rhs), _p(d_x), _p(d_info), _s(stream)), "sfft_solve")


def sfft_solve_static(d_M, d_rhs, n, precision, d_x, d_info=None, stream=None):
    """Solve without a plan on the library's static workspace (n <= SFFT_SOLVE_STATIC_MAX_N)."""
    prec = {"fp64": SFFT_PREC_FP64, "mixed": SFFT_PREC_MIXED}.get(precision, precision)
    rc = library().sfft_solve_static(_p(d_M), _p(d_rhs), int(n), int(prec), _p(d_x), _p(d_info), _s(stream))
    if rc == SFFT_ERR_UNSUPPORTED and int(n) > SFFT_SOLVE_STATIC_MAX_N:
        raise SfftError(rc, f"sfft_solve_static: n={int(n)} exceeds SFFT_SOLVE_STATIC_MAX_N={SFFT_SOLVE_STATIC_MAX_N}")
    _check(rc, "sfft_solve_static")


def sfft_decorrelate(plan, d_x, xt0, yt0, sigma_ref, sigma_sci, d_diff, d_out, stream=None):
    _check(library().sfft_decorrelate(plan, _p(d_x), float(xt0), float(yt0), float(sigma_ref), float(sigma_sci),
                                      _p(d_diff), _p(d_out), _s(stream)), "sfft_decorrelate")


def sfft_decorrelate_coadd(plan, d_x, xt0, yt0, d_G, sigma_sci, d_H, sigma_ref, d_diff, d_out, stream=None):
    """d_G: [n_sci, 2g0+1, 2g1+1] and d_H: [n_ref, 2g0+1, 2g1+1] FP64 device tensors; sigma_*: sequences."""
    n_sci, n_ref = int(d_G.shape[0]), int(d_H.shape[0])
    g0, g1 = int(d_G.shape[1]) // 2, int(d_G.shape[2]) // 2
    if tuple(d_H.shape[1:]) != tuple(d_G.shape[1:]) or len(sigma_sci) != n_sci or len(sigma_ref) != n_ref:
        raise ValueError("sfft_decorrelate_coadd: kernel shapes and noise levels do not match")
    ss = (ctypes.c_double * n_sci)(*[float(v) for v in sigma_sci])
    sr = (ctypes.c_double * n_ref)(*[float(v) for v in sigma_ref])
    _check(library().sfft_decorrelate_coadd(plan, _p(d_x), float(xt0), float(yt0), n_sci, _p(d_G), ss, n_ref,
                                            _p(d_H), sr, g0, g1, _p(d_diff), _p(d_out), _s(stream)),
           "sfft_decorrelate_coadd")


def sfft_saturation_mask(d_ref, d_sci, sat_ref, sat_sci, grow, d_mask_out, d_mask_in=None, stream=None):
    """Crowded-flavor mask of a pair of 2-D float32/float64 CUDA tensors into a uint8 tensor."""
    n0, n1 = int(d_ref.shape[0]), int(d_ref.shape[1])
    dt = SFFT_F64 if d_ref.element_size() == 8 else SFFT_F32
    _check(library().sfft_saturation_mask(n0, n1, dt, _p(d_ref), _p(d_sci), float(sat_ref), float(sat_sci),
                                          int(grow), _p(d_mask_in), _p(d_mask_out), _s(stream)),
           "sfft_saturation_mask")


def sfft_subtract(plan, d_ref, d_sci, d_x, d_diff, stream=None):
    _check(library().sfft_subtract(plan, _p(d_ref), _p(d_sci), _p(d_x), _p(d_diff), _s(stream)), "sfft_subtract")


def sfft_run_pair(plan, d_ref, d_sci, d_mask, d_M, d_rhs, d_x, d_info, d_diff, stream=None):
    _check(library().sfft_run_pair(plan, _p(d_ref), _p(d_sci), _p(d_mask), _p(d_M), _p(d_rhs), _p(d_x),
                                   _p(d_info), _p(d_diff), _s(stream)), "sfft_run_pair")


def _ptr_array(items):
    """A C array of the items' addresses, or NULL when items is None."""
    if items is None:
        return None
    return (ctypes.c_void_p * len(items))(*[_p(v) for v in items])


def sfft_run_pairs(plans, d_refs, d_scis, d_masks, d_xs, d_infos, d_diffs, stream=None):
    """Several pairs, each with its own plan; d_masks, d_xs, d_infos may be None or hold None."""
    n = len(plans)
    for name, v in (("d_refs", d_refs), ("d_scis", d_scis), ("d_diffs", d_diffs), ("d_masks", d_masks),
                    ("d_xs", d_xs), ("d_infos", d_infos)):
        if v is not None and len(v) != n:
            raise ValueError(f"sfft_run_pairs: {name} has {len(v)} entries for {n} plans")
    hp = (ctypes.c_void_p * n)(*plans)
    _check(library().sfft_run_pairs(hp, n, _ptr_array(d_refs), _ptr_array(d_scis), _ptr_array(d_masks),
                                    _ptr_array(d_xs), _ptr_array(d_infos), _ptr_array(d_diffs), _s(stream)),
           "sfft_run_pairs")


def sfft_solve_batch(plans, d_Ms, d_rhss, d_xs, d_infos=None, stream=None):
    """Several built systems solved in one launch, system i on plans[i]."""
    n = len(plans)
    for name, v in (("d_Ms", d_Ms), ("d_rhss", d_rhss), ("d_xs", d_xs), ("d_infos", d_infos)):
        if v is not None and len(v) != n:
            raise ValueError(f"sfft_solve_batch: {name} has {len(v)} entries for {n} plans")
    hp = (ctypes.c_void_p * n)(*plans)
    _check(library().sfft_solve_batch(hp, n, _ptr_array(d_Ms), _ptr_array(d_rhss), _ptr_array(d_xs),
                                      _ptr_array(d_infos), _s(stream)), "sfft_solve_batch")


def sfft_batch_create(plans, d_refs, d_scis, d_masks, d_xs, d_infos, d_diffs, solve_group=0):
    """Capture the pairs of sfft_run_pairs into a CUDA graph; returns the batch handle."""
    n = len(plans)
    for name, v in (("d_refs", d_refs), ("d_scis", d_scis), ("d_diffs", d_diffs), ("d_masks", d_masks),
                    ("d_xs", d_xs), ("d_infos", d_infos)):
        if v is not None and len(v) != n:
            raise ValueError(f"sfft_batch_create: {name} has {len(v)} entries for {n} plans")
    hp = (ctypes.c_void_p * n)(*plans)
    h = ctypes.c_void_p()
    _check(library().sfft_batch_create(hp, n, _ptr_array(d_refs), _ptr_array(d_scis), _ptr_array(d_masks),
                                       _ptr_array(d_xs), _ptr_array(d_infos), _ptr_array(d_diffs),
                                       int(solve_group), ctypes.byref(h)), "sfft_batch_create")
    return h.value


def sfft_batch_launch(batch, stream=None):
    _check(library().sfft_batch_launch(batch, _s(stream)), "sfft_batch_launch")


def sfft_batch_info(batch):
    g, nl = ctypes.c_int32(), ctypes.c_int32()
    t = (ctypes.c_float * 4)()
    _check(library().sfft_batch_info(batch, ctypes.byref(g), ctypes.byref(nl), t), "sfft_batch_info")
    return {"solve_group": g.value, "launches": nl.value, "tune_ms": {k: t[i] for i, k in enumerate((8, 4, 2, 1))}}


def sfft_batch_destroy(batch):
    _check(library().sfft_batch_destroy(batch), "sfft_batch_destroy")


def sfft_run_pair_host(plan, h_ref, h_sci, h_mask, h_x, h_info, h_diff, stream=None):
    _check(library().sfft_run_pair_host(plan, _p(h_ref), _p(h_sci), _p(h_mask), _p(h_x), _p(h_info),
                                        _p(h_diff), _s(stream)), "sfft_run_pair_host")


def sfft_server_create(cfg, depth=2, batch=1):
    h = ctypes.c_void_p()
    _check(library().sfft_server_create(ctypes.byref(cfg), int(depth), int(batch), ctypes.byref(h)),
           "sfft_server_create")
    return h.value


def sfft_flush(server):
    _check(library().sfft_flush(server), "sfft_flush")


def sfft_server_destroy(server):
    _check(library().sfft_server_destroy(server), "sfft_server_destroy")


def sfft_server_workspace_bytes(server):
    b = ctypes.c_uint64()
    _check(library().sfft_server_workspace_bytes(server, ctypes.byref(b)), "sfft_server_workspace_bytes")
    return b.value


def make_request(ref, sci, diff, mask=None, x=None, info=None, stream=None, host=False):
    return sfft_request(SFFT_REQ_HOST if host else SFFT_REQ_DEVICE, _p(ref), _p(sci), _p(mask), _p(x), _p(info),
                        _p(diff), None if host else _s(stream))


def sfft_submit(server, req):
    t = sfft_ticket()
    _check(library().sfft_submit(server, ctypes.byref(req), ctypes.byref(t)), "sfft_submit")
    return t


def sfft_poll(server, ticket):
    """True if the ticket's request has completed."""
    rc = library().sfft_poll(server, ctypes.byref(ticket))
    if rc == SFFT_ERR_BUSY:
        return False
    _check(rc, "sfft_poll")
    return True


def sfft_wait(server, ticket, timeout_us=-1):
    """True once completed; False on timeout."""
    rc = library().sfft_wait(server, ctypes.byref(ticket), int(timeout_us))
    if rc == SFFT_ERR_TIMEOUT:
        return False
    _check(rc, "sfft_wait")
    return True


def sfft_stream_wait_ticket(server, ticket, stream=None):
    _check(library().sfft_stream_wait_ticket(server, ctypes.byref(ticket), _s(stream)), "sfft_stream_wait_ticket")


def sfft_server_launch_count(server):
    c = ctypes.c_uint64()
    _check(library().sfft_server_launch_count(server, ctypes.byref(c)), "sfft_server_launch_count")
    return c.value


def sfft_server_debug_fail_queries(server, enable):
    """Testing hook: make the server's completion queries report a CUDA error."""
    _check(library().sfft_server_debug_fail_queries(server, int(bool(enable))), "sfft_server_debug_fail_queries")


def sfft_server_set_eager(server, enable):
    _check(library().sfft_server_set_eager(server, int(bool(enable))), "sfft_server_set_eager")


def sfft_pool_set_eager(pool, enable):
    _check(library().sfft_pool_set_eager(pool, int(bool(enable))), "sfft_pool_set_eager")


def sfft_pool_create(budget_bytes, depth=2, batch=1):
    h = ctypes.c_void_p()
    _check(library().sfft_pool_create(int(budget_bytes), int(depth), int(batch), ctypes.byref(h)), "sfft_pool_create")
    return h.value


def sfft_pool_destroy(pool):
    _check(library().sfft_pool_destroy(pool), "sfft_pool_destroy")


def sfft_pool_submit(pool, cfg, req):
    """Ticket, or None if the configuration cannot be admitted now (SFFT_ERR_BUSY)."""
    t = sfft_pool_ticket()
    rc = library().sfft_pool_submit(pool, ctypes.byref(cfg), ctypes.byref(req), ctypes.byref(t))
    if rc == SFFT_ERR_BUSY:
        return None
    _check(rc, "sfft_pool_submit")
    return t


def sfft_pool_poll(pool, ticket):
    rc = library().sfft_pool_poll(pool, ctypes.byref(ticket))
    if rc == SFFT_ERR_BUSY:
        return False
    _check(rc, "sfft_pool_poll")
    return True


def sfft_pool_wait(pool, ticket, timeout_us=-1):
    rc = library().sfft_pool_wait(pool, ctypes.byref(ticket), int(timeout_us))
    if rc == SFFT_ERR_TIMEOUT:
        return False
    _check(rc, "sfft_pool_wait")
    return True


def sfft_pool_usage(pool):
    b, n = ctypes.c_uint64(), ctypes.c_int32()
    _check(library().sfft_pool_usage(pool, ctypes.byref(b), ctypes.byref(n)), "sfft_pool_usage")
    return b.value, n.value


def sfft_plan_autotune(plan, d_ref, d_sci, d_diff, stream=None):
    _check(library().sfft_plan_autotune(plan, _p(d_ref), _p(d_sci), _p(d_diff), _s(stream)), "sfft_plan_autotune")


SFFT_TUNING_LEN = 5
TUNING_KEYS = ("rows_per_block", "images_per_block", "row_pairs_per_block", "solve_grid", "solve_tensor_cores")


def sfft_plan_tuning(plan):
    out = (ctypes.c_int32 * SFFT_TUNING_LEN)()
    _check(library().sfft_plan_tuning(plan, out), "sfft_plan_tuning")
    return dict(zip(TUNING_KEYS, list(out)))


def sfft_plan_set_tuning(plan, shapes):
    """shapes: a dict with TUNING_KEYS (missing keys: 0) or SFFT_TUNING_LEN integers."""
    if isinstance(shapes, dict):
        shapes = [int(shapes.get(k, 0)) for k in TUNING_KEYS]
    if len(shapes) != SFFT_TUNING_LEN:
        raise ValueError(f"sfft_plan_set_tuning: {SFFT_TUNING_LEN} values expected")
    _check(library().sfft_plan_set_tuning(plan, (ctypes.c_int32 * SFFT_TUNING_LEN)(*shapes)),
           "sfft_plan_set_tuning")


def sfft_plan_launch_count(plan):
    c = ctypes.c_uint64()
    _check(library().sfft_plan_launch_count(plan, ctypes.byref(c)), "sfft_plan_launch_count")
    return c.value


def sfft_replay_stage(plan, stage, stream=None):
    _check(library().sfft_replay_stage(plan, int(stage), _s(stream)), "sfft_replay_stage")
