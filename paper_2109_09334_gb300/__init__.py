"""GB300 (sm_103a) implementation of the SFFT hot path (arXiv:2109.09334).

Image subtraction in Fourier space: the delta-function-basis least-squares
system (Eq. 18-24, App. B) is built from FFTs of the monomial-weighted
images, spectrum products and a pruned inverse DFT; it is solved by a
Jacobi-scaled Cholesky with FP64 refinement; and the difference image
(Eq. 12-13) is formed in Fourier space.  All arithmetic runs in the CUDA
library ``libsfft.so`` behind the C ABI of ``include/sfft.h``; this package is
its ctypes binding plus a small convenience wrapper over torch tensors (torch
only provides device memory and streams).
"""
from __future__ import annotations

import atexit
import ctypes
import weakref

from . import binding
from .binding import make_request  # noqa: F401
from .binding import (  # noqa: F401
    SfftError,
    make_config,
    sfft_build_system,
    sfft_num_unknowns,
    sfft_plan_create,
    sfft_plan_destroy,
    sfft_plan_workspace_bytes,
    sfft_run_pair,
    sfft_run_pair_host,
    sfft_run_pairs,
    sfft_server_create,
    sfft_server_destroy,
    sfft_server_workspace_bytes,
    sfft_poll,
    sfft_solve,
    sfft_solve_static,
    sfft_stream_wait_ticket,
    sfft_submit,
    sfft_wait,
    sfft_solve_info,
    sfft_subtract,
    status_string,
)


def _torch():
    import torch
    return torch


_live = weakref.WeakSet()  # objects that hold library handles
_registered = False


def _close_all():
    """Release the handles still open (batches, servers and pools before
    plans) while torch and the CUDA runtime are still up."""
    for o in sorted(list(_live), key=lambda o: isinstance(o, SfftPlan)):
        try:
            o.close()
        except Exception:
            pass


def _track(obj):
    # registered with the first object, after torch is imported, so that it
    # runs before torch's own exit handlers
    global _registered
    if not _registered:
        atexit.register(_close_all)
        _registered = True
    _live.add(obj)


def info_from_bytes(buf):
    """Parse a 24-byte sfft_solve_info copied to the host."""
    raw = bytes(buf)
    s = sfft_solve_info.from_buffer_copy(raw[: ctypes.sizeof(sfft_solve_info)])
    return {"status": s.status, "iters": s.iters, "rel_residual": s.rel_residual, "min_pivot": s.min_pivot}


class SfftPlan:
    """One plan (workspace + tables) for a fixed image size and fit configuration."""

    def __init__(self, n0, n1, w0, w1, dk, db, const_phot_ratio, dtype="float32", precision="mixed",
                 stream=None, spline=None):
        """spline: None (polynomial basis of degrees dk, db) or (kdeg, kint, bdeg, bint) for
        tensor-product B-splines (Eq. 7-9), with dk = db = 0."""
        torch = _torch()
        self.cfg = make_config(n0, n1, w0, w1, dk, db, const_phot_ratio, dtype, precision, spline)
        self.n = sfft_num_unknowns(self.cfg)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = sfft_plan_create(self.cfg, self.stream)
        _track(self)
        self.shape = (n0, n1)
        self.dtype = {"float32": torch.float32, "f32": torch.float32,
                      "float64": torch.float64, "f64": torch.float64}[str(dtype)]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if self.handle:
            sfft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self):
        return sfft_plan_workspace_bytes(self.handle)

    @property
    def solve_panel(self):
        """Panel width of the FP32 solve's blocked Cholesky (32 or 64)."""
        return binding.sfft_plan_solve_panel(self.handle)

    @solve_panel.setter
    def solve_panel(self, width):
        binding.sfft_plan_set_solve_panel(self.handle, width)

    def _check_img(self, t):
        torch = _torch()
        assert t.is_cuda and t.dtype == self.dtype and tuple(t.shape) == self.shape and t.is_contiguous(), \
            f"expected a contiguous {self.dtype} CUDA tensor of shape {self.shape}"
        return t

    def build_system(self, ref, sci, mask=None):
        torch = _torch()
        self._check_img(ref), self._check_img(sci)
        M = torch.empty((self.n, self.n), dtype=torch.float64, device=self.device)
        rhs = torch.empty(self.n, dtype=torch.float64, device=self.device)
        sfft_build_system(self.handle, ref, sci, mask, M, rhs, self.stream)
        return M, rhs

    def solve(self, M, rhs):
        torch = _torch()
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        info = torch.zeros(ctypes.sizeof(sfft_solve_info), dtype=torch.uint8, device=self.device)
        sfft_solve(self.handle, M, rhs, x, info, self.stream)
        return x, info

    def subtract(self, ref, sci, x):
        torch = _torch()
        self._check_img(ref), self._check_img(sci)
        D = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        sfft_subtract(self.handle, ref, sci, x, D, self.stream)
        return D

    def autotune(self, ref, sci):
        """Pick the fastest launch shapes for this plan (sfft_plan_autotune); returns them."""
        torch = _torch()
        self._check_img(ref), self._check_img(sci)
        D = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        binding.sfft_plan_autotune(self.handle, ref, sci, D, self.stream)
        return binding.sfft_plan_tuning(self.handle)

    def decorrelate(self, x, diff, sigma_ref, sigma_sci, xt0=0.0, yt0=0.0, out=None):
        """Noise decorrelation of a difference image (App. C); see sfft_decorrelate."""
        torch = _torch()
        self._check_img(diff)
        out = out if out is not None else torch.empty_like(diff)
        binding.sfft_decorrelate(self.handle, x, xt0, yt0, sigma_ref, sigma_sci, diff, out, self.stream)
        return out

    def decorrelate_coadd(self, x, diff, G, sigma_sci, H, sigma_ref, xt0=0.0, yt0=0.0, out=None):
        """Noise decorrelation in the co-added form of App. C (sfft_decorrelate_coadd):
        G, H: FP64 CUDA tensors [n, 2g0+1, 2g1+1] of the homogenisation kernels."""
        torch = _torch()
        out = out if out is not None else torch.empty_like(diff)
        binding.sfft_decorrelate_coadd(self.handle, x, xt0, yt0, G.contiguous(), sigma_sci, H.contiguous(),
                                       sigma_ref, diff, out, self.stream)
        return out

    def run_pair(self, ref, sci, mask=None, out=None, keep_system=False):
        torch = _torch()
        self._check_img(ref), self._check_img(sci)
        D = out if out is not None else torch.empty(self.shape, dtype=self.dtype, device=self.device)
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        info = torch.zeros(ctypes.sizeof(sfft_solve_info), dtype=torch.uint8, device=self.device)
        M = rhs = None
        if keep_system:
            M = torch.empty((self.n, self.n), dtype=torch.float64, device=self.device)
            rhs = torch.empty(self.n, dtype=torch.float64, device=self.device)
        sfft_run_pair(self.handle, ref, sci, mask, M, rhs, x, info, D, self.stream)
        return D, x, info, M, rhs

    def run_pair_host(self, ref, sci, mask=None, x_out=None, diff_out=None):
        """Host (preferably pinned) tensors in and out; synchronises before returning."""
        torch = _torch()
        D = diff_out if diff_out is not None else torch.empty(self.shape, dtype=self.dtype)
        x = x_out if x_out is not None else torch.empty(self.n, dtype=torch.float64)
        info = sfft_solve_info()
        sfft_run_pair_host(self.handle, ref, sci, mask, x, info, D, self.stream)
        return D, x, {"status": info.status, "iters": info.iters, "rel_residual": info.rel_residual,
                      "min_pivot": info.min_pivot}


def run_pairs(plans, refs, scis, masks=None, outs=None):
    """Pairs i = 0..len(plans)-1, pair i on plans[i] (SfftPlan objects, all
    distinct, one precision), through sfft_run_pairs on the first plan's
    stream: systems built pair by pair, solved up to eight per launch, then
    subtracted.  Returns [(D, x, info)] as SfftPlan.run_pair does."""
    torch = _torch()
    if not plans:
        return []
    for p, r, s in zip(plans, refs, scis):
        p._check_img(r), p._check_img(s)
    Ds = [outs[i] if outs is not None and outs[i] is not None else
          torch.empty(p.shape, dtype=p.dtype, device=p.device) for i, p in enumerate(plans)]
    xs = [torch.empty(p.n, dtype=torch.float64, device=p.device) for p in plans]
    infos = [torch.zeros(ctypes.sizeof(sfft_solve_info), dtype=torch.uint8, device=p.device) for p in plans]
    sfft_run_pairs([p.handle for p in plans], refs, scis, masks, xs, infos, Ds, plans[0].stream)
    return list(zip(Ds, xs, infos))


class SfftBatch:
    """A batch of pairs captured once into a CUDA graph (sfft_batch_*) and
    replayed by launch(): pair i on plans[i] (distinct SfftPlan objects of one
    precision) with the fixed device tensors refs[i], scis[i] (and masks[i]);
    write new images into those tensors between launches.  Outputs D, x and
    info per pair are allocated here (or taken from outs) and rewritten by
    every launch.  solve_group: systems per solve launch (1..8), or 0 to pick
    the fastest grouping by timing replays at creation."""

    def __init__(self, plans, refs, scis, masks=None, outs=None, solve_group=0):
        torch = _torch()
        for p, r, s in zip(plans, refs, scis):
            p._check_img(r), p._check_img(s)
        self.plans = list(plans)
        self.refs, self.scis = list(refs), list(scis)
        self.masks = None if masks is None else list(masks)
        self.D = [outs[i] if outs is not None and outs[i] is not None else
                  torch.empty(p.shape, dtype=p.dtype, device=p.device) for i, p in enumerate(plans)]
        self.x = [torch.empty(p.n, dtype=torch.float64, device=p.device) for p in plans]
        self.info = [torch.zeros(ctypes.sizeof(sfft_solve_info), dtype=torch.uint8, device=p.device)
                     for p in plans]
        self.handle = binding.sfft_batch_create([p.handle for p in plans], self.refs, self.scis, self.masks,
                                                self.x, self.info, self.D, solve_group)
        _track(self)

    @property
    def info_dict(self):
        return binding.sfft_batch_info(self.handle)

    def launch(self, stream=None):
        """Enqueue the whole batch on `stream` (default: torch's current stream)."""
        if stream is None:
            stream = _torch().cuda.current_stream()
        binding.sfft_batch_launch(self.handle, stream)

    def close(self):
        if self.handle:
            binding.sfft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SfftServer:
    """Several pairs of one configuration in flight (sfft_submit / sfft_poll / sfft_wait).

    Tensors on the GPU make device requests (inputs ready in ``stream``'s
    order, by default torch's current stream); CPU tensors (pinned for
    overlap) make host requests.  The server keeps every tensor of a request
    alive until its ticket has been waited for.
    """

    def __init__(self, n0, n1, w0, w1, dk, db, const_phot_ratio, dtype="float32", precision="mixed", depth=2,
                 batch=1, spline=None, eager=False):
        torch = _torch()
        self.cfg = make_config(n0, n1, w0, w1, dk, db, const_phot_ratio, dtype, precision, spline)
        self.n = sfft_num_unknowns(self.cfg)
        self.shape = (n0, n1)
        self.dtype = {"float32": torch.float32, "f32": torch.float32,
                      "float64": torch.float64, "f64": torch.float64}[str(dtype)]
        self.handle = sfft_server_create(self.cfg, depth, batch)
        _track(self)
        self._pending = {}
        if eager:
            binding.sfft_server_set_eager(self.handle, True)

    @property
    def workspace_bytes(self):
        return sfft_server_workspace_bytes(self.handle)

    def submit(self, ref, sci, mask=None, diff=None, x=None, info=None, stream=None):
        """Enqueue one pair; returns (ticket, diff, x, info) with the outputs still being written."""
        torch = _torch()
        host = not ref.is_cuda
        dev = "cpu" if host else ref.device
        for t in (ref, sci):
            assert t.dtype == self.dtype and tuple(t.shape) == self.shape and t.is_contiguous()
            assert t.is_cuda != host
        pin = dict(pin_memory=True) if host else {}
        if diff is None:
            diff = torch.empty(self.shape, dtype=self.dtype, device=dev, **pin)
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=dev, **pin)
        if info is None:
            info = torch.zeros(ctypes.sizeof(sfft_solve_info), dtype=torch.uint8, device=dev, **pin)
        if stream is None and not host:
            stream = torch.cuda.current_stream()
        req = make_request(ref, sci, diff, mask=mask, x=x, info=info, stream=stream, host=host)
        ticket = sfft_submit(self.handle, req)
        self._pending[ticket.seq] = (req, ref, sci, mask, diff, x, info)
        return ticket, diff, x, info

    def _release(self, seq):
        # requests complete in submission order
        for k in [k for k in self._pending if k <= seq]:
            del self._pending[k]

    def poll(self, ticket):
        done = sfft_poll(self.handle, ticket)
        if done:
            self._release(ticket.seq)
        return done

    def wait(self, ticket, timeout_us=-1):
        done = sfft_wait(self.handle, ticket, timeout_us)
        if done:
            self._release(ticket.seq)
        return done

    @property
    def launch_count(self):
        return binding.sfft_server_launch_count(self.handle)

    def flush(self):
        binding.sfft_flush(self.handle)

    def stream_wait(self, ticket, stream=None):
        """Order `stream` (default: torch's current stream) after the ticket's request."""
        if stream is None:
            stream = _torch().cuda.current_stream()
        sfft_stream_wait_ticket(self.handle, ticket, stream)

    def close(self):
        if self.handle:
            sfft_server_destroy(self.handle)
            self.handle = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SfftPool:
    """Pairs of many configurations under one device-memory budget
    (sfft_pool_*): one lane per configuration, created on first use,
    idle lanes released least recently used first to admit new ones."""

    def __init__(self, budget_bytes, depth=2, batch=1, eager=False):
        self.handle = binding.sfft_pool_create(budget_bytes, depth, batch)
        _track(self)
        self._keep = {}
        if eager:
            binding.sfft_pool_set_eager(self.handle, True)

    def submit(self, ref, sci, w0, w1, dk, db, const_phot_ratio, precision="mixed", mask=None, diff=None,
               stream=None, spline=None):
        """Enqueue a pair; returns (ticket, diff, x, info), or None if it cannot be admitted now."""
        torch = _torch()
        host = not ref.is_cuda
        dtype = {torch.float32: "float32", torch.float64: "float64"}[ref.dtype]
        n0, n1 = ref.shape
        cfg = make_config(n0, n1, w0, w1, dk, db, const_phot_ratio, dtype, precision, spline)
        n = sfft_num_unknowns(cfg)
        dev = "cpu" if host else ref.device
        pin = dict(pin_memory=True) if host else {}
        if diff is None:
            diff = torch.empty((n0, n1), dtype=ref.dtype, device=dev, **pin)
        x = torch.empty(n, dtype=torch.float64, device=dev, **pin)
        info = torch.zeros(ctypes.sizeof(sfft_solve_info), dtype=torch.uint8, device=dev, **pin)
        if stream is None and not host:
            stream = torch.cuda.current_stream()
        req = make_request(ref, sci, diff, mask=mask, x=x, info=info, stream=stream, host=host)
        t = binding.sfft_pool_submit(self.handle, cfg, req)
        if t is None:
            return None
        self._keep[(t.lane, t.seq)] = (req, ref, sci, mask, diff, x, info)
        return t, diff, x, info

    def wait(self, ticket, timeout_us=-1):
        done = binding.sfft_pool_wait(self.handle, ticket, timeout_us)
        if done:
            self._keep.pop((ticket.lane, ticket.seq), None)
        return done

    def poll(self, ticket):
        return binding.sfft_pool_poll(self.handle, ticket)

    @property
    def usage(self):
        return binding.sfft_pool_usage(self.handle)

    def close(self):
        if self.handle:
            binding.sfft_pool_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
