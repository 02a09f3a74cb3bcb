"""Thin ctypes binding of libhydro.so (include/hydro.h).

Argument marshalling only: every stage of the step runs in the library's CUDA
kernels.  Functions keep the C names.  Tensors are PyTorch CUDA float64
tensors of shape (5, gz, gy, gx) over the grown box (x fastest); PyTorch is
used for device memory and streams only.  There is no CPU fallback: if the
library cannot be loaded, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "_build")

HYDRO_OK, HYDRO_EINVAL, HYDRO_ENOMEM, HYDRO_ECUDA = 0, -1, -2, -3
HYDRO_EBADSTATE, HYDRO_EAGAIN, HYDRO_ETIMEDOUT, HYDRO_ENOTIMPL = -4, -5, -6, -7
HYDRO_ETOOBIG = -8
HYDRO_ECANCELED = -9
NOALLOC_MAX_ZONES = 64000
BC_OUTFLOW, BC_REFLECT, BC_PERIODIC, BC_PREFILLED = 0, 1, 2, 3
MOL_MAX_SPECIES = 32  # HYDRO_MOL_MAX_SPECIES
FLAG_NO_FLATTEN = 1
FLAG_NO_AUTOTUNE = 2
FLAG_EINFELDT = 4
FLAG_FLUX_GRAV_ENERGY = 8
NG = 4


class HydroError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class hydro_params_t(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("grav", ctypes.c_double * 3),
        ("small_dens", ctypes.c_double),
        ("small_pres", ctypes.c_double),
        ("dim", ctypes.c_int),
        ("flags", ctypes.c_uint),
    ]


class hydro_box_t(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_void_p),
        ("n", ctypes.c_int * 3),
        ("ng", ctypes.c_int),
        ("stride", ctypes.c_longlong * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
    ]


class hydro_amr_t(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("domain", ctypes.c_int * 3),
        ("domain_bc", (ctypes.c_int * 2) * 3),
        ("ncoarse", ctypes.c_int),
        ("coarse_in", ctypes.POINTER(hydro_box_t)),
        ("coarse_out", ctypes.POINTER(hydro_box_t)),
        ("coarse_lo", ctypes.POINTER(ctypes.c_int)),
        ("nfine", ctypes.c_int),
        ("fine_in", ctypes.POINTER(hydro_box_t)),
        ("fine_out", ctypes.POINTER(hydro_box_t)),
        ("fine_lo", ctypes.POINTER(ctypes.c_int)),
    ]


PROB_SOD, PROB_SEDOV, PROB_TWO_STATE = 0, 1, 2


class hydro_request_t(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("n", ctypes.c_int), ("steps", ctypes.c_int),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("p_l", ctypes.c_double), ("rho_r", ctypes.c_double), ("p_r", ctypes.c_double),
        ("energy", ctypes.c_double), ("p_ambient", ctypes.c_double),
        ("result_host", ctypes.c_void_p),
    ]


class hydro_result_t(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("steps_done", ctypes.c_int), ("t_final", ctypes.c_double),
        ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("zone_updates", ctypes.c_longlong),
    ]


class hydro_serve_stats_t(ctypes.Structure):
    _fields_ = [
        ("queued", ctypes.c_int), ("active", ctypes.c_int),
        ("admitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("iterations", ctypes.c_longlong),
        ("zone_updates", ctypes.c_longlong), ("busy_ms", ctypes.c_double),
        ("hbm_budget", ctypes.c_size_t), ("hbm_states", ctypes.c_size_t), ("hbm_scratch_pool", ctypes.c_size_t),
        ("box_steps", ctypes.c_longlong), ("enqueue_ms", ctypes.c_double), ("ms_per_unit", ctypes.c_double),
    ]


SERVE_ALL, SERVE_RESPONSE_RATIO = 0, 1


_LIBS = {}


def library_path(variant="default"):
    name = "libhydro.so" if variant == "default" else "libhydro_exact.so"
    return os.path.join(LIBDIR, name)


def lib(variant="default"):
    """Load libhydro (variant 'default') or its no-contraction build ('exact')."""
    if variant in _LIBS:
        return _LIBS[variant]
    path = library_path(variant)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1711_06203_b300/build.py)")
    L = ctypes.CDLL(path)
    vp, P, B = ctypes.c_void_p, ctypes.POINTER(hydro_params_t), ctypes.POINTER(hydro_box_t)
    D = ctypes.POINTER(ctypes.c_double)
    L.hydro_ctx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.hydro_ctx_destroy.argtypes = [vp]
    L.hydro_ctx_destroy.restype = None
    L.hydro_ctx_check.argtypes = [vp]
    L.hydro_strerror.argtypes = [ctypes.c_int]
    L.hydro_strerror.restype = ctypes.c_char_p
    L.hydro_dt.argtypes = [vp, B, P, D, vp]
    L.hydro_advance_box.argtypes = [vp, B, B, P, ctypes.c_double, D, vp]
    L.hydro_advance_box_noalloc.argtypes = [B, B, P, ctypes.c_double, D, vp]
    L.hydro_advance_box_host.argtypes = [vp, B, B, P, ctypes.c_double, D, vp]
    L.hydro_advance_box_retry.argtypes = [vp, B, B, P, ctypes.c_double, ctypes.c_int, D, D, vp]
    L.hydro_advance_batch.argtypes = [vp, B, B, ctypes.c_int, P, vp, vp, ctypes.POINTER(ctypes.c_int), vp]
    L.hydro_batch_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    IP = ctypes.POINTER(ctypes.c_int)
    L.hydro_fill_boundary.argtypes = [vp, B, IP, ctypes.c_int, ctypes.c_int, IP, IP, vp]
    L.hydro_level_min_dt.argtypes = [vp, vp, ctypes.c_int, vp]
    L.hydro_selftest_scale2.argtypes = [vp, vp, vp, ctypes.c_longlong, vp]
    L.hydro_selftest_divsqrt.argtypes = [vp, vp, vp, vp, vp, ctypes.c_longlong, vp]
    L.hydro_selftest_intpipe.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, vp]
    L.hydro_mol_advance_box.argtypes = [vp, B, B, P, ctypes.c_int, ctypes.c_double, D, vp]
    L.hydro_amr_advance.argtypes = [vp, ctypes.POINTER(hydro_amr_t), P, vp, vp, ctypes.POINTER(ctypes.c_int), vp]
    L.serve_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_int]
    L.serve_submit.argtypes = [vp, ctypes.POINTER(hydro_request_t), ctypes.POINTER(ctypes.c_uint64)]
    L.serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(hydro_result_t), ctypes.c_int]
    L.serve_stats.argtypes = [vp, ctypes.POINTER(hydro_serve_stats_t)]
    L.serve_set_policy.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.serve_cancel.argtypes = [vp, ctypes.c_uint64]
    L.serve_destroy.argtypes = [vp]
    L.serve_destroy.restype = None
    L.hydro_ctx_set_profiling.argtypes = [vp, ctypes.c_int]
    L.hydro_ctx_stage_times.argtypes = [vp, D, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    L.hydro_ctx_launches.argtypes = [vp]
    L.hydro_ctx_launches.restype = ctypes.c_longlong
    L.hydro_ctx_record_face_fluxes.argtypes = [vp, ctypes.c_int]
    L.hydro_ctx_set_scratch_limit.argtypes = [vp, ctypes.c_size_t]
    L.hydro_ctx_fail_allocations.argtypes = [vp, ctypes.c_int]
    L.hydro_selftest_fp64_rate.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    L.hydro_selftest_rsqrt.argtypes = [vp, vp, ctypes.c_longlong, vp]
    L.hydro_advance_box_steps.argtypes = [vp, ctypes.POINTER(hydro_box_t), ctypes.POINTER(hydro_box_t),
                                          ctypes.POINTER(hydro_params_t), ctypes.c_int, vp, vp, vp]
    L.hydro_ctx_face_flux.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
    L.hydro_pipe_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    _LIBS[variant] = L
    return L


def strerror(status):
    try:
        return lib().hydro_strerror(int(status)).decode()
    except Exception:
        return "unknown"


def params(dim, gamma=1.4, cfl=0.5, grav=(0.0, 0.0, 0.0), small_dens=1e-200, small_pres=1e-200, flatten=True,
           einfeldt=False, flux_grav_energy=False):
    p = hydro_params_t()
    p.gamma, p.cfl, p.dim = gamma, cfl, dim
    for a in range(3):
        p.grav[a] = grav[a]
    p.small_dens, p.small_pres = small_dens, small_pres
    p.flags = (0 if flatten else FLAG_NO_FLATTEN) | (FLAG_EINFELDT if einfeldt else 0) | \
        (FLAG_FLUX_GRAV_ENERGY if flux_grav_energy else 0)
    return p


def box(t, n, dx, bc=BC_OUTFLOW):
    """hydro_box_t describing tensor t (5 [+ species], gz, gy, gx), float64, x contiguous.
    n: interior (nx, ny, nz); bc: one kind for every face or a 3x2 nested sequence."""
    if t.dtype.itemsize != 8 or t.dim() != 4 or t.shape[0] < 5 or t.stride(3) != 1:
        raise ValueError("box tensor must be float64 of shape (5 [+ species], gz, gy, gx) with x contiguous")
    b = hydro_box_t()
    b.u = t.data_ptr()
    for a in range(3):
        b.n[a] = int(n[a]) if a < len(n) else 1
        b.dx[a] = float(dx[a])
        for s in range(2):
            b.bc[a][s] = bc if isinstance(bc, int) else bc[a][s]
    b.ng = NG
    b.stride[0], b.stride[1], b.stride[2] = t.stride(2), t.stride(1), t.stride(0)
    return b


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def hydro_selftest_scale2(x, variant="default", stream=None):
    """Run the kernels' integer-pipe 2x and x/2 over a CUDA float64 tensor;
    returns (twice, half) tensors."""
    import torch
    x = x.contiguous()
    t, h = torch.empty_like(x), torch.empty_like(x)
    rc = lib(variant).hydro_selftest_scale2(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                            ctypes.c_void_p(h.data_ptr()), x.numel(), _stream_handle(stream))
    if rc:
        raise HydroError(rc, "hydro_selftest_scale2")
    return t, h


PIPE_RANGES = ("h2d", "prim", "xy", "tz", "f1z", "f2xz", "f2z", "f3xy", "f3z", "upd")


def hydro_pipe_plan(nz, nchunk, bc_low):
    """The host-buffer step's chunk schedule (host only): (pre_lo, [per chunk
    {range name: (lo, hi)} plus "ghosts_low", "ghosts_high"])."""
    pre = ctypes.c_int(0)
    out = (ctypes.c_int * (22 * max(nchunk, 1)))()
    rc = lib().hydro_pipe_plan(int(nz), int(nchunk), int(bc_low), ctypes.byref(pre), out)
    if rc:
        raise HydroError(rc, "hydro_pipe_plan")
    chunks = []
    for k in range(nchunk):
        o = out[22 * k: 22 * k + 22]
        c = {name: (o[2 * r], o[2 * r + 1]) for r, name in enumerate(PIPE_RANGES)}
        c["ghosts_low"], c["ghosts_high"] = bool(o[20]), bool(o[21])
        chunks.append(c)
    return pre.value, chunks


def hydro_selftest_rsqrt(x, variant="default", stream=None):
    """Run the kernels' refined reciprocal square root over a CUDA float64 tensor."""
    import torch
    x = x.contiguous()
    out = torch.empty_like(x)
    rc = lib(variant).hydro_selftest_rsqrt(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
                                           _stream_handle(stream))
    if rc:
        raise HydroError(rc, "hydro_selftest_rsqrt")
    return out


def hydro_selftest_fp64_rate(nblocks=148 * 8, iters=4096, variant="default", stream=None, reps=3):
    """Measured FP64 rate of the device in GFLOP/s (2 flops per multiply-add),
    best of `reps` timed launches after one warm-up launch."""
    import torch
    out = torch.empty(nblocks * 256, dtype=torch.float64, device="cuda")
    st = stream or torch.cuda.current_stream()
    best = None
    for rep in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = lib(variant).hydro_selftest_fp64_rate(ctypes.c_void_p(out.data_ptr()), int(nblocks), int(iters),
                                                   _stream_handle(st))
        e1.record(st)
        if rc:
            raise HydroError(rc, "hydro_selftest_fp64_rate")
        e1.synchronize()
        if rep:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    return 2.0 * nblocks * 256 * 8 * iters / (best * 1e-3) / 1e9


def hydro_selftest_divsqrt(x, y, variant="default", stream=None):
    """Run the kernels' reciprocal, quotient and square root over CUDA float64
    tensors x, y; returns (1/x, y/x, sqrt(x)) tensors."""
    import torch
    x, y = x.contiguous(), y.contiguous()
    r, q, s = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    rc = lib(variant).hydro_selftest_divsqrt(*[ctypes.c_void_p(t.data_ptr()) for t in (x, y, r, q, s)], x.numel(),
                                             _stream_handle(stream))
    if rc:
        raise HydroError(rc, "hydro_selftest_divsqrt")
    return r, q, s


def hydro_selftest_intpipe(x, y, variant="default", stream=None):
    """Run the kernels' integer-pipe product and sum over CUDA float64 tensors
    x, y; returns (x*y, x+y) tensors."""
    import torch
    x, y = x.contiguous(), y.contiguous()
    p, s = torch.empty_like(x), torch.empty_like(x)
    rc = lib(variant).hydro_selftest_intpipe(*[ctypes.c_void_p(t.data_ptr()) for t in (x, y, p, s)], x.numel(),
                                             _stream_handle(stream))
    if rc:
        raise HydroError(rc, "hydro_selftest_intpipe")
    return p, s


def hydro_advance_box_noalloc(bin_, bout, p, dt, want_dt_next=False, stream=None, variant="default"):
    """The allocation-free step: no context, fixed library-owned scratch (see
    include/hydro.h).  Returns (status, dt_next or None); never raises on a
    status so callers can test HYDRO_ETOOBIG and friends."""
    L = lib(variant)
    out = ctypes.c_double(0.0)
    rc = L.hydro_advance_box_noalloc(ctypes.byref(bin_), ctypes.byref(bout), ctypes.byref(p), float(dt),
                                     ctypes.byref(out) if want_dt_next else None, _stream_handle(stream))
    return rc, (out.value if want_dt_next else None)


class Context:
    """A hydro_ctx_t on one device (owns scratch and flags)."""

    def __init__(self, device=0, variant="default"):
        self.L = lib(variant)
        h = ctypes.c_void_p()
        rc = self.L.hydro_ctx_create(ctypes.byref(h), int(device))
        if rc:
            raise HydroError(rc, "hydro_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.hydro_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hydro_dt(self, b, p, stream=None):
        out = ctypes.c_double(0.0)
        rc = self.L.hydro_dt(self.h, ctypes.byref(b), ctypes.byref(p), ctypes.byref(out), _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_dt")
        return out.value

    def hydro_advance_box(self, bin_, bout, p, dt, want_dt_next=False, stream=None, raise_on_error=True):
        out = ctypes.c_double(0.0)
        rc = self.L.hydro_advance_box(self.h, ctypes.byref(bin_), ctypes.byref(bout), ctypes.byref(p), float(dt),
                                      ctypes.byref(out) if want_dt_next else None, _stream_handle(stream))
        if rc and raise_on_error:
            raise HydroError(rc, "hydro_advance_box")
        return (out.value if want_dt_next else None) if raise_on_error else (rc, out.value)

    def hydro_mol_advance_box(self, bin_, bout, p, nspec, dt, want_dt_next=False, stream=None, raise_on_error=True):
        """Method-of-lines step of a box with nspec passive species (5 + nspec components)."""
        out = ctypes.c_double(0.0)
        rc = self.L.hydro_mol_advance_box(self.h, ctypes.byref(bin_), ctypes.byref(bout), ctypes.byref(p), int(nspec),
                                          float(dt), ctypes.byref(out) if want_dt_next else None,
                                          _stream_handle(stream))
        if rc and raise_on_error:
            raise HydroError(rc, "hydro_mol_advance_box")
        return (out.value if want_dt_next else None) if raise_on_error else (rc, out.value)

    def hydro_advance_box_host(self, bin_, bout, p, dt, want_dt_next=False, stream=None):
        """The step on host buffers (hydro_box_t of CPU tensors in the natural
        grown layout); returns once the host output is written."""
        out = ctypes.c_double(0.0)
        rc = self.L.hydro_advance_box_host(self.h, ctypes.byref(bin_), ctypes.byref(bout), ctypes.byref(p), float(dt),
                                           ctypes.byref(out) if want_dt_next else None, _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_advance_box_host")
        return out.value if want_dt_next else None

    def hydro_advance_box_retry(self, bin_, bout, p, dt, max_retries=3, stream=None):
        """Returns (status, dt_taken, dt_next) of the step with retries on bad states."""
        taken, nxt = ctypes.c_double(0.0), ctypes.c_double(0.0)
        rc = self.L.hydro_advance_box_retry(self.h, ctypes.byref(bin_), ctypes.byref(bout), ctypes.byref(p), float(dt),
                                            int(max_retries), ctypes.byref(taken), ctypes.byref(nxt),
                                            _stream_handle(stream))
        return rc, taken.value, nxt.value

    def hydro_ctx_check(self):
        return self.L.hydro_ctx_check(self.h)

    def hydro_advance_batch(self, bins, bouts, p, dt_dev, dt_next_dev=None, want_bad=False, stream=None,
                            raise_on_error=True):
        """Batched step of a level.  bins/bouts: lists of hydro_box_t; dt_dev,
        dt_next_dev: CUDA float64 tensors of len(bins) (dt_next_dev optional).
        Returns the index of the first bad box (-1) when want_bad, else None."""
        n = len(bins)
        arr_in = (hydro_box_t * n)(*bins)
        arr_out = (hydro_box_t * n)(*bouts)
        bad = ctypes.c_int(-1)
        rc = self.L.hydro_advance_batch(self.h, arr_in, arr_out, n, ctypes.byref(p), ctypes.c_void_p(dt_dev.data_ptr()),
                                        ctypes.c_void_p(dt_next_dev.data_ptr()) if dt_next_dev is not None else None,
                                        ctypes.byref(bad) if want_bad else None, _stream_handle(stream))
        if rc and raise_on_error:
            raise HydroError(rc, "hydro_advance_batch")
        if not raise_on_error:
            return rc, bad.value
        return bad.value if want_bad else None

    def hydro_fill_boundary(self, boxes, lo, dim, domain, domain_bc, stream=None):
        """Fill the ghost zones of a level tiling [0, domain): boxes (hydro_box_t list),
        lo (per-box global corner triples), domain_bc ((lo, hi) kinds per axis)."""
        n = len(boxes)
        arr = (hydro_box_t * n)(*boxes)
        lo_arr = (ctypes.c_int * (3 * n))(*[int(v) for c in lo for v in (tuple(c) + (0,) * (3 - len(c)))])
        dom = (ctypes.c_int * 3)(*(list(domain) + [1] * (3 - len(domain))))
        bcs = (ctypes.c_int * 6)(*[int(k) for pair in domain_bc for k in pair] + [0] * (6 - 2 * len(domain_bc)))
        rc = self.L.hydro_fill_boundary(self.h, arr, lo_arr, n, dim, dom, bcs, _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_fill_boundary")

    def hydro_amr_advance(self, coarse_in, coarse_out, coarse_lo, fine_in, fine_out, fine_lo, dim, domain,
                          domain_bc, p, dt_dev, dt_next_dev, want_bad=False, stream=None):
        """One coarse step of a two-level hierarchy (refinement ratio 2).
        coarse_*/fine_*: lists of hydro_box_t; *_lo: corner triples (fine ones
        in the fine index space); dt_dev, dt_next_dev: CUDA float64 tensors of
        one element.  Returns the bad-state flag when want_bad, else None."""
        def boxes(lst):
            return (hydro_box_t * max(len(lst), 1))(*lst)

        def corners(lst):
            return (ctypes.c_int * max(3 * len(lst), 1))(*[int(v) for c in lst for v in (tuple(c) + (0,) * (3 - len(c)))])

        keep = [boxes(coarse_in), boxes(coarse_out), corners(coarse_lo), boxes(fine_in), boxes(fine_out), corners(fine_lo)]
        h = hydro_amr_t()
        h.dim = dim
        for a in range(3):
            h.domain[a] = int(domain[a]) if a < len(domain) else 1
            for s_ in range(2):
                h.domain_bc[a][s_] = int(domain_bc[a][s_]) if a < len(domain_bc) else 0
        h.ncoarse, h.nfine = len(coarse_in), len(fine_in)
        h.coarse_in, h.coarse_out, h.coarse_lo = keep[0], keep[1], keep[2]
        h.fine_in, h.fine_out, h.fine_lo = keep[3], keep[4], keep[5]
        bad = ctypes.c_int(0)
        rc = self.L.hydro_amr_advance(self.h, ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(dt_dev.data_ptr()),
                                      ctypes.c_void_p(dt_next_dev.data_ptr()), ctypes.byref(bad) if want_bad else None,
                                      _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_amr_advance")
        return bad.value if want_bad else None

    def hydro_level_min_dt(self, dt_next_dev, dt_dev, stream=None):
        rc = self.L.hydro_level_min_dt(ctypes.c_void_p(dt_next_dev.data_ptr()), ctypes.c_void_p(dt_dev.data_ptr()),
                                       dt_dev.numel(), _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_level_min_dt")

    def hydro_batch_tuning(self):
        """{(axis, extent): zones per sweep segment, or 0 for the warp rows / tiles}"""
        ax = (ctypes.c_int * 192)()
        ext = (ctypes.c_int * 192)()
        seg = (ctypes.c_int * 192)()
        k = self.L.hydro_batch_tuning(self.h, ax, ext, seg, 192)
        return {(ax[i], ext[i]): seg[i] for i in range(min(k, 192))}

    STAGES = ("prim", "trace", "flux1", "flux2", "flux3", "update")

    def hydro_ctx_set_profiling(self, enable):
        rc = self.L.hydro_ctx_set_profiling(self.h, 1 if enable else 0)
        if rc:
            raise HydroError(rc, "hydro_ctx_set_profiling")

    def hydro_ctx_stage_times(self):
        ms = (ctypes.c_double * 8)()
        calls = ctypes.c_longlong(0)
        n = self.L.hydro_ctx_stage_times(self.h, ms, 8, ctypes.byref(calls))
        if n < 0:
            raise HydroError(n, "hydro_ctx_stage_times")
        return {self.STAGES[i]: ms[i] for i in range(n)}, calls.value

    def hydro_ctx_launches(self):
        return self.L.hydro_ctx_launches(self.h)

    def hydro_advance_box_steps(self, a, b, p, nsteps, dt_dev, t_dev=None, stream=None):
        """nsteps steps alternating a -> b -> a ..., dt kept on the device in
        dt_dev (2 float64 on the device; dt_dev[0] = first dt); t_dev (1
        float64 on the device, optional) accumulates the steps' dts."""
        rc = self.L.hydro_advance_box_steps(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(p), int(nsteps),
                                            ctypes.c_void_p(dt_dev.data_ptr()),
                                            ctypes.c_void_p(t_dev.data_ptr()) if t_dev is not None else None,
                                            _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_advance_box_steps")

    def hydro_ctx_set_scratch_limit(self, nbytes):
        """Step 3-D boxes whose whole-box scratch exceeds nbytes slab by slab (0: never)."""
        rc = self.L.hydro_ctx_set_scratch_limit(self.h, int(nbytes))
        if rc:
            raise HydroError(rc, "hydro_ctx_set_scratch_limit")

    def hydro_ctx_fail_allocations(self, enable=True):
        """Fault injection: make the context's large device allocations fail (HYDRO_ENOMEM)."""
        rc = self.L.hydro_ctx_fail_allocations(self.h, 1 if enable else 0)
        if rc:
            raise HydroError(rc, "hydro_ctx_fail_allocations")

    def hydro_ctx_record_face_fluxes(self, enable=True):
        rc = self.L.hydro_ctx_record_face_fluxes(self.h, 1 if enable else 0)
        if rc:
            raise HydroError(rc, "hydro_ctx_record_face_fluxes")

    def hydro_ctx_face_flux(self, d, side, dst, stream=None):
        """Copy the recorded final fluxes through face `side` of axis d of the
        last recorded step into the device tensor dst (5 x n_t2 x n_t1 doubles)."""
        import torch
        assert dst.is_cuda and dst.dtype == torch.float64 and dst.is_contiguous()
        rc = self.L.hydro_ctx_face_flux(self.h, int(d), int(side), ctypes.c_void_p(dst.data_ptr()),
                                        _stream_handle(stream))
        if rc:
            raise HydroError(rc, "hydro_ctx_face_flux")


class Server:
    """A serve_t: continuous batching of independent hydro problems on one device."""

    def __init__(self, device=0, hbm_budget=0, max_slots=64, variant="default"):
        self.L = lib(variant)
        h = ctypes.c_void_p()
        rc = self.L.serve_create(ctypes.byref(h), int(device), int(hbm_budget), int(max_slots))
        if rc:
            raise HydroError(rc, "serve_create")
        self.h = h
        self._bufs = {}

    def serve_submit(self, kind, n, steps, gamma=1.4, cfl=0.5, rho_l=1.0, p_l=1.0, rho_r=0.125, p_r=0.1,
                     energy=1.0, p_ambient=1e-5, want_state=False):
        """Queue a request; returns its id.  want_state: keep a host copy of the final grown state."""
        import numpy as np
        r = hydro_request_t(kind, n, steps, gamma, cfl, rho_l, p_l, rho_r, p_r, energy, p_ambient, None)
        buf = None
        if want_state:
            buf = np.empty((5, n + 2 * NG, n + 2 * NG, n + 2 * NG), dtype=np.float64)
            r.result_host = buf.ctypes.data
        rid = ctypes.c_uint64(0)
        rc = self.L.serve_submit(self.h, ctypes.byref(r), ctypes.byref(rid))
        if rc:
            raise HydroError(rc, "serve_submit")
        self._bufs[rid.value] = buf
        return rid.value

    def serve_poll(self, rid, timeout_ms=-1):
        """Result dict of a finished request, or None if it is not finished within timeout_ms."""
        res = hydro_result_t()
        rc = self.L.serve_poll(self.h, ctypes.c_uint64(rid), ctypes.byref(res), int(timeout_ms))
        if rc in (HYDRO_EAGAIN, HYDRO_ETIMEDOUT):
            return None
        if rc:
            raise HydroError(rc, "serve_poll")
        out = {k: getattr(res, k) for k, _ in hydro_result_t._fields_}
        out["state"] = self._bufs.pop(rid, None)
        return out

    def serve_cancel(self, rid):
        """Cancel a request: its result (collected by serve_poll) carries HYDRO_ECANCELED
        unless it had already finished."""
        rc = self.L.serve_cancel(self.h, ctypes.c_uint64(rid))
        if rc:
            raise HydroError(rc, "serve_cancel")

    def serve_set_policy(self, policy, quantum_ms=2.5):
        """HYDRO_SERVE_ALL (0) or HYDRO_SERVE_RESPONSE_RATIO (1, the default) with
        its per-iteration quantum; only while the server is idle."""
        rc = self.L.serve_set_policy(self.h, int(policy), float(quantum_ms))
        if rc:
            raise HydroError(rc, "serve_set_policy")

    def serve_stats(self):
        st = hydro_serve_stats_t()
        rc = self.L.serve_stats(self.h, ctypes.byref(st))
        if rc:
            raise HydroError(rc, "serve_stats")
        return {k: getattr(st, k) for k, _ in hydro_serve_stats_t._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
