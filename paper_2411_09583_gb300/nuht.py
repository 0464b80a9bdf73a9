"""Python binding of the GB300 NUHT library (argument marshalling only).

    g_k = sum_j c_j J_nu(omega_k r_j)      (the discrete Hankel transform, Sec. 1)

Every step of the transform runs in libnuht.so (CUDA, sm_103a); this module
only checks tensors, passes device pointers and the current CUDA stream, and
wraps status codes.  PyTorch provides device memory and streams.
"""
import ctypes

import numpy as np
import torch

from . import _native as N


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(x, name):
    if not isinstance(x, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not x.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if x.dtype not in (torch.float64, torch.complex128):
        raise TypeError("%s must be float64 or complex128, got %s" % (name, x.dtype))
    return x.contiguous()


def make_opts(precision="fp64", min_size=1024, n_split_cand=16, m_terms=0, class_mask=7,
              timing=False, spread_tile=0, deterministic=False, persistent=False, interp_tile=0,
              vec_group=0):
    o = N.NuhtOpts()
    N.lib().nuht_default_opts(ctypes.byref(o))
    o.precision = {"fp64": N.PREC_FP64, "mixed": N.PREC_MIXED}[precision]
    o.min_size = int(min_size)
    o.n_split_cand = int(n_split_cand)
    o.m_terms = int(m_terms)
    o.class_mask = int(class_mask)
    # False: off; True: stage events on each stage's stream (the block classes
    # overlap); "serial": every stage in order on the caller's stream
    o.timing = 2 if timing == "serial" else (1 if timing else 0)
    o.spread_tile = int(spread_tile)
    o.deterministic = 1 if deterministic else 0
    o.persistent = 1 if persistent else 0
    o.interp_tile = int(interp_tile)
    o.vec_group = int(vec_group)
    return o


def kernel_launch_count():
    """Kernels launched by libnuht.so in this process so far."""
    return int(N.lib().nuht_kernel_launch_count())


def probe_alu(kind, iters=1 << 16, stream=None):
    """Time the throughput probe nuht_probe_alu: kind "ffma" (FP32), "dfma"
    (FP64) or "acc_fma" (double-float compensated multiply-add).  Returns
    (milliseconds, multiply-adds, FLOP/s with 2 FLOP per multiply-add)."""
    k = {"ffma": 0, "dfma": 1, "acc_fma": 2}[kind]
    ms, ops = ctypes.c_double(), ctypes.c_double()
    N.check(N.lib().nuht_probe_alu(k, int(iters), ctypes.byref(ms), ctypes.byref(ops),
                                   _stream_ptr(stream)), "nuht_probe_alu")
    return ms.value, ops.value, 2.0 * ops.value / (ms.value * 1e-3)


def check_blocks(nu, eps, r_sorted, omega_sorted, ranges, classes, min_size=1024, m_terms=0):
    """Host check of a work list through nuht_check_blocks: ranges (count, 4) of
    (k0, k1, j0, j1) into the sorted arrays, classes (count,) of NUHT_BLOCK_*.
    Returns the status code (NUHT_OK when the list is a valid subdivision)."""
    r = np.ascontiguousarray(r_sorted, dtype=np.float64)
    w = np.ascontiguousarray(omega_sorted, dtype=np.float64)
    rg = np.ascontiguousarray(np.asarray(ranges, dtype=np.int64).reshape(-1, 4))
    cl = np.ascontiguousarray(classes, dtype=np.int32)
    if cl.size != rg.shape[0]:
        raise ValueError("one class per block")
    return int(N.lib().nuht_check_blocks(int(nu), float(eps), int(m_terms), r.ctypes.data_as(ctypes.c_void_p),
                                         r.size, w.ctypes.data_as(ctypes.c_void_p), w.size, int(min_size),
                                         rg.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                                         cl.size))


def stage_names():
    return [N.lib().nuht_stage_name(i).decode() for i in range(N.NUM_STAGES)]


def choose_params(nu, eps, m_terms=0):
    """(M, z, L) of Sec. 3.3 as chosen by the library (host computation)."""
    M, z, L = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    N.check(N.lib().nuht_choose_params(int(nu), float(eps), int(m_terms), ctypes.byref(M),
                                       ctypes.byref(z), ctypes.byref(L)), "nuht_choose_params")
    return M.value, z.value, L.value


class Plan:
    """A plan for order nu, points r (n,) and frequencies omega (m,), tolerance eps.

    r and omega are float64 CUDA tensors (any order, values >= 0).
    """

    def __init__(self, nu, r, omega, eps, stream=None, **opts):
        r = _dev_f64(r, "r")
        omega = _dev_f64(omega, "omega")
        if r.dtype != torch.float64 or omega.dtype != torch.float64:
            raise TypeError("r and omega must be float64")
        self.n, self.m = r.numel(), omega.numel()
        self.device = r.device
        self._opts = make_opts(**opts)
        self._h = ctypes.c_void_p()
        self._stream = stream
        with torch.cuda.device(self.device):
            N.check(N.lib().nuht_plan(ctypes.byref(self._h), int(nu), ctypes.c_void_p(r.data_ptr()),
                                      self.n, ctypes.c_void_p(omega.data_ptr()), self.m,
                                      float(eps), ctypes.byref(self._opts),
                                      _stream_ptr(stream)), "nuht_plan")

    @classmethod
    def many(cls, nus, r, n, omega, m, eps, stream=None, **opts):
        """A batch plan: problem i has order nus[i], n[i] points and m[i]
        frequencies; r and omega are the concatenations (float64 CUDA tensors).
        execute / adjoint then take and return concatenated vectors."""
        r = _dev_f64(r, "r")
        omega = _dev_f64(omega, "omega")
        nus = np.ascontiguousarray(nus, dtype=np.int32)
        n = np.ascontiguousarray(n, dtype=np.int64)
        m = np.ascontiguousarray(m, dtype=np.int64)
        if not (nus.size == n.size == m.size) or n.sum() != r.numel() or m.sum() != omega.numel():
            raise ValueError("sizes of the batch do not match r / omega")
        self = cls.__new__(cls)
        self.n, self.m = r.numel(), omega.numel()
        self.device = r.device
        self._opts = make_opts(**opts)
        self._h = ctypes.c_void_p()
        self._stream = stream
        self.sizes = (n.copy(), m.copy())
        with torch.cuda.device(self.device):
            N.check(N.lib().nuht_plan_many(
                ctypes.byref(self._h), int(nus.size), nus.ctypes.data_as(ctypes.c_void_p),
                ctypes.c_void_p(r.data_ptr()), n.ctypes.data_as(ctypes.c_void_p),
                ctypes.c_void_p(omega.data_ptr()), m.ctypes.data_as(ctypes.c_void_p), float(eps),
                ctypes.byref(self._opts), _stream_ptr(stream)), "nuht_plan_many")
        return self

    def _apply(self, fn, x, rows_in, rows_out, out, what):
        x = _dev_f64(x, "input")
        if x.shape[0] != rows_in:
            raise ValueError("%s: input must have %d rows, got %d" % (what, rows_in, x.shape[0]))
        is_c = x.dtype == torch.complex128
        nvec = 1 if x.dim() == 1 else int(np.prod(x.shape[1:]))
        shape = (rows_out,) + tuple(x.shape[1:])
        if out is None:
            out = torch.empty(shape, dtype=x.dtype, device=x.device)
        elif out.shape != shape or out.dtype != x.dtype or not out.is_contiguous():
            raise ValueError("%s: bad output tensor" % what)
        xin = torch.view_as_real(x) if is_c else x
        xo = torch.view_as_real(out) if is_c else out
        with torch.cuda.device(self.device):
            N.check(fn(self._h, ctypes.c_void_p(xin.data_ptr()), ctypes.c_void_p(xo.data_ptr()),
                       nvec, 1 if is_c else 0, _stream_ptr(self._stream)), what)
        return out

    def execute(self, c, out=None):
        """g = A c; c has n rows (float64 or complex128), g has m rows."""
        return self._apply(N.lib().nuht_execute, c, self.n, self.m, out, "nuht_execute")

    def adjoint(self, g, out=None):
        """c = A^T g; g has m rows, c has n rows."""
        return self._apply(N.lib().nuht_adjoint, g, self.m, self.n, out, "nuht_adjoint")

    def deriv(self):
        """The derivative plan (orders nu - 1 and nu + 1 on the same, already
        sorted points and frequencies) for gradients in r and omega."""
        return DerivPlan(self)

    def status(self):
        """Device errors since the last call (waits for the stream): NUHT_OK or,
        for instance, NUHT_ERR_TIMEOUT from a bounded wait that gave up."""
        return int(N.lib().nuht_status(self._h, _stream_ptr(self._stream)))

    def info(self):
        inf = N.NuhtPlanInfo()
        N.check(N.lib().nuht_info(self._h, ctypes.byref(inf)), "nuht_info")
        d = {f: getattr(inf, f) for f, _ in N.NuhtPlanInfo._fields_}
        d["plan_ms"] = list(d["plan_ms"])
        return d

    def blocks(self, cls):
        """(count, 4) int64 array of (k0, k1, j0, j1) for block class cls (0 local, 1 asy, 2 direct)."""
        cnt = ctypes.c_int64()
        N.check(N.lib().nuht_get_blocks(self._h, int(cls), None, 0, ctypes.byref(cnt)), "nuht_get_blocks")
        out = np.zeros((cnt.value, 4), dtype=np.int64)
        if cnt.value:
            N.check(N.lib().nuht_get_blocks(self._h, int(cls), out.ctypes.data_as(ctypes.c_void_p),
                                            cnt.value, ctypes.byref(cnt)), "nuht_get_blocks")
        return out

    def stage_times(self):
        """{stage: device ms} of the most recent execute (plan built with timing=True or
        "serial"; with True the stages of different block classes overlap)."""
        ms = (ctypes.c_double * N.NUM_STAGES)()
        N.check(N.lib().nuht_stage_times(self._h, ms, N.NUM_STAGES), "nuht_stage_times")
        return dict(zip(stage_names(), list(ms)))

    def permutations(self):
        pr = np.zeros(self.n, dtype=np.int32)
        pw = np.zeros(self.m, dtype=np.int32)
        N.check(N.lib().nuht_get_permutations(self._h, pr.ctypes.data_as(ctypes.c_void_p),
                                              pw.ctypes.data_as(ctypes.c_void_p)),
                "nuht_get_permutations")
        return pr, pw

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            N.lib().nuht_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class DerivPlan:
    """Gradients of sum_k e_k g_k, g = A c, with respect to r and omega
    (nuht_plan_deriv / nuht_grad_r / nuht_grad_omega); real c and e."""

    def __init__(self, base):
        self.n, self.m, self.device = base.n, base.m, base.device
        self._stream = base._stream
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            N.check(N.lib().nuht_plan_deriv(ctypes.byref(self._h), base._h, _stream_ptr(self._stream)),
                    "nuht_plan_deriv")

    def _grad(self, fn, c, e, rows, what):
        c, e = _dev_f64(c, "c"), _dev_f64(e, "e")
        if c.dtype != torch.float64 or e.dtype != torch.float64:
            raise TypeError("%s: real c and e" % what)
        if c.shape[0] != self.n or e.shape[0] != self.m or c.shape[1:] != e.shape[1:]:
            raise ValueError("%s: c must have %d rows and e %d, with the same vectors" % (what, self.n, self.m))
        nvec = 1 if c.dim() == 1 else int(np.prod(c.shape[1:]))
        out = torch.empty(rows, dtype=torch.float64, device=c.device)
        with torch.cuda.device(self.device):
            N.check(fn(self._h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                       ctypes.c_void_p(out.data_ptr()), nvec, _stream_ptr(self._stream)), what)
        return out

    def grad_r(self, c, e):
        """sum_v c[j, v] sum_k e[k, v] omega_k J_nu'(omega_k r_j), n entries."""
        return self._grad(N.lib().nuht_grad_r, c, e, self.n, "nuht_grad_r")

    def grad_omega(self, c, e):
        """sum_v e[k, v] sum_j c[j, v] r_j J_nu'(omega_k r_j), m entries."""
        return self._grad(N.lib().nuht_grad_omega, c, e, self.m, "nuht_grad_omega")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            N.lib().nuht_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def local_apply_noalloc(nu, r, omega, c, eps, r_max, omega_max, out=None, stream=None):
    """g = A c through nuht_local_apply_noalloc (no device allocation inside the call).

    For transforms whose whole matrix is local: r_max >= every r_j, omega_max >=
    every omega_k and omega_max * r_max <= z(nu, eps).  c: (n,) or (n, nvec) float64
    CUDA tensor; returns g with m rows.  `out` may pass a preallocated output.
    """
    r = _dev_f64(r, "r")
    omega = _dev_f64(omega, "omega")
    c = _dev_f64(c, "c")
    nvec = 1 if c.dim() == 1 else int(np.prod(c.shape[1:]))
    shape = (omega.numel(),) + tuple(c.shape[1:])
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=c.device)
    with torch.cuda.device(c.device):
        N.check(N.lib().nuht_local_apply_noalloc(
            int(nu), float(eps), ctypes.c_void_p(r.data_ptr()), r.numel(), float(r_max),
            ctypes.c_void_p(omega.data_ptr()), omega.numel(), float(omega_max),
            ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(out.data_ptr()), nvec,
            _stream_ptr(stream)), "nuht_local_apply_noalloc")
    return out


def nuht(nu, r, omega, c, eps, **opts):
    """One-shot transform on device tensors: plan, execute, release."""
    with Plan(nu, r, omega, eps, **opts) as p:
        return p.execute(c)


def transform_host(nu, r, omega, c, eps, stream=None, out=None, **opts):
    """Whole transform from host arrays through nuht_transform_host (real c).

    out: optional C-contiguous float64 host array of shape (m,) + c.shape[1:]
    for the result (pinned memory makes the device-to-host copy direct)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    nvec = 1 if c.ndim == 1 else int(np.prod(c.shape[1:]))
    shape = (omega.size,) + c.shape[1:]
    if out is None:
        g = np.empty(shape, dtype=np.float64)
    else:
        g = out
        if g.shape != shape or g.dtype != np.float64 or not g.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of shape %s" % (shape,))
    o = make_opts(**opts)
    N.check(N.lib().nuht_transform_host(int(nu), r.ctypes.data_as(ctypes.c_void_p), r.size,
                                        omega.ctypes.data_as(ctypes.c_void_p), omega.size,
                                        float(eps), c.ctypes.data_as(ctypes.c_void_p),
                                        g.ctypes.data_as(ctypes.c_void_p), nvec, ctypes.byref(o),
                                        _stream_ptr(stream)), "nuht_transform_host")
    return g
