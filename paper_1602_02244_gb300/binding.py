"""ctypes binding of ``libfmm.so`` (include/fmm.h).

Argument marshalling only: every step of the FMM runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the
library has not been built, every call raises ``FMMError`` -- there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm.so")

FMM_FP64, FMM_MIXED = 0, 1
_STATUS = {0: "FMM_OK", 1: "FMM_ERR_INVALID_ARG", 2: "FMM_ERR_CUDA", 3: "FMM_ERR_OOM",
           4: "FMM_ERR_TIMEOUT", 5: "FMM_ERR_NONFINITE_INPUT", 6: "FMM_ERR_UNSUPPORTED"}

EXPORTS = ("fmm_plan_create", "fmm_plan_create_batch", "fmm_plan_rebuild", "fmm_plan_set_points",
           "fmm_eval", "fmm_eval_graph", "fmm_adjoint", "fmm_solve_host", "fmm_solve_adjoint_host",
           "fmm_sync", "fmm_plan_sizes", "fmm_plan_export", "fmm_plan_destroy", "fmm_direct",
           "fmm_laplace7_apply", "fmm_wait_selftest", "fmm_fp32_peak", "fmm_plan_tiles",
           "fmm_status_string", "fmm_last_error_message", "fmm_helmholtz_eval",
           "fmm_helmholtz7_apply", "fmm_fp64_peak")

EXPORT_FIELDS = ("keys", "perm", "level_offset", "box_key", "box_level", "box_first", "box_count",
                 "box_parent", "box_child", "box_nchild", "u_off", "u_idx", "v_off", "v_idx",
                 "w_off", "w_idx", "x_off", "x_idx", "root", "offsets", "radius")


class FMMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("coarse_fp64_levels", ctypes.c_int),
                ("max_depth", ctypes.c_int), ("m2l_path", ctypes.c_int),
                ("interaction", ctypes.c_int), ("p2p_tile", ctypes.c_int),
                ("mac_theta", ctypes.c_double), ("m2l_tile", ctypes.c_int),
                ("wx_direct", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


def library():
    """Load libfmm.so (raises FMMError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FMMError(2, "libfmm.so is not built; run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        L.fmm_plan_create.argtypes = [_vp, _i64, _int, _int, ctypes.POINTER(Options), _vp,
                                      ctypes.POINTER(_vp)]
        L.fmm_plan_create_batch.argtypes = [_vp, ctypes.POINTER(_i64), _int, _int, _int,
                                            ctypes.POINTER(Options), _vp, ctypes.POINTER(_vp)]
        L.fmm_plan_rebuild.argtypes = [_vp, _vp, _i64, _vp]
        L.fmm_plan_set_points.argtypes = [_vp, _vp, _vp]
        L.fmm_eval.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.fmm_helmholtz_eval.argtypes = [_vp, ctypes.c_double, _int, _vp, _vp, _vp]
        L.fmm_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.fmm_eval_graph.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.fmm_sync.argtypes = [_vp, _vp]
        L.fmm_solve_host.argtypes = [_vp, _vp, _vp, _i64, _vp, _vp, _vp]
        L.fmm_solve_adjoint_host.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]
        L.fmm_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), _vp]
        L.fmm_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double), _vp]
        L.fmm_plan_tiles.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)]
        L.fmm_plan_sizes.argtypes = [_vp, ctypes.POINTER(_i64)]
        L.fmm_plan_export.argtypes = [_vp, _int, _vp, ctypes.c_size_t]
        L.fmm_plan_destroy.argtypes = [_vp]
        L.fmm_direct.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _vp, _vp]
        L.fmm_laplace7_apply.argtypes = [_vp, _vp, _i64, ctypes.c_double, _vp]
        L.fmm_helmholtz7_apply.argtypes = [_vp, _vp, _i64, ctypes.c_double, ctypes.c_double, _vp]
        L.fmm_wait_selftest.argtypes = [_int, ctypes.c_longlong, _vp]
        L.fmm_status_string.argtypes = [_int]
        L.fmm_status_string.restype = ctypes.c_char_p
        L.fmm_last_error_message.restype = ctypes.c_char_p
        for f in EXPORTS:
            if f not in ("fmm_status_string", "fmm_last_error_message"):
                getattr(L, f).restype = _int
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        msg = library().fmm_last_error_message().decode(errors="replace")
        raise FMMError(status, msg)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _dev_f64(t, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t.contiguous()


class Plan:
    """Tree, interaction lists and workspace of one FMM problem (fmm_plan_t).

    ``points``: (N, 3) float64 CUDA tensor.  ``order`` is the largest harmonic
    degree p; ``precision`` is "fp64" or "mixed"; ``leaf_size`` 0 autotunes.
    ``offsets`` (sequence of B+1 ints) makes a batch of B independent problems
    over the concatenated points (fmm_plan_create_batch).  ``interaction`` is
    "lists" (U/V/W/X) or "dual" (dual-tree walk with acceptance criterion
    r_T + r_S < theta |c_T - c_S|; ``theta`` 0 = default 0.5).  ``p2p_tile``
    picks the staging shape of the FP32 near-field kernel, ``m2l_tile`` the
    operand form of the tensor-core M2L (1 TF32, 2 FP16; 0 = default).
    ``wx_direct`` evaluates W/X pairs of two leaves whose W leaf holds at most
    (order+1)^2 points by the direct sum (both leaves join each other's U list).
    """

    def __init__(self, points, leaf_size=64, order=8, precision="fp64", coarse_fp64_levels=0,
                 max_depth=0, stream=None, offsets=None, m2l_path="auto", interaction="lists",
                 theta=0.0, p2p_tile=0, m2l_tile=0, wx_direct=False):
        L = library()
        self.device = points.device
        self.n = int(points.shape[0])
        pts = _dev_f64(points, (self.n, 3), "points")
        opts = Options()
        opts.precision = {"fp64": FMM_FP64, "mixed": FMM_MIXED}[precision]
        opts.coarse_fp64_levels = coarse_fp64_levels
        opts.max_depth = max_depth
        opts.m2l_path = {"auto": 0, "simt": 1, "tensor": 2, "rotation": 3}[m2l_path]
        opts.interaction = {"lists": 0, "dual": 1}[interaction]
        opts.mac_theta = float(theta)
        opts.p2p_tile = int(p2p_tile)
        opts.m2l_tile = int(m2l_tile)
        opts.wx_direct = int(bool(wx_direct))
        self.interaction = interaction
        self.precision, self.order, self.leaf_size = precision, order, leaf_size
        h = _vp()
        self.nproblems = 1 if offsets is None else len(offsets) - 1
        with torch.cuda.device(self.device):
            if offsets is None:
                _check(L.fmm_plan_create(_ptr(pts), self.n, leaf_size, order, ctypes.byref(opts),
                                         _stream(stream), ctypes.byref(h)))
            else:
                off = (_i64 * len(offsets))(*[int(v) for v in offsets])
                if off[len(offsets) - 1] != self.n:
                    raise ValueError("offsets[-1] must equal the number of points")
                _check(L.fmm_plan_create_batch(_ptr(pts), off, self.nproblems, leaf_size, order,
                                               ctypes.byref(opts), _stream(stream),
                                               ctypes.byref(h)))
        self._h = h

    # -------------------------------------------------------------- life
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(library().fmm_plan_destroy(self._h))
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rebuild(self, points, stream=None):
        self.n = int(points.shape[0])
        pts = _dev_f64(points, (self.n, 3), "points")
        with torch.cuda.device(self.device):
            _check(library().fmm_plan_rebuild(self._h, _ptr(pts), self.n, _stream(stream)))

    def set_points(self, points, stream=None):
        pts = _dev_f64(points, (self.n, 3), "points")
        with torch.cuda.device(self.device):
            _check(library().fmm_plan_set_points(self._h, _ptr(pts), _stream(stream)))

    # -------------------------------------------------------------- math
    def eval(self, q, grad=True, out=None, stream=None):
        """phi = A~ q (and grad phi).  Returns (phi, grad or None)."""
        q = _dev_f64(q, (self.n,), "q")
        if out is None:
            phi = torch.empty(self.n, dtype=torch.float64, device=self.device)
            g = torch.empty(self.n, 3, dtype=torch.float64, device=self.device) if grad else None
        else:
            phi, g = out
        with torch.cuda.device(self.device):
            _check(library().fmm_eval(self._h, _ptr(q), _ptr(phi), _ptr(g), _stream(stream)))
        return phi, g

    __call__ = eval

    def helmholtz(self, q, kappa, order=8, out=None, stream=None):
        """phi_i = sum_j q_j e^{i kappa r_ij} / r_ij by the low-frequency FMM of
        ``order`` on this plan's tree (``fmm_helmholtz_eval``).  ``q``: (N,)
        complex128 CUDA tensor; returns (N,) complex128."""
        if not isinstance(q, torch.Tensor) or not q.is_cuda or q.dtype != torch.complex128:
            raise TypeError("q must be a CUDA complex128 tensor")
        if tuple(q.shape) != (self.n,):
            raise ValueError("q must have shape (%d,)" % self.n)
        q = q.contiguous()
        phi = torch.empty(self.n, dtype=torch.complex128, device=self.device) if out is None else out
        with torch.cuda.device(self.device):
            _check(library().fmm_helmholtz_eval(self._h, float(kappa), int(order), _ptr(q),
                                                _ptr(phi), _stream(stream)))
        return phi

    def adjoint(self, w, q, grad_q=None, want_dx=True, out=None, stream=None):
        """dL/dq and dL/dx for L = sum w_i phi_i (frozen plan).  ``out``:
        optional (dq, dx) tensors to write into."""
        w = _dev_f64(w, (self.n,), "w")
        q = _dev_f64(q, (self.n,), "q")
        if grad_q is not None:
            grad_q = _dev_f64(grad_q, (self.n, 3), "grad_q")
        if out is not None:
            dq, dx = out
        else:
            dq = torch.empty(self.n, dtype=torch.float64, device=self.device)
            dx = torch.empty(self.n, 3, dtype=torch.float64, device=self.device) if want_dx else None
        with torch.cuda.device(self.device):
            _check(library().fmm_adjoint(self._h, _ptr(w), _ptr(q), _ptr(grad_q), _ptr(dq),
                                         _ptr(dx), _stream(stream)))
        return dq, dx

    def eval_graph(self, q, phi, grad, w=None, dq=None, dx=None, stream=None):
        """fmm_eval (+ fmm_adjoint when w is given) replayed as one CUDA graph
        on a non-default stream; outputs are written into the given tensors."""
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.device(self.device):
            _check(library().fmm_eval_graph(self._h, _ptr(q), _ptr(phi), _ptr(grad), _ptr(w),
                                            _ptr(dq), _ptr(dx), _vp(s.cuda_stream)))

    def sync(self, stream=None):
        """Synchronise the stream; raises FMMError(FMM_ERR_TIMEOUT) if a
        bounded device-side wait of this plan gave up since the last call."""
        with torch.cuda.device(self.device):
            _check(library().fmm_sync(self._h, _stream(stream)))

    def solve_host(self, xyz, q, grad=True, stream=None):
        """End to end on host arrays: H2D, rebuild, eval, D2H (fmm_solve_host)."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = len(q)
        phi = np.empty(n)
        g = np.empty((n, 3)) if grad else None
        with torch.cuda.device(self.device):
            _check(library().fmm_solve_host(self._h, _vp(xyz.ctypes.data), _vp(q.ctypes.data), n,
                                            _vp(phi.ctypes.data),
                                            None if g is None else _vp(g.ctypes.data),
                                            _stream(stream)))
        self.n = n
        return phi, g

    def solve_adjoint_host_ptr(self, xyz_ptr, q_ptr, w_ptr, n, phi_ptr, grad_ptr, dq_ptr, dx_ptr,
                               stream=None):
        """fmm_solve_adjoint_host on raw host pointers: rebuild, forward and
        adjoint (stored forward gradient) with the copies both ways."""
        with torch.cuda.device(self.device):
            _check(library().fmm_solve_adjoint_host(self._h, _vp(xyz_ptr), _vp(q_ptr), _vp(w_ptr), n,
                                                    _vp(phi_ptr), _vp(grad_ptr), _vp(dq_ptr),
                                                    _vp(dx_ptr), _stream(stream)))
        self.n = n

    def solve_host_ptr(self, xyz_ptr, q_ptr, n, phi_ptr, grad_ptr, stream=None):
        """fmm_solve_host on raw host pointers (e.g. pinned torch tensors)."""
        with torch.cuda.device(self.device):
            _check(library().fmm_solve_host(self._h, _vp(xyz_ptr), _vp(q_ptr), n, _vp(phi_ptr),
                                            _vp(grad_ptr) if grad_ptr else None, _stream(stream)))
        self.n = n

    # ------------------------------------------------------------ layout
    def sizes(self):
        s = (_i64 * 10)()
        _check(library().fmm_plan_sizes(self._h, s))
        keys = ("n", "nboxes", "nlevels", "nu", "nv", "nw", "nx", "order", "leaf_size", "precision")
        return dict(zip(keys, [int(v) for v in s]))

    def tiles(self):
        """(p2p_tile, m2l_tile) this plan evaluates with (fmm_plan_tiles)."""
        a, b = _int(), _int()
        _check(library().fmm_plan_tiles(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"p2p_tile": a.value, "m2l_tile": b.value}

    def export(self):
        """All plan arrays as numpy arrays (see fmm_plan_export)."""
        sz = self.sizes()
        n, nb, nl = sz["n"], sz["nboxes"], sz["nlevels"]
        nb1 = nb + 1 if nb else 0
        spec = [(np.uint64, n), (np.int32, n), (np.int32, nl + 1), (np.uint64, nb)] + \
               [(np.int32, nb)] * 6 + \
               [(np.int32, nb1), (np.int32, sz["nu"]), (np.int32, nb1), (np.int32, sz["nv"]),
                (np.int32, nb1), (np.int32, sz["nw"]), (np.int32, nb1), (np.int32, sz["nx"]),
                (np.float64, 4 * self.nproblems), (np.int64, self.nproblems + 1),
                (np.float64, nb if self.interaction == "dual" else 0)]
        out = {}
        for i, (name, (dt, cnt)) in enumerate(zip(EXPORT_FIELDS, spec)):
            a = np.zeros(cnt, dtype=dt)
            _check(library().fmm_plan_export(self._h, i, _vp(a.ctypes.data) if cnt else None,
                                             a.nbytes))
            out[name] = a
        return out


class FMMFunction(torch.autograd.Function):
    """phi = FMM(points, q) with a hand-written adjoint (frozen plan).

    backward gives dL/dq = A~ g_phi (the FMM operator is symmetric) and
    dL/dx_k = g_k grad phi^q_k + q_k grad phi^g_k.
    """

    @staticmethod
    def forward(ctx, points, q, plan):
        phi, g = plan.eval(q, grad=True)
        ctx.plan = plan
        ctx.save_for_backward(q, g)
        return phi

    @staticmethod
    def backward(ctx, gphi):
        q, g = ctx.saved_tensors
        need_x = ctx.needs_input_grad[0]
        dq, dx = ctx.plan.adjoint(gphi.contiguous(), q, grad_q=g, want_dx=need_x)
        return dx, dq, None


def evaluate(points, q, leaf_size=64, order=8, precision="fp64"):
    """One-shot plan + eval.  Returns (phi, grad)."""
    plan = Plan(points, leaf_size=leaf_size, order=order, precision=precision)
    try:
        return plan.eval(q)
    finally:
        plan.close()


def direct(points, q, targets, grad=True, stream=None):
    """Brute-force potential and gradient at ``targets`` (M, 3) of the charges
    ``q`` (N,) at ``points`` (N, 3): the plain definition the FMM approximates,
    evaluated on the GPU in FP64 (``fmm_direct``).  Returns (phi, grad)."""
    if not isinstance(points, torch.Tensor) or points.dim() != 2:
        raise TypeError("points must be an (N, 3) CUDA float64 tensor")
    n, m = points.shape[0], targets.shape[0] if isinstance(targets, torch.Tensor) else -1
    pts = _dev_f64(points, (n, 3), "points")
    qq = _dev_f64(q, (n,), "q")
    tgt = _dev_f64(targets, (m, 3), "targets")
    phi = torch.empty(m, dtype=torch.float64, device=tgt.device)
    g = torch.empty(m, 3, dtype=torch.float64, device=tgt.device) if grad else None
    with torch.cuda.device(tgt.device):
        _check(library().fmm_direct(_ptr(pts), _ptr(qq), n, _ptr(tgt), m, _ptr(phi), _ptr(g),
                                    _stream(stream)))
    return phi, g


def fp32_peak(stream=None):
    """Measured FP32 rate of the current device in TFLOP/s (fmm_fp32_peak)."""
    v = ctypes.c_double()
    _check(library().fmm_fp32_peak(ctypes.byref(v), _stream(stream)))
    return v.value


def fp64_peak(stream=None):
    """Measured FP64 rate of the current device in TFLOP/s (fmm_fp64_peak)."""
    v = ctypes.c_double()
    _check(library().fmm_fp64_peak(ctypes.byref(v), _stream(stream)))
    return v.value


def laplace7(u, h, out=None, stream=None):
    """The 7-point Laplacian with zero Dirichlet boundary values applied to the
    interior grid function ``u`` (CUDA float64, shape (m, m, m) indexed [k, j, i]
    or flat m^3) with spacing ``h`` (``fmm_laplace7_apply``)."""
    if not isinstance(u, torch.Tensor) or not u.is_cuda or u.dtype != torch.float64:
        raise TypeError("u must be a CUDA float64 tensor")
    m = round(u.numel() ** (1.0 / 3.0))
    if m ** 3 != u.numel():
        raise ValueError("u must hold m^3 values")
    u = u.contiguous()
    out = torch.empty_like(u) if out is None else out
    with torch.cuda.device(u.device):
        _check(library().fmm_laplace7_apply(_ptr(u), _ptr(out), m, float(h), _stream(stream)))
    return out


def helmholtz7(u, h, kappa, out=None, stream=None):
    """(7-point Laplacian - kappa^2) u with zero Dirichlet boundary values, as
    ``laplace7`` (``fmm_helmholtz7_apply``)."""
    if not isinstance(u, torch.Tensor) or not u.is_cuda or u.dtype != torch.float64:
        raise TypeError("u must be a CUDA float64 tensor")
    m = round(u.numel() ** (1.0 / 3.0))
    if m ** 3 != u.numel():
        raise ValueError("u must hold m^3 values")
    u = u.contiguous()
    out = torch.empty_like(u) if out is None else out
    with torch.cuda.device(u.device):
        _check(library().fmm_helmholtz7_apply(_ptr(u), _ptr(out), m, float(h), float(kappa),
                                              _stream(stream)))
    return out
