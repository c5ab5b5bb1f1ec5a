"""GB300 incoherent harmonic sum (simple and greedy forms of arXiv:2202.12817).

A thin Python binding over the C ABI of ``libhs.so`` (``include/hs.h``): it marshals torch
tensors (device memory) and CUDA streams into plain pointers.  Every step of the harmonic
sum runs in the library's CUDA kernels; there is no Python or CPU fallback -- importing
this package without a built ``libhs.so`` raises.

    plan = Plan(H=32, forms=SIMPLE | GREEDY, lengths=[N])
    out = plan.forward(x, norms)             # dict of torch tensors per form
    snr = HarmonicSum.apply(p, w, plan, GREEDY, mu, sigma)   # differentiable in p and w
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = ["Plan", "FormIO", "Tuning", "HarmonicSum", "HSError", "run", "run_host", "run_fixed_scratch", "run_optimal", "backward",
           "norm_exponential", "OPTIMAL",
           "check_device_error", "selftest_timeout", "decode_argmax", "status_string", "SIMPLE", "GREEDY", "F32", "F16", "BF16",
           "FLAG_NO_MITIGATION", "FLAG_PER_SPECTRUM_NORM", "FLAG_WHITENING", "FLAG_AUTOTUNE", "FLAG_GRAPH",
           "FLAG_NO_DEVICE", "FLAG_CHECKED", "FLAG_TRUNCATE_TAIL", "lib", "LIB_PATH"]

SIMPLE, GREEDY, OPTIMAL = 1, 2, 4
F32, F16, BF16 = 0, 1, 2
FLAG_NO_MITIGATION = 1 << 0
FLAG_PER_SPECTRUM_NORM = 1 << 1
FLAG_WHITENING = 1 << 2
FLAG_AUTOTUNE = 1 << 3
FLAG_GRAPH = 1 << 4
FLAG_NO_DEVICE = 1 << 5
FLAG_CHECKED = 1 << 6
FLAG_TRUNCATE_TAIL = 1 << 7

STATUS = {0: "HS_OK", 1: "HS_ERR_INVALID_ARG", 2: "HS_ERR_UNSUPPORTED", 3: "HS_ERR_OOM", 4: "HS_ERR_CUDA",
          5: "HS_ERR_DEVICE_BOUNDS", 6: "HS_ERR_DEVICE_TIMEOUT", 7: "HS_ERR_NO_DEVICE"}

LIB_PATH = _build.LIB


class HSError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)}"
        if status == 4 and _lib is not None:
            msg += f" ({_lib.hs_last_cuda_error().decode()})"
        super().__init__(msg)


# ---------------------------------------------------------------------------------------------
# ctypes mirror of hs.h
# ---------------------------------------------------------------------------------------------
class _Desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("H", ctypes.c_int32), ("forms", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("num_spectra", ctypes.c_int64),
                ("lengths", ctypes.POINTER(ctypes.c_int64)), ("offsets", ctypes.POINTER(ctypes.c_int64)),
                ("n_freq", ctypes.c_int64), ("n_rows", ctypes.c_int64), ("z0_row", ctypes.c_int64),
                ("flags", ctypes.c_uint32)]


class _FormIO(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("snr", ctypes.c_void_p),
                ("best_h", ctypes.c_void_p), ("path", ctypes.c_void_p), ("argmax", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("threads", ctypes.c_int32), ("fund_per_thread", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("dynamic", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("stage_kb", ctypes.c_int32), ("prefetch", ctypes.c_int32), ("producers", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_V, _I32, _I64, _P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)


def lib():
    """Load libhs.so (built in-tree by ``__graft_entry__.build()`` / ``_build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhs.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.hs_plan_create.argtypes = [ctypes.POINTER(_V), ctypes.POINTER(_Desc), ctypes.c_int]
        L.hs_plan_destroy.argtypes = [_V]
        L.hs_plan_fundamentals.argtypes = [_V, _P, _P]
        L.hs_plan_input_offsets.argtypes = [_V, _P]
        L.hs_plan_domain_2d.argtypes = [_V, _P, _P, _P, _P]
        L.hs_plan_workspace.argtypes = [_V, ctypes.POINTER(ctypes.c_size_t)]
        L.hs_plan_get_tuning.argtypes = [_V, ctypes.POINTER(Tuning)]
        L.hs_plan_set_tuning.argtypes = [_V, ctypes.POINTER(Tuning)]
        L.hs_run.argtypes = [_V, _V, _V, ctypes.POINTER(_FormIO), ctypes.POINTER(_FormIO), _V, _V]
        L.hs_backward.argtypes = [_V, _I32, _V, ctypes.POINTER(_FormIO), _V, _V, _V, _V, _V, _V]
        L.hs_run_fixed_scratch.argtypes = [_V, _V, _V, ctypes.POINTER(_FormIO), ctypes.POINTER(_FormIO), _V]
        L.hs_plan_set_host_chunks.argtypes = [_V, _I32]
        L.hs_run_host.argtypes = [_V, _V, _V, _V, ctypes.POINTER(_FormIO), ctypes.POINTER(_FormIO),
                                  ctypes.POINTER(_FormIO), ctypes.POINTER(_FormIO), _V, _V]
        L.hs_run_optimal.argtypes = [_V, _V, _V, ctypes.POINTER(_FormIO), _V]
        L.hs_check_device_error.argtypes = [_V, _V]
        L.hs_selftest_timeout.argtypes = [_V, ctypes.c_uint32, _V]
        L.hs_norm_exponential.argtypes = [_I32, _I32, _I32, _I32, ctypes.c_double, _V, _V]
        L.hs_status_string.argtypes = [ctypes.c_int]
        L.hs_status_string.restype = ctypes.c_char_p
        L.hs_last_cuda_error.restype = ctypes.c_char_p
        L.hs_version.restype = ctypes.c_char_p
        for name in ("hs_plan_create", "hs_plan_destroy", "hs_plan_fundamentals", "hs_plan_input_offsets",
                     "hs_plan_domain_2d", "hs_plan_workspace", "hs_plan_get_tuning", "hs_plan_set_tuning",
                     "hs_run", "hs_backward", "hs_check_device_error", "hs_norm_exponential",
                     "hs_run_fixed_scratch", "hs_run_optimal"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().hs_status_string(int(s)).decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise HSError(rc, what)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------------------------
# per-form I/O
# ---------------------------------------------------------------------------------------------
@dataclass
class FormIO:
    """Device tensors of one form: mu/sigma [H] (or [B,H]); snr/best_h [F]; path [F] or None;
    argmax [B] (int64 storage of the uint64 key) or None."""
    mu: object
    sigma: object
    snr: object
    best_h: object
    path: object = None
    argmax: object = None

    def _c(self):
        return _FormIO(_ptr(self.mu), _ptr(self.sigma), _ptr(self.snr), _ptr(self.best_h), _ptr(self.path),
                       _ptr(self.argmax))


def norm_exponential(form: int, dims: int, H: int, mitigation: bool = True, mean1: float = 1.0):
    """Closed-form float32 (mu[H], sigma[H]) for i.i.d. exponential noise of mean ``mean1``."""
    mu = np.zeros(H, np.float32)
    sg = np.zeros(H, np.float32)
    _check(lib().hs_norm_exponential(form, dims, H, int(bool(mitigation)), float(mean1),
                                     mu.ctypes.data_as(_V), sg.ctypes.data_as(_V)), "hs_norm_exponential")
    return mu, sg


def decode_argmax(key):
    """uint64 key (as numpy/int) -> (snr float32, n)."""
    k = int(np.uint64(np.int64(key).astype(np.uint64))) if not isinstance(key, int) else key & (2 ** 64 - 1)
    hi = (k >> 32) & 0xFFFFFFFF
    lo = k & 0xFFFFFFFF
    u = (hi & 0x7FFFFFFF) if hi & 0x80000000 else (~hi & 0xFFFFFFFF)
    snr = np.frombuffer(np.uint32(u).tobytes(), np.float32)[0]
    return float(snr), 0xFFFFFFFF - lo


# ---------------------------------------------------------------------------------------------
# plan
# ---------------------------------------------------------------------------------------------
class Plan:
    """Owns an ``hs_plan``.  1D: ``Plan(H, forms, lengths=[...], dtype=F32, offsets=None)``.
    2D: ``Plan(H, GREEDY, dims=2, n_freq=..., n_rows=..., z0_row=...)``."""

    def __init__(self, H: int, forms: int = SIMPLE | GREEDY, lengths=None, dtype: int = F32, offsets=None,
                 flags: int = 0, device: int = 0, dims: int = 1, n_freq: int = 0, n_rows: int = 0,
                 z0_row: int = 0):
        L = lib()
        self.dims, self.H, self.forms, self.dtype, self.flags, self.device = dims, H, forms, dtype, flags, device
        if dims == 1:
            self._lengths = np.ascontiguousarray(lengths, dtype=np.int64)
            B = int(self._lengths.shape[0])
        else:
            self._lengths = None
            B = 1
        self._offsets = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
        d = _Desc(dims, H, forms, dtype, B,
                  self._lengths.ctypes.data_as(_P) if self._lengths is not None else None,
                  self._offsets.ctypes.data_as(_P) if self._offsets is not None else None,
                  n_freq, n_rows, z0_row, flags)
        h = _V()
        _check(L.hs_plan_create(ctypes.byref(h), ctypes.byref(d), device), "hs_plan_create")
        self._h = h
        self.B = B
        self.counts = np.zeros(B, np.int64)
        self.fund_offsets = np.zeros(B + 1, np.int64)
        _check(L.hs_plan_fundamentals(h, self.counts.ctypes.data_as(_P), self.fund_offsets.ctypes.data_as(_P)),
               "hs_plan_fundamentals")
        self.input_offsets = np.zeros(B + 1, np.int64)
        _check(L.hs_plan_input_offsets(h, self.input_offsets.ctypes.data_as(_P)), "hs_plan_input_offsets")
        ws = ctypes.c_size_t()
        _check(L.hs_plan_workspace(h, ctypes.byref(ws)), "hs_plan_workspace")
        self.workspace_bytes = int(ws.value)
        self.domain = None
        if dims == 2:
            v = [ctypes.c_int64() for _ in range(4)]
            _check(L.hs_plan_domain_2d(h, *[ctypes.byref(x) for x in v]), "hs_plan_domain_2d")
            self.domain = tuple(int(x.value) for x in v)
        self._ws = None

    # -- properties -------------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    @property
    def total_fundamentals(self) -> int:
        return int(self.fund_offsets[-1])

    @property
    def extent(self) -> int:
        return int(self.input_offsets[-1])

    @property
    def path_bytes(self) -> int:
        if self.dims == 2:
            return 4
        return 1 if self.H <= 8 else (2 if self.H <= 16 else 4)

    def path_dtype(self):
        import torch
        return {1: torch.uint8, 2: torch.int16, 4: torch.int32}[self.path_bytes]

    @property
    def tuning(self) -> Tuning:
        t = Tuning()
        _check(lib().hs_plan_get_tuning(self._h, ctypes.byref(t)), "hs_plan_get_tuning")
        return t

    @tuning.setter
    def tuning(self, t):
        if isinstance(t, dict):
            t = Tuning(**{"fund_per_thread": 1, "ctas_per_sm": 0, "dynamic": 0, "stages": 0, "stage_kb": 0,
                          "prefetch": 0, "producers": 0, **t})
        _check(lib().hs_plan_set_tuning(self._h, ctypes.byref(t)), "hs_plan_set_tuning")

    def workspace(self, device=None):
        """A cached device workspace of ``workspace_bytes`` (None when 0)."""
        if self.workspace_bytes == 0:
            return None
        if self._ws is None:
            import torch
            self._ws = torch.zeros(self.workspace_bytes, dtype=torch.uint8,
                                   device=device or torch.device("cuda", self.device))
        return self._ws

    # -- lifetime -------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().hs_plan_destroy(self._h)
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

    # -- convenience: allocate outputs with torch and run ---------------------------------------
    def alloc_form(self, mu, sigma, path=True, argmax=True):
        import torch
        dev = mu.device
        F = self.total_fundamentals
        return FormIO(mu, sigma, torch.empty(F, dtype=torch.float32, device=dev),
                      torch.empty(F, dtype=torch.uint8, device=dev),
                      torch.empty(F, dtype=self.path_dtype(), device=dev) if path else None,
                      torch.empty(self.B, dtype=torch.int64, device=dev) if argmax else None)

    @property
    def host_chunks(self) -> int:
        return getattr(self, "_host_chunks", 0)

    @host_chunks.setter
    def host_chunks(self, k: int):
        """Chunks of ``run_host``'s pipeline (0: about 16 MiB of input per chunk)."""
        _check(lib().hs_plan_set_host_chunks(self._h, int(k)), "hs_plan_set_host_chunks")
        self._host_chunks = int(k)

    def alloc_form_host(self, path=True, argmax=True):
        """Pinned host buffers for the outputs of one form (for ``run_host``): snr, best_h, path, argmax."""
        import torch
        F = self.total_fundamentals
        return FormIO(None, None, torch.empty(F, dtype=torch.float32).pin_memory(),
                      torch.empty(F, dtype=torch.uint8).pin_memory(),
                      torch.empty(F, dtype=self.path_dtype()).pin_memory() if path else None,
                      torch.empty(self.B, dtype=torch.int64).pin_memory() if argmax else None)

    def forward(self, spectra, simple_norm=None, greedy_norm=None, w=None, path=True, argmax=True, stream=None,
                optimal_norm=None):
        """Run the planned forms; ``*_norm`` = (mu, sigma) device tensors.  Returns {form: FormIO}."""
        s = self.alloc_form(*simple_norm, path=False, argmax=argmax) if self.forms & SIMPLE else None
        g = self.alloc_form(*greedy_norm, path=path, argmax=argmax) if self.forms & GREEDY else None
        if s is not None or g is not None:
            run(self, spectra, w, s, g, stream=stream)
        out = {}
        if self.forms & OPTIMAL:
            out[OPTIMAL] = self.alloc_form(*optimal_norm, path=path, argmax=argmax)
            run_optimal(self, spectra, w, out[OPTIMAL], stream=stream)
        if s is not None:
            out[SIMPLE] = s
        if g is not None:
            out[GREEDY] = g
        return out


def run(plan: Plan, spectra, w=None, simple: FormIO | None = None, greedy: FormIO | None = None, workspace=None,
        stream=None):
    """hs_run: enqueue the forward pass on ``stream`` (default: torch's current stream)."""
    ws = workspace if workspace is not None else plan.workspace(spectra.device)
    cs = simple._c() if simple is not None else None
    cg = greedy._c() if greedy is not None else None
    _check(lib().hs_run(plan.handle, _ptr(spectra), _ptr(w), ctypes.byref(cs) if cs else None,
                        ctypes.byref(cg) if cg else None, _ptr(ws), _stream_ptr(stream)), "hs_run")


def run_host(plan: Plan, host_spectra, spectra, w=None, simple: FormIO | None = None, greedy: FormIO | None = None,
             host_simple: FormIO | None = None, host_greedy: FormIO | None = None, workspace=None, stream=None):
    """hs_run_host: copy ``host_spectra`` (pinned CPU tensor in the plan's layout) into the device
    tensor ``spectra`` chunk by chunk while the chunks already copied run; optional pinned host
    copies of the outputs (``plan.alloc_form_host``) come back chunk by chunk.  Ordered on
    ``stream`` (default: torch's current stream)."""
    ws = workspace if workspace is not None else plan.workspace(spectra.device)
    cs = simple._c() if simple is not None else None
    cg = greedy._c() if greedy is not None else None
    hs_ = host_simple._c() if host_simple is not None else None
    hg = host_greedy._c() if host_greedy is not None else None
    _check(lib().hs_run_host(plan.handle, _ptr(host_spectra), _ptr(spectra), _ptr(w),
                             ctypes.byref(cs) if cs else None, ctypes.byref(cg) if cg else None,
                             ctypes.byref(hs_) if hs_ else None, ctypes.byref(hg) if hg else None,
                             _ptr(ws), _stream_ptr(stream)), "hs_run_host")


def run_fixed_scratch(plan: Plan, spectra, w=None, simple: FormIO | None = None, greedy: FormIO | None = None,
                      stream=None):
    """hs_run_fixed_scratch: the forward without a workspace, for callers that cannot allocate
    device memory; its scratch is a fixed array inside the library shared by every call, so calls
    that overlap on the GPU must be serialised by the caller."""
    cs = simple._c() if simple is not None else None
    cg = greedy._c() if greedy is not None else None
    _check(lib().hs_run_fixed_scratch(plan.handle, _ptr(spectra), _ptr(w), ctypes.byref(cs) if cs else None,
                                      ctypes.byref(cg) if cg else None, _stream_ptr(stream)), "hs_run_fixed_scratch")


def run_optimal(plan: Plan, spectra, w=None, io: FormIO | None = None, stream=None):
    """hs_run_optimal: the optimal form (DP over drift paths) of a plan with OPTIMAL."""
    c = io._c()
    _check(lib().hs_run_optimal(plan.handle, _ptr(spectra), _ptr(w), ctypes.byref(c), _stream_ptr(stream)),
           "hs_run_optimal")


def backward(plan: Plan, form: int, grad_snr, fwd: FormIO, spectra=None, w=None, grad_in=None, grad_w=None,
             workspace=None, stream=None, mark_blocks=True):
    """hs_backward: dL/d(spectra) into ``grad_in`` and/or dL/dw into ``grad_w``.  With the plan's
    workspace (the default) the library first marks the bin blocks that receive contributions and
    skips the rest; ``mark_blocks=False`` passes no workspace where none is required (every block
    is then visited; results are identical)."""
    c = fwd._c()
    out = grad_w if grad_w is not None else grad_in
    if workspace is None and out is not None and (mark_blocks or grad_w is not None):
        workspace = plan.workspace(out.device)
    _check(lib().hs_backward(plan.handle, form, _ptr(grad_snr), ctypes.byref(c), _ptr(spectra), _ptr(w),
                             _ptr(grad_in), _ptr(grad_w), _ptr(workspace), _stream_ptr(stream)), "hs_backward")


def check_device_error(plan: Plan, stream=None):
    _check(lib().hs_check_device_error(plan.handle, _stream_ptr(stream)), "device error")


def selftest_timeout(plan: Plan, limit_us: int, stream=None):
    """hs_selftest_timeout: run the bounded-wait path once (a wait that nothing completes gives up
    after ``limit_us``); ``check_device_error`` then raises with HS_ERR_DEVICE_TIMEOUT."""
    _check(lib().hs_selftest_timeout(plan.handle, int(limit_us), _stream_ptr(stream)), "hs_selftest_timeout")


# ---------------------------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------------------------
def _autograd():
    import torch

    class HarmonicSum(torch.autograd.Function):
        """snr = HS(p, w) for one form of a 1D plan.  ``w`` is the whitening vector (plan with
        FLAG_WHITENING) or None.  Backward runs the library's adjoint kernel: gradients flow to
        ``p`` (dL/dp = w dL/dx) and ``w`` (sum over spectra of p dL/dx) along the recorded
        drift paths and best h (a subgradient through the maximum over h)."""

        @staticmethod
        def forward(ctx, p, w, plan, form, mu, sigma):
            io = plan.alloc_form(mu, sigma, path=(form != SIMPLE), argmax=False)
            if form == OPTIMAL:
                run_optimal(plan, p, w, io)
            else:
                run(plan, p, w, io if form == SIMPLE else None, io if form == GREEDY else None)
            ctx.plan, ctx.form = plan, form
            ctx.io = io
            ctx.save_for_backward(p, w if w is not None else torch.empty(0, device=p.device))
            ctx.mark_non_differentiable(io.best_h)
            if io.path is not None:
                ctx.mark_non_differentiable(io.path)
                return io.snr, io.best_h, io.path
            return io.snr, io.best_h

        @staticmethod
        def backward(ctx, g_snr, *unused):
            p, w = ctx.saved_tensors
            w = w if w.numel() else None
            plan = ctx.plan
            need_p = ctx.needs_input_grad[0]
            need_w = ctx.needs_input_grad[1] and w is not None
            g_snr = g_snr.contiguous().float()
            grad_p = torch.empty(p.shape, dtype=torch.float32, device=p.device) if need_p else None
            grad_w = torch.empty(w.shape[0], dtype=torch.float32, device=p.device) if need_w else None
            if need_p and p.numel() != int(plan._lengths.sum()):
                grad_p.zero_()      # alignment padding between spectra receives no gradient
            backward(plan, ctx.form, g_snr, ctx.io, p, w, grad_p, grad_w)
            if grad_p is not None and p.dtype != torch.float32:
                grad_p = grad_p.to(p.dtype)
            return grad_p, grad_w, None, None, None, None

    return HarmonicSum


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _autograd()
        return getattr(_Lazy._cls, name)


HarmonicSum = _Lazy()

# fail loudly at import when the CUDA library is missing
lib()
