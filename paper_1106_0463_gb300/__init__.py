"""GB300-native Legendre coefficients by the Abel-transform + FFT method.

Thin Python binding of the C ABI in ``include/leg.h`` (libleg.so): argument
marshalling only -- every step of the computation runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.

Method: De Micheli & Viano, arXiv:1106.0463, Theorem 1 (Eq. 2.4, Eq. 2.5):
c_n / (2n+1) are the nonnegative-index Fourier coefficients of the Abel-type
transform of f, evaluated on an M-point periodic grid by Gauss-Legendre
quadrature after the substitution x = cos y + s^2, followed by one FFT.

The library must have been built (``python -c "import __graft_entry__ as g;
g.build()"``); the first call into it raises ImportError otherwise.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

__all__ = [
    "F64", "F32", "BF16", "SPLIT_FP16", "FLAG_TAU_LITERAL", "FLAG_COLLAPSED", "FLAG_SINE_FORM",
    "TRANSFORM_REG", "TRANSFORM_STOCKHAM", "TRANSFORM_SINE",
    "FAMILY_GENFN", "FAMILY_EXP", "FAMILY_CHEB", "FAMILY_ABSPOW",
    "Ragged", "forward_ragged", "sample_cl",
    "LegError", "Plan", "LegendreFn", "legendre", "library_path", "declared_symbols", "load_library",
    "memory_info",
]

F64, F32, BF16, SPLIT_FP16 = 0, 1, 2, 3
FLAG_TAU_LITERAL = 1
FLAG_COLLAPSED = 2    # c = L f with L = R A multiplied out at plan time (one GEMM, no transform)
FLAG_SINE_FORM = 4    # forward transform by the half-range sine form (Eq. 2.13)
TRANSFORM_REG, TRANSFORM_STOCKHAM, TRANSFORM_SINE = 0, 1, 2
FAMILY_GENFN, FAMILY_EXP, FAMILY_CHEB, FAMILY_ABSPOW = 0, 1, 2, 3
_ERR_NAMES = {1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "UNSUPPORTED", 5: "TIMEOUT"}

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libleg.so")
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "leg.h")


def library_path() -> str:
    return _LIB_PATH


def declared_symbols() -> list[str]:
    """Names of every entry point declared (LEG_API) in include/leg.h."""
    with open(_HEADER) as fh:
        text = fh.read()
    return re.findall(r"LEG_API\s+[\w\s\*]*?\b(leg_\w+)\s*\(", text)


class LegError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("LEG_ERR_%s: %s" % (_ERR_NAMES.get(code, str(code)), msg))
        self.code = code


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libleg.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
    sig = {
        "leg_plan_create": ([ctypes.POINTER(vp), i, i, i, i, i], i),
        "leg_plan_create_ex": ([ctypes.POINTER(vp), i, i, i, i, i, u], i),
        "leg_plan_create_like": ([ctypes.POINTER(vp), vp, i], i),
        "leg_plan_destroy": ([vp], i),
        "leg_plan_reserve": ([vp, i], i),
        "leg_plan_info": ([vp] + [ctypes.POINTER(i)] * 7, i),
        "leg_forward": ([vp, vp, vp, i, vp], i),
        "leg_forward_batches": ([vp, vp, vp, i, i, vp], i),
        "leg_forward_batches_profiled": ([vp, vp, vp, i, i, vp, ctypes.POINTER(ctypes.c_float)], i),
        "leg_forward_host_batches": ([vp, vp, vp, i, i, vp], i),
        "leg_forward_profiled": ([vp, vp, vp, i, vp, ctypes.POINTER(ctypes.c_float)], i),
        "leg_backward": ([vp, vp, vp, i, vp], i),
        "leg_forward_noalloc": ([vp, vp, vp, i, vp], i),
        "leg_forward_host": ([vp, vp, vp, i, vp], i),
        "leg_plain_forward": ([vp, i, vp, i, vp, vp], i),
        "leg_plain_forward_cheb": ([vp, vp, i, i, vp, vp], i),
        "leg_plan_status": ([vp, i], i),
        "leg_plan_set_wait_limit": ([vp, ctypes.c_longlong], i),
        "leg_plan_set_tile": ([vp, i], i),
        "leg_plan_set_host_overlap": ([vp, i], i),
        "leg_plan_set_transform": ([vp, i, i], i),
        "leg_plan_get_transform": ([vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "leg_plan_autotune": ([vp, vp, vp, i, vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "leg_plan_tile_info": ([vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "leg_ragged_create": ([ctypes.POINTER(vp), ctypes.POINTER(vp), i, i, vp, vp, vp, vp], i),
        "leg_ragged_forward": ([vp, vp, vp, vp], i),
        "leg_ragged_forward_profiled": ([vp, vp, vp, vp, ctypes.POINTER(ctypes.c_float)], i),
        "leg_ragged_set_tile": ([vp, i], i),
        "leg_ragged_tile_info": ([vp, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "leg_ragged_autotune": ([vp, vp, vp, vp, ctypes.POINTER(i)], i),
        "leg_forward_ragged": ([ctypes.POINTER(vp), i, i, vp, vp, vp, vp, vp, vp, vp], i),
        "leg_ragged_status": ([vp, i], i),
        "leg_ragged_destroy": ([vp], i),
        "leg_sample_cl": ([i, vp, vp, vp, vp, vp, vp, vp, vp], i),
        "leg_memory_info": ([ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], i),
        "leg_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


class _LazyLib:
    """Loads libleg.so on first use and raises ImportError if it is missing."""

    _handle = None

    def __getattr__(self, name):
        if _LazyLib._handle is None:
            _LazyLib._handle = _load()
        return getattr(_LazyLib._handle, name)


_lib = _LazyLib()


def load_library():
    """Load libleg.so now (raises ImportError when it has not been built)."""
    return _lib.leg_last_error


def memory_info() -> tuple[int, int]:
    """(live device allocations, bytes) the library holds (leg_memory_info)."""
    n, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.leg_memory_info(ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def _check(rc: int):
    if rc != 0:
        raise LegError(rc, _lib.leg_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_tensor(t: torch.Tensor, dtype: torch.dtype, shape, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _host_tensor(t: torch.Tensor, dtype: torch.dtype, shape, name: str):
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError("%s must be a CPU tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _batch_args(f, c, K: int, N: int, dtype: torch.dtype, check, suffix: str):
    """Pointers and sizes of a stack of batches: f (nbatch, B, K) and c
    (nbatch, B, N), both contiguous, checked by `check` (_dev_tensor or
    _host_tensor) as (nbatch * B, K) and (nbatch * B, N) matrices."""
    for t, name, w in ((f, "f" + suffix, K), (c, "c" + suffix, N)):
        if not isinstance(t, torch.Tensor) or t.dim() != 3:
            raise ValueError("%s must be a tensor of shape (nbatch, B, %d)" % (name, w))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    nb, B = f.shape[0], f.shape[1]
    if tuple(c.shape[:2]) != (nb, B):
        raise ValueError("c%s must have shape (%d, %d, %d)" % (suffix, nb, B, N))
    pf = check(f.view(nb * B, f.shape[2]), dtype, (nb * B, K), "f" + suffix)
    pc = check(c.view(nb * B, c.shape[2]), dtype, (nb * B, N), "c" + suffix)
    return pf, pc, nb, B


class Plan:
    """An operator for one (N, M, K, Q, dtype); owns its device buffers.

    N coefficients, M trapezoid points (power of two), K Chebyshev-Lobatto
    samples per function, Q Gauss nodes per y-point (0: exact for degree K-1).
    """

    def __init__(self, N: int, M: int, K: int, Q: int = 0, dtype: int = SPLIT_FP16, flags: int = 0,
                 like: "Plan | None" = None):
        h = ctypes.c_void_p()
        if like is not None:
            _check(_lib.leg_plan_create_like(ctypes.byref(h), like._h, dtype))
            flags = like.flags
        else:
            _check(_lib.leg_plan_create_ex(ctypes.byref(h), N, M, K, Q, dtype, flags))
        self._h = h
        vals = [ctypes.c_int() for _ in range(7)]
        _check(_lib.leg_plan_info(h, *[ctypes.byref(v) for v in vals]))
        self.N, self.M, self.K, self.Q, self.dtype, self.K_padded, self.rows = (v.value for v in vals)
        self.flags = flags

    @classmethod
    def like(cls, src: "Plan", dtype: int) -> "Plan":
        """Same sizes as src with another dtype, reusing src's operator (leg_plan_create_like)."""
        return cls(src.N, src.M, src.K, src.Q, dtype, like=src)

    @property
    def io_dtype(self) -> torch.dtype:
        return torch.float64 if self.dtype == F64 else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            _lib.leg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, B: int):
        _check(_lib.leg_plan_reserve(self._h, B))

    def status(self, reset: bool = True):
        """Raise LegError(TIMEOUT) if a bounded device wait expired (synchronises)."""
        _check(_lib.leg_plan_status(self._h, int(bool(reset))))

    def set_wait_limit(self, cycles: int):
        _check(_lib.leg_plan_set_wait_limit(self._h, int(cycles)))

    def set_tile(self, tn: int):
        """Functions per CTA-pair tile of the tensor-core GEMM (0 = automatic)."""
        _check(_lib.leg_plan_set_tile(self._h, int(tn)))

    def set_host_overlap(self, on: bool):
        """leg_plan_set_host_overlap: with on, forward_host on pinned buffers
        copies each batch's input with a copy engine ordered only after the
        previous use of its staging buffer, so that it overlaps the previous
        call's kernels; f_host must hold the batch when the call is made."""
        _check(_lib.leg_plan_set_host_overlap(self._h, 1 if on else 0))

    def set_transform(self, variant: int, radix: int = 0):
        """Kernel of the forward transform stage: TRANSFORM_REG, TRANSFORM_STOCKHAM
        or TRANSFORM_SINE, and the radix (8 or 16 values per thread; 0 = 8) of
        the register-tiled kernels (leg_plan_set_transform); same map, rounding
        differs."""
        _check(_lib.leg_plan_set_transform(self._h, int(variant), int(radix)))

    @property
    def transform(self) -> int:
        v = ctypes.c_int()
        _check(_lib.leg_plan_get_transform(self._h, ctypes.byref(v), None))
        return v.value

    @property
    def transform_radix(self) -> int:
        r = ctypes.c_int()
        _check(_lib.leg_plan_get_transform(self._h, None, ctypes.byref(r)))
        return r.value

    def autotune(self, f: torch.Tensor, c: torch.Tensor | None = None, stream=None) -> dict:
        """leg_plan_autotune: time the GEMM tile widths and the transform
        kernels on this batch and keep the fastest (synchronises)."""
        B = f.shape[0] if f.dim() == 2 else -1
        pf = _dev_tensor(f, self.io_dtype, (B, self.K), "f")
        if c is None:
            c = torch.empty((B, self.N), dtype=self.io_dtype, device=f.device)
        pc = _dev_tensor(c, self.io_dtype, (B, self.N), "c")
        tn, fft = ctypes.c_int(), ctypes.c_int()
        _check(_lib.leg_plan_autotune(self._h, pf, pc, B, _stream(stream), ctypes.byref(tn), ctypes.byref(fft)))
        return {"tn": tn.value, "fft": fft.value}

    def tile_info(self, B: int) -> dict:
        """Tile of the split forward GEMM for B functions: tn, resident pairs, tiles."""
        tn, pairs, tiles = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.leg_plan_tile_info(self._h, int(B), ctypes.byref(tn), ctypes.byref(pairs),
                                       ctypes.byref(tiles)))
        return {"tn": tn.value, "pairs": pairs.value, "tiles": tiles.value}

    def forward(self, f: torch.Tensor, c: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """c = L f for f of shape (B, K) on the device (leg_forward)."""
        B = f.shape[0] if f.dim() == 2 else -1
        pf = _dev_tensor(f, self.io_dtype, (B, self.K), "f")
        if c is None:
            c = torch.empty((B, self.N), dtype=self.io_dtype, device=f.device)
        pc = _dev_tensor(c, self.io_dtype, (B, self.N), "c")
        _check(_lib.leg_forward(self._h, pf, pc, B, _stream(stream)))
        return c

    def forward_batches(self, f: torch.Tensor, c: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """leg_forward_batches: f of shape (nbatch, B, K) on the device, c of
        shape (nbatch, B, N); the batches one after another, pipelined for
        split-FP16 plans (each batch's transform beside the next one's GEMM)."""
        if c is None and isinstance(f, torch.Tensor) and f.dim() == 3:
            c = torch.empty((f.shape[0], f.shape[1], self.N), dtype=self.io_dtype, device=f.device)
        pf, pc, nb, B = _batch_args(f, c, self.K, self.N, self.io_dtype, _dev_tensor, "")
        _check(_lib.leg_forward_batches(self._h, pf, pc, B, nb, _stream(stream)))
        return c

    def forward_batches_profiled(self, f: torch.Tensor, c: torch.Tensor, stream=None):
        """leg_forward_batches_profiled: the pipelined batches with the mean
        time per batch of each stage inside the pipeline; synchronises.
        Returns (prep_ms, gemm_ms, fft_ms)."""
        pf, pc, nb, B = _batch_args(f, c, self.K, self.N, self.io_dtype, _dev_tensor, "")
        ms = (ctypes.c_float * 3)()
        _check(_lib.leg_forward_batches_profiled(self._h, pf, pc, B, nb, _stream(stream), ms))
        return tuple(float(v) for v in ms)

    def forward_noalloc(self, f: torch.Tensor, c: torch.Tensor, stream=None) -> torch.Tensor:
        """leg_forward_noalloc: the split-FP16 forward pass for callers that
        must not allocate device memory at call time; its intermediates live in
        the library's static 64 MiB device scratch (shared by all calls on a
        device, so overlapping calls race).  c must be preallocated."""
        B = f.shape[0] if f.dim() == 2 else -1
        pf = _dev_tensor(f, torch.float32, (B, self.K), "f")
        pc = _dev_tensor(c, torch.float32, (B, self.N), "c")
        _check(_lib.leg_forward_noalloc(self._h, pf, pc, B, _stream(stream)))
        return c

    def forward_host(self, f_host: torch.Tensor, c_host: torch.Tensor | None = None, stream=None,
                     sync: bool = True) -> torch.Tensor:
        """c = L f for host tensors (leg_forward_host): the copies to and from the
        device overlap the computation.  f_host (B, K) on the CPU, ideally pinned;
        c_host (B, N) on the CPU (pinned and allocated when None).  With
        sync=False the call returns at once and c_host is complete when the
        stream has reached it."""
        B = f_host.shape[0] if f_host.dim() == 2 else -1
        pf = _host_tensor(f_host, self.io_dtype, (B, self.K), "f_host")
        if c_host is None:
            c_host = torch.empty((B, self.N), dtype=self.io_dtype).pin_memory()
        pc = _host_tensor(c_host, self.io_dtype, (B, self.N), "c_host")
        st = _stream(stream)
        _check(_lib.leg_forward_host(self._h, pf, pc, B, st))
        if sync:
            (stream or torch.cuda.current_stream()).synchronize()
        return c_host

    def forward_host_batches(self, f_host: torch.Tensor, c_host: torch.Tensor | None = None, stream=None,
                             sync: bool = True) -> torch.Tensor:
        """leg_forward_host_batches: f_host (nbatch, B, K) and c_host (nbatch, B,
        N) on the CPU, ideally pinned (c_host pinned and allocated when None);
        pipelined for split-FP16 plans.  With sync=False the call returns at
        once and c_host is complete when the stream has reached it."""
        if c_host is None and isinstance(f_host, torch.Tensor) and f_host.dim() == 3:
            c_host = torch.empty((f_host.shape[0], f_host.shape[1], self.N), dtype=self.io_dtype).pin_memory()
        pf, pc, nb, B = _batch_args(f_host, c_host, self.K, self.N, self.io_dtype, _host_tensor, "_host")
        st = _stream(stream)
        _check(_lib.leg_forward_host_batches(self._h, pf, pc, B, nb, st))
        if sync:
            (stream or torch.cuda.current_stream()).synchronize()
        return c_host

    def forward_profiled(self, f: torch.Tensor, c: torch.Tensor, stream=None):
        """Forward pass timed per stage (leg_forward_profiled); synchronises.

        Returns (prep_ms, gemm_ms, fft_ms)."""
        B = f.shape[0]
        pf = _dev_tensor(f, self.io_dtype, (B, self.K), "f")
        pc = _dev_tensor(c, self.io_dtype, (B, self.N), "c")
        ms = (ctypes.c_float * 3)()
        _check(_lib.leg_forward_profiled(self._h, pf, pc, B, _stream(stream), ms))
        return tuple(float(v) for v in ms)

    def backward(self, dc: torch.Tensor, df: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """df = L^T dc for dc of shape (B, N) (leg_backward)."""
        B = dc.shape[0] if dc.dim() == 2 else -1
        pdc = _dev_tensor(dc, self.io_dtype, (B, self.N), "dc")
        if df is None:
            df = torch.empty((B, self.K), dtype=self.io_dtype, device=dc.device)
        pdf = _dev_tensor(df, self.io_dtype, (B, self.K), "df")
        _check(_lib.leg_backward(self._h, pdc, pdf, B, _stream(stream)))
        return df

    def plain_forward(self, family: int, params: torch.Tensor, c: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
        """Plain method for closed-form families (leg_plain_forward); FP64."""
        B = params.shape[0]
        pp = _dev_tensor(params, torch.float64, (B,), "params")
        if c is None:
            c = torch.empty((B, self.N), dtype=torch.float64, device=params.device)
        pc = _dev_tensor(c, torch.float64, (B, self.N), "c")
        _check(_lib.leg_plain_forward(self._h, family, pp, B, pc, _stream(stream)))
        return c

    def plain_forward_cheb(self, coef: torch.Tensor, c: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Plain method for Chebyshev series sum_m coef[b, m] T_m(x) (leg_plain_forward_cheb); FP64."""
        if coef.dim() != 2:
            raise ValueError("coef must be B x Kc")
        B, Kc = coef.shape
        pk = _dev_tensor(coef, torch.float64, (B, Kc), "coef")
        if c is None:
            c = torch.empty((B, self.N), dtype=torch.float64, device=coef.device)
        pc = _dev_tensor(c, torch.float64, (B, self.N), "c")
        _check(_lib.leg_plain_forward_cheb(self._h, pk, Kc, B, pc, _stream(stream)))
        return c


class LegendreFn(torch.autograd.Function):
    """c = L f with the exact adjoint df = L^T dc as its backward."""

    @staticmethod
    def forward(ctx, f: torch.Tensor, plan: Plan):
        ctx.plan = plan
        return plan.forward(f.contiguous())

    @staticmethod
    def backward(ctx, dc: torch.Tensor):
        return ctx.plan.backward(dc.contiguous()), None


def legendre(f: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable Legendre coefficients of the rows of f (B x K CL samples)."""
    return LegendreFn.apply(f, plan)


class Ragged:
    """A ragged batch over size-bucket plans (leg_ragged_create / leg_ragged_forward).

    plans: list of SPLIT_FP16 Plans; plan_idx, n_out, in_off, out_off: per
    function (host sequences).  forward() reads the packed FP32 samples and
    writes the packed coefficients (device tensors)."""

    def __init__(self, plans, plan_idx, n_out, in_off, out_off):
        import numpy as np
        self.plans = list(plans)   # keep the plans alive
        pi = np.ascontiguousarray(plan_idx, dtype=np.int32)
        no = np.ascontiguousarray(n_out, dtype=np.int32)
        io = np.ascontiguousarray(in_off, dtype=np.int64)
        oo = np.ascontiguousarray(out_off, dtype=np.int64)
        self.count = int(pi.size)
        hp = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(_lib.leg_ragged_create(ctypes.byref(h), hp, len(self.plans), self.count,
                                      pi.ctypes.data_as(ctypes.c_void_p), no.ctypes.data_as(ctypes.c_void_p),
                                      io.ctypes.data_as(ctypes.c_void_p), oo.ctypes.data_as(ctypes.c_void_p)))
        self._h = h
        self.n_in = int((io + np.array([p.K for p in self.plans])[pi]).max()) if self.count else 0
        self.n_out = int((oo + no).max()) if self.count else 0

    def _io(self, f_packed, c_packed):
        for t, nm, n in ((f_packed, "f_packed", self.n_in), (c_packed, "c_packed", self.n_out)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("%s must be a contiguous float32 CUDA tensor" % nm)
            if t.numel() < n:
                raise ValueError("%s needs at least %d elements" % (nm, n))
        return ctypes.c_void_p(f_packed.data_ptr()), ctypes.c_void_p(c_packed.data_ptr())

    def forward(self, f_packed: torch.Tensor, c_packed: torch.Tensor, stream=None) -> torch.Tensor:
        pf, pc = self._io(f_packed, c_packed)
        _check(_lib.leg_ragged_forward(self._h, pf, pc, _stream(stream)))
        return c_packed

    def forward_profiled(self, f_packed: torch.Tensor, c_packed: torch.Tensor, stream=None):
        """Stage times in ms (split, grouped GEMM, transforms); synchronises."""
        pf, pc = self._io(f_packed, c_packed)
        ms = (ctypes.c_float * 3)()
        _check(_lib.leg_ragged_forward_profiled(self._h, pf, pc, _stream(stream), ms))
        return tuple(float(v) for v in ms)

    def set_tile(self, tn: int):
        """Tile width of the grouped GEMM (0 = the cost model's choice)."""
        _check(_lib.leg_ragged_set_tile(self._h, int(tn)))

    def tile_info(self) -> dict:
        tn, tiles = ctypes.c_int(), ctypes.c_int()
        _check(_lib.leg_ragged_tile_info(self._h, ctypes.byref(tn), ctypes.byref(tiles)))
        return {"tn": tn.value, "tiles": tiles.value}

    def autotune(self, f_packed: torch.Tensor, c_packed: torch.Tensor, stream=None) -> int:
        """leg_ragged_autotune: time the grouped GEMM's tile widths on this data, keep the fastest."""
        pf, pc = self._io(f_packed, c_packed)
        tn = ctypes.c_int()
        _check(_lib.leg_ragged_autotune(self._h, pf, pc, _stream(stream), ctypes.byref(tn)))
        return tn.value

    def status(self, reset: bool = True):
        _check(_lib.leg_ragged_status(self._h, int(bool(reset))))

    def close(self):
        if getattr(self, "_h", None):
            _lib.leg_ragged_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward_ragged(plans, plan_idx: torch.Tensor, n_out: torch.Tensor, in_off: torch.Tensor,
                   out_off: torch.Tensor, f_packed: torch.Tensor, c_packed: torch.Tensor, stream=None) -> torch.Tensor:
    """leg_forward_ragged: a ragged batch in one call, the per-function arrays
    given as CUDA tensors (plan_idx, n_out int32; in_off, out_off int64).  The
    library reads the arrays back and caches the batch built from them."""
    count = plan_idx.numel()
    for t, nm, dt in ((plan_idx, "plan_idx", torch.int32), (n_out, "n_out", torch.int32),
                      (in_off, "in_off", torch.int64), (out_off, "out_off", torch.int64)):
        _dev_tensor(t, dt, (count,), nm)
    for t, nm in ((f_packed, "f_packed"), (c_packed, "c_packed")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("%s must be a contiguous float32 CUDA tensor" % nm)
    plans = list(plans)
    hp = (ctypes.c_void_p * len(plans))(*[p._h.value for p in plans])
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    _check(_lib.leg_forward_ragged(hp, len(plans), count, ptr(plan_idx), ptr(n_out), ptr(in_off), ptr(out_off),
                                   ptr(f_packed), ptr(c_packed), _stream(stream)))
    return c_packed


def sample_cl(family, param, K, in_off, f_packed, coef=None, coef_off=None, stream=None):
    """leg_sample_cl: closed-form functions sampled at their CL nodes on the device.

    All arguments are CUDA tensors: family int32, param float64, K int32,
    in_off int64, f_packed float32; coef float64 and coef_off int64 for
    FAMILY_CHEB."""
    n = family.numel()

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()
    _check(_lib.leg_sample_cl(n, ptr(family), ptr(param), ptr(K), ptr(coef_off), ptr(coef), ptr(in_off),
                              ptr(f_packed), _stream(stream)))
    return f_packed
