"""Python binding of libmz (include/mz.h): fast zeta and Moebius transforms on posets.

Argument marshalling only. Every transform runs in the CUDA kernels of
libmz.so; there is no CPU or PyTorch fallback, and importing this package
fails if the library cannot be loaded (or built with nvcc).

Two layers:

* ``mz_build``, ``mz_zeta``, ``mz_mobius``, ... : one function per C entry
  point, same names and arguments (device pointers as integers, the stream
  as an integer ``cudaStream_t``). Errors raise ``MzError``.
* ``Plan``: owns a plan handle and a cached workspace, and takes PyTorch CUDA
  tensors; ``ZetaFn`` / ``MobiusFn`` are ``torch.autograd.Function``s whose
  backward passes are the transposed transforms (Z^T, M^T).

Value layouts (the C ABI's): ``[n]`` or ``[n, batch]`` contiguous tensors of
int64 (``MZ_I64``) or float64 (``MZ_F64``); ``MZ_F32C`` uses a float32 tensor
of shape ``[2, n]`` or ``[2, n, batch]`` holding the hi plane and the lo plane.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MZ_OK, MZ_ERR_INVALID_ARG, MZ_ERR_CYCLE, MZ_ERR_BAD_CHAINS, MZ_ERR_OOM, MZ_ERR_CUDA, \
    MZ_ERR_TIMEOUT, MZ_ERR_UNSUPPORTED, MZ_ERR_NO_DEVICE, MZ_ERR_BOUNDS = range(10)
MZ_I64, MZ_F64, MZ_F32C = 0, 1, 2
MZ_SCHED_ULEVEL, MZ_SCHED_ANTICHAIN = 0, 1
MZ_EXPORT_CHAIN_ID, MZ_EXPORT_CHAIN_POS, MZ_EXPORT_NIV, MZ_EXPORT_LEVEL, MZ_EXPORT_ULEVEL, MZ_EXPORT_TOPO = range(6)

# every symbol include/mz.h declares
EXPORTED = ["mz_build", "mz_build_batch", "mz_destroy", "mz_workspace_size", "mz_zeta", "mz_zeta_noalloc", "mz_mobius",
            "mz_zeta_T", "mz_mobius_T",
            "mz_check", "mz_plan_tune", "mz_plan_info", "mz_plan_export", "mz_plan_save", "mz_plan_load",
            "mz_last_launch_count", "mz_set_launch_events", "mz_status_string", "mz_last_error"]


class MzError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_status_string(status)}" + (f" ({detail})" if detail else ""))


class _Opts(ctypes.Structure):
    _fields_ = [("build_transpose", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("mobius_schedule", ctypes.c_int32), ("mobius_blocks_per_sm", ctypes.c_int32),
                ("mobius_pace_ns", ctypes.c_int32), ("niv_format", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("debug_withhold", ctypes.c_int64),
                ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p), ("alloc_ctx", ctypes.c_void_p),
                ("device_build", ctypes.c_int32)]


# Plan memory through PyTorch's caching allocator (mz_build_opts::dev_alloc / dev_free):
# the plan's buffers then show up in torch.cuda.memory_allocated and share its pool.
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def _torch_alloc(nbytes, ctx):
    """dev_alloc callback. Only an allocation failure (torch.cuda.OutOfMemoryError)
    becomes NULL, which the library reports as MZ_ERR_OOM; any other error is kept in
    _ALLOC_ERRORS and also returns NULL (an exception cannot cross the C boundary),
    and the binding re-raises it after the failed build instead of reporting OOM."""
    import torch
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes))
    except torch.cuda.OutOfMemoryError:
        return None
    except BaseException as exc:   # noqa: BLE001  (re-raised by _check_alloc_errors)
        _ALLOC_ERRORS.append(exc)
        return None


_ALLOC_ERRORS: list = []


def _check_alloc_errors():
    if _ALLOC_ERRORS:
        exc = _ALLOC_ERRORS[0]
        _ALLOC_ERRORS.clear()
        raise RuntimeError(f"device allocation callback failed: {exc!r}") from exc


def _torch_free(ptr, ctx):
    try:
        import torch
        torch.cuda.caching_allocator_delete(ptr)
    except Exception:       # interpreter shutdown: the process releases the memory
        pass


_TORCH_ALLOC = _ALLOC_T(_torch_alloc)
_TORCH_FREE = _FREE_T(_torch_free)


def _opts(build_transpose, host_only, mobius_schedule, mobius_blocks_per_sm, mobius_pace_ns, niv_format,
          spin_limit, debug_withhold, device_build, torch_allocator):
    alloc = ctypes.cast(_TORCH_ALLOC, ctypes.c_void_p).value if torch_allocator else None
    free = ctypes.cast(_TORCH_FREE, ctypes.c_void_p).value if torch_allocator else None
    return _Opts(int(build_transpose), int(host_only), int(mobius_schedule), int(mobius_blocks_per_sm),
                 int(mobius_pace_ns), int(niv_format), int(spin_limit), int(debug_withhold), alloc, free, None,
                 int(device_build))


class Tuning(ctypes.Structure):
    _fields_ = [("mobius_blocks_per_sm", ctypes.c_int32), ("mobius_pace_ns", ctypes.c_int32),
                ("gather_blocks_per_sm", ctypes.c_int32), ("mobius_lanes", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("has_transpose", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("edges", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("ulevels", ctypes.c_int32), ("schedule", ctypes.c_int32), ("levels_T", ctypes.c_int32),
                ("ulevels_T", ctypes.c_int32), ("max_chain", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("components", ctypes.c_int32), ("sparse", ctypes.c_int32), ("wave_rows", ctypes.c_int64),
                ("wave_entries", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load():
    # MZ_LIBRARY=debug loads the MZ_DEBUG build (bounds-checked kernels, poisoned
    # workspaces); MZ_LIBRARY=<path> loads another build of the same C ABI.
    which = os.environ.get("MZ_LIBRARY", "")
    if which == "debug":
        path = _build.build(debug=True)
    elif which:
        path = os.path.abspath(which)
    else:
        path = _build.build()
    lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.mz_build.argtypes = [i64, i64, vp, vp, vp, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.mz_build_batch.argtypes = [i32, vp, vp, vp, vp, vp, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.mz_destroy.argtypes = [vp]
    lib.mz_destroy.restype = None
    lib.mz_workspace_size.argtypes = [vp, ctypes.c_int, i32, ctypes.POINTER(sz)]
    for name in ("mz_zeta", "mz_mobius", "mz_zeta_T", "mz_mobius_T"):
        getattr(lib, name).argtypes = [vp, ctypes.c_int, vp, vp, i32, vp, sz, vp]
    lib.mz_zeta_noalloc.argtypes = [vp, ctypes.c_int, vp, vp, i32, vp]
    lib.mz_check.argtypes = [vp, vp]
    lib.mz_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.mz_plan_tune.argtypes = [vp, ctypes.POINTER(Tuning), ctypes.POINTER(Tuning)]
    lib.mz_plan_export.argtypes = [vp, i32, i32, vp, sz]
    lib.mz_plan_save.argtypes = [vp, ctypes.c_char_p]
    lib.mz_plan_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.mz_last_launch_count.argtypes = []
    lib.mz_last_launch_count.restype = i32
    lib.mz_set_launch_events.argtypes = [vp, i32]
    lib.mz_set_launch_events.restype = None
    lib.mz_status_string.argtypes = [ctypes.c_int]
    lib.mz_status_string.restype = ctypes.c_char_p
    lib.mz_last_error.argtypes = []
    lib.mz_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("mz_destroy", "mz_last_launch_count", "mz_set_launch_events", "mz_status_string",
                        "mz_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()
LIBRARY_PATH = lib._name


def _status_string(s: int) -> str:
    return lib.mz_status_string(int(s)).decode()


def _check(st: int, where: str):
    if st != MZ_OK:
        raise MzError(st, where, lib.mz_last_error().decode())


# ----------------------------------------------------------------------------- C entry points

def mz_build(n: int, src, dst, chain_id=None, *, build_transpose: bool = False, host_only: bool = False,
             mobius_schedule: int = MZ_SCHED_ULEVEL, spin_limit: int = 0, debug_withhold: int = 0,
             mobius_blocks_per_sm: int = 0, mobius_pace_ns: int = 0, niv_format: int = 0,
             device_build: int = 0, torch_allocator: bool = False) -> int:
    """mz_build: returns the plan handle (an integer). Host arrays are int32.
    torch_allocator: the plan's device memory (and the build's scratch) comes from
    PyTorch's caching allocator through the dev_alloc / dev_free callbacks."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    cid = None if chain_id is None else np.ascontiguousarray(chain_id, dtype=np.int32)
    opts = _opts(build_transpose, host_only, mobius_schedule, mobius_blocks_per_sm, mobius_pace_ns, niv_format,
                 spin_limit, debug_withhold, device_build, torch_allocator)
    out = ctypes.c_void_p()
    st = lib.mz_build(int(n), int(src.size), src.ctypes.data, dst.ctypes.data,
                      None if cid is None else cid.ctypes.data, ctypes.byref(opts), ctypes.byref(out))
    if st != MZ_OK:
        _check_alloc_errors()
    _check(st, "mz_build")
    return out.value


def mz_build_batch(posets, *, build_transpose: bool = False, host_only: bool = False,
                   mobius_schedule: int = MZ_SCHED_ULEVEL, spin_limit: int = 0, debug_withhold: int = 0,
                   mobius_blocks_per_sm: int = 0, mobius_pace_ns: int = 0, niv_format: int = 0,
                   device_build: int = 0, torch_allocator: bool = False) -> int:
    """mz_build_batch: `posets` is a list of (n, src, dst, chain_id or None)."""
    count = len(posets)
    ns = np.array([int(p[0]) for p in posets], dtype=np.int64)
    srcs = [np.ascontiguousarray(p[1], dtype=np.int32) for p in posets]
    dsts = [np.ascontiguousarray(p[2], dtype=np.int32) for p in posets]
    cids = [None if p[3] is None else np.ascontiguousarray(p[3], dtype=np.int32) for p in posets]
    ms = np.array([a.size for a in srcs], dtype=np.int64)
    ptr = lambda arrs: (ctypes.c_void_p * count)(*[None if a is None else a.ctypes.data for a in arrs])
    psrc, pdst, pcid = ptr(srcs), ptr(dsts), ptr(cids)
    opts = _opts(build_transpose, host_only, mobius_schedule, mobius_blocks_per_sm, mobius_pace_ns, niv_format,
                 spin_limit, debug_withhold, device_build, torch_allocator)
    out = ctypes.c_void_p()
    st = lib.mz_build_batch(count, ns.ctypes.data, ms.ctypes.data, psrc, pdst,
                            None if all(c is None for c in cids) else pcid, ctypes.byref(opts), ctypes.byref(out))
    if st != MZ_OK:
        _check_alloc_errors()
    _check(st, "mz_build_batch")
    return out.value


def mz_destroy(plan: int) -> None:
    lib.mz_destroy(plan)


def mz_workspace_size(plan: int, dtype: int, batch: int) -> int:
    out = ctypes.c_size_t()
    _check(lib.mz_workspace_size(plan, dtype, batch, ctypes.byref(out)), "mz_workspace_size")
    return out.value


def _transform(name: str, plan: int, dtype: int, x_ptr: int, y_ptr: int, batch: int, ws_ptr: int,
               ws_bytes: int, stream: int) -> None:
    _check(getattr(lib, name)(plan, dtype, x_ptr, y_ptr, batch, ws_ptr, ws_bytes, stream), name)


def mz_zeta(plan, dtype, f_ptr, g_ptr, batch, ws_ptr, ws_bytes, stream=0):
    _transform("mz_zeta", plan, dtype, f_ptr, g_ptr, batch, ws_ptr, ws_bytes, stream)


def _header_scratch_bytes() -> int:
    """MZ_NOALLOC_SCRATCH_BYTES as include/mz.h defines it (the header the library is
    compiled from), so that the binding cannot drift from the library."""
    import re
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "include", "mz.h")
    with open(path) as fh:
        m = re.search(r"#define\s+MZ_NOALLOC_SCRATCH_BYTES\s+\(\(size_t\)(\d+)\s*<<\s*(\d+)\)", fh.read())
    if not m:
        raise RuntimeError("MZ_NOALLOC_SCRATCH_BYTES not found in include/mz.h")
    return int(m.group(1)) << int(m.group(2))


# Bytes of the library's fixed scratch array used by mz_zeta_noalloc.
MZ_NOALLOC_SCRATCH_BYTES = _header_scratch_bytes()


def mz_zeta_noalloc(plan, dtype, f_ptr, g_ptr, batch, stream=0):
    """mz_zeta without a workspace: uses the library's fixed scratch array and allocates
    nothing (for callers that must not allocate device memory at call time)."""
    _check(lib.mz_zeta_noalloc(plan, dtype, f_ptr, g_ptr, batch, stream), "mz_zeta_noalloc")


def mz_mobius(plan, dtype, g_ptr, f_ptr, batch, ws_ptr, ws_bytes, stream=0):
    _transform("mz_mobius", plan, dtype, g_ptr, f_ptr, batch, ws_ptr, ws_bytes, stream)


def mz_zeta_T(plan, dtype, h_ptr, r_ptr, batch, ws_ptr, ws_bytes, stream=0):
    _transform("mz_zeta_T", plan, dtype, h_ptr, r_ptr, batch, ws_ptr, ws_bytes, stream)


def mz_mobius_T(plan, dtype, h_ptr, r_ptr, batch, ws_ptr, ws_bytes, stream=0):
    _transform("mz_mobius_T", plan, dtype, h_ptr, r_ptr, batch, ws_ptr, ws_bytes, stream)


def mz_check(plan: int, stream: int = 0) -> None:
    _check(lib.mz_check(plan, stream), "mz_check")


def mz_plan_tune(plan: int, mobius_blocks_per_sm: int = 0, mobius_pace_ns: int = 0,
                 gather_blocks_per_sm: int = 0, mobius_lanes: int = 0) -> dict:
    """mz_plan_tune: sets the given launch shapes (0 keeps one) and returns the current ones."""
    cur = Tuning()
    want = Tuning(int(mobius_blocks_per_sm), int(mobius_pace_ns), int(gather_blocks_per_sm), int(mobius_lanes))
    _check(lib.mz_plan_tune(plan, ctypes.byref(want), ctypes.byref(cur)), "mz_plan_tune")
    return cur.as_dict()


def mz_plan_info(plan: int) -> dict:
    info = PlanInfo()
    _check(lib.mz_plan_info(plan, ctypes.byref(info)), "mz_plan_info")
    return info.as_dict()


def mz_plan_export(plan: int, what: int, dual: bool = False) -> np.ndarray:
    info = mz_plan_info(plan)
    count = info["n"] * (info["k"] if what == MZ_EXPORT_NIV else 1)
    out = np.empty(count, dtype=np.int32)
    _check(lib.mz_plan_export(plan, what, int(dual), out.ctypes.data, out.nbytes), "mz_plan_export")
    return out.reshape(info["n"], info["k"]) if what == MZ_EXPORT_NIV else out


def mz_plan_save(plan: int, path: str) -> None:
    """mz_plan_save: the plan's precomputation to a file."""
    _check(lib.mz_plan_save(plan, os.fsencode(path)), "mz_plan_save")


def mz_plan_load(path: str, *, host_only: bool = False, mobius_schedule: int = MZ_SCHED_ULEVEL,
                 spin_limit: int = 0, debug_withhold: int = 0, mobius_blocks_per_sm: int = 0,
                 mobius_pace_ns: int = 0, torch_allocator: bool = False) -> int:
    """mz_plan_load: a plan handle from a file written by mz_plan_save."""
    opts = _opts(False, host_only, mobius_schedule, mobius_blocks_per_sm, mobius_pace_ns, 0,
                 spin_limit, debug_withhold, 0, torch_allocator)
    out = ctypes.c_void_p()
    st = lib.mz_plan_load(os.fsencode(path), ctypes.byref(opts), ctypes.byref(out))
    if st != MZ_OK:
        _check_alloc_errors()
    _check(st, "mz_plan_load")
    return out.value


def mz_last_launch_count() -> int:
    return int(lib.mz_last_launch_count())


def mz_set_launch_events(handles) -> None:
    """handles: a list of cudaEvent_t integers (e.g. torch.cuda.Event(...).cuda_event), or None."""
    if not handles:
        lib.mz_set_launch_events(None, 0)
        mz_set_launch_events._keep = None
        return
    arr = (ctypes.c_void_p * len(handles))(*handles)
    mz_set_launch_events._keep = arr        # the library keeps the pointer until reset
    lib.mz_set_launch_events(arr, len(handles))


# ----------------------------------------------------------------------------- torch-facing plan

_TORCH_DTYPE = {MZ_I64: "int64", MZ_F64: "float64", MZ_F32C: "float32"}


def dtype_of(t) -> int:
    import torch
    if t.dtype == torch.int64:
        return MZ_I64
    if t.dtype == torch.float64:
        return MZ_F64
    if t.dtype == torch.float32:
        return MZ_F32C
    raise TypeError(f"unsupported dtype {t.dtype}")


class Plan:
    """A built poset plan plus a cached device workspace (allocated through torch)."""

    def __init__(self, n: int, src, dst, chain_id=None, *, _handle=None, **opts):
        self.handle = _handle if _handle is not None else mz_build(n, src, dst, chain_id, **opts)
        self.info = mz_plan_info(self.handle)
        self.n = self.info["n"]
        self._ws = {}

    @classmethod
    def batch(cls, posets, **opts):
        """One plan for many posets: a list of (n, src, dst, chain_id or None). Values are
        [sum n] or [sum n, batch] arrays, poset after poset."""
        return cls(0, None, None, _handle=mz_build_batch(posets, **opts))

    @classmethod
    def load(cls, path, **opts):
        """A plan from a file written by Plan.save (mz_plan_load); opts as mz_plan_load."""
        return cls(0, None, None, _handle=mz_plan_load(path, **opts))

    def save(self, path):
        """Writes the plan's precomputation to `path` (mz_plan_save)."""
        mz_plan_save(self.handle, path)

    def close(self):
        if getattr(self, "handle", None):
            mz_destroy(self.handle)
            self.handle = None
        self._ws = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, what: int, dual: bool = False) -> np.ndarray:
        return mz_plan_export(self.handle, what, dual)

    def workspace(self, dtype: int, batch: int, device=None):
        import torch
        key = (dtype, batch)
        ws = self._ws.get(key)
        if ws is None:
            nbytes = mz_workspace_size(self.handle, dtype, batch)
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
            self._ws[key] = ws
        base = ws.data_ptr()
        aligned = (base + 255) & ~255
        return aligned, ws.numel() - (aligned - base)

    def _shape(self, x, dtype):
        if dtype == MZ_F32C:
            if x.dim() not in (2, 3) or x.shape[0] != 2 or x.shape[1] != self.n:
                raise ValueError("F32C values are [2, n] or [2, n, batch] (hi plane, lo plane)")
            return 1 if x.dim() == 2 else x.shape[2]
        if x.dim() not in (1, 2) or x.shape[0] != self.n:
            raise ValueError("values are [n] or [n, batch]")
        return 1 if x.dim() == 1 else x.shape[1]

    def _run(self, name, x, out=None, stream=None):
        import torch
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("expects a contiguous CUDA tensor")
        dtype = dtype_of(x)
        batch = self._shape(x, dtype)
        y = torch.empty_like(x) if out is None else out
        ws, wsb = self.workspace(dtype, batch, x.device)
        s = torch.cuda.current_stream(x.device).cuda_stream if stream is None else stream
        _transform(name, self.handle, dtype, x.data_ptr(), y.data_ptr(), batch, ws, wsb, s)
        return y

    def zeta(self, f, out=None, stream=None):
        return self._run("mz_zeta", f, out, stream)

    def mobius(self, g, out=None, stream=None):
        return self._run("mz_mobius", g, out, stream)

    def zeta_T(self, h, out=None, stream=None):
        return self._run("mz_zeta_T", h, out, stream)

    def mobius_T(self, h, out=None, stream=None):
        return self._run("mz_mobius_T", h, out, stream)

    def check(self, stream=None):
        import torch
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        mz_check(self.handle, s)


def f32c(x):
    """fp32 tensor [n] / [n, B] -> the F32C pair tensor [2, n(, B)] with a zero lo plane."""
    import torch
    return torch.stack([x.float(), torch.zeros_like(x, dtype=torch.float32)])


def _apply(plan, name, x):
    """Runs transform `name` on a float64 tensor (MZ_F64) or a plain float32 tensor
    (MZ_F32C with a zero lo plane; the hi plane, the result rounded to fp32, is returned)."""
    import torch
    x = x.contiguous()
    if x.dtype == torch.float32:
        return getattr(plan, name)(torch.stack([x, torch.zeros_like(x)]))[0].contiguous()
    return getattr(plan, name)(x)


def _autograd():
    import torch

    class ZetaFn(torch.autograd.Function):
        """g = Z f; the gradient of a loss L is dL/df = Z^T dL/dg (the dual poset's zeta).
        float64 tensors use MZ_F64; float32 tensors the compensated MZ_F32C path."""

        @staticmethod
        def forward(ctx, f, plan):
            ctx.plan = plan
            return _apply(plan, "zeta", f)

        @staticmethod
        def backward(ctx, grad):
            return _apply(ctx.plan, "zeta_T", grad), None

    class MobiusFn(torch.autograd.Function):
        """f = M g; dL/dg = M^T dL/df (the dual poset's Moebius transform)."""

        @staticmethod
        def forward(ctx, g, plan):
            ctx.plan = plan
            return _apply(plan, "mobius", g)

        @staticmethod
        def backward(ctx, grad):
            return _apply(ctx.plan, "mobius_T", grad), None

    return ZetaFn, MobiusFn


def __getattr__(name):
    if name in ("ZetaFn", "MobiusFn"):
        z, m = _autograd()
        globals()["ZetaFn"], globals()["MobiusFn"] = z, m
        return globals()[name]
    raise AttributeError(name)
