"""Python binding of libpms, the GB300 library for exact planted (l,d)-motif search.

Argument marshalling only: every step of the search runs in the library's
CUDA kernels (see include/pms.h). The module-level functions carry the C
names (pms_create, pms_solve, ...); ``Context`` wraps them for convenience.
If the compiled library is missing or fails to load, every entry point raises
``PMSError``: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PMS_OK, PMS_EINVAL, PMS_ENOMEM, PMS_ECUDA, PMS_ETIMEDOUT, PMS_ETOOMANY, PMS_EBUSY, PMS_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
PMS_ESCRATCH = -8
PMS_ECANCELED = -9
ERROR_NAMES = {0: "PMS_OK", -1: "PMS_EINVAL", -2: "PMS_ENOMEM", -3: "PMS_ECUDA", -4: "PMS_ETIMEDOUT",
               -5: "PMS_ETOOMANY", -6: "PMS_EBUSY", -7: "PMS_ENOTFOUND", -8: "PMS_ESCRATCH", -9: "PMS_ECANCELED"}
PMS_FAULT_ALLOC = 1
PMS_FAULT_UPLOAD = 2
LMAX, NMAX = 32, 64

#: names the C ABI exports (include/pms.h)
ABI_FUNCTIONS = ["pms_create", "pms_set_stream", "pms_set_allocator", "pms_set_options", "pms_get_options",
                 "pms_solve", "pms_solve_device", "pms_solve_batch", "pms_submit", "pms_wait", "pms_release",
                 "pms_get_stats", "pms_decode", "pms_last_error", "pms_probe_int_rate", "pms_destroy",
                 "pms_solve_device_noalloc", "pms_autotune", "pms_save_tuning", "pms_load_tuning",
                 "pms_solve_sigma", "pms_kernel_binary_version", "pms_cancel", "pms_inject_fault"]

#: the twenty amino acids, one-letter codes (an alphabet for solve_sigma)
PROTEIN = b"ACDEFGHIKLMNPQRSTVWY"


class PMSError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")


class pms_instance(ctypes.Structure):
    _fields_ = [("seqs", ctypes.POINTER(ctypes.c_uint8)), ("n", ctypes.c_int), ("m", ctypes.c_int),
                ("l", ctypes.c_int), ("d", ctypes.c_int)]


class pms_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("motifs", ctypes.POINTER(ctypes.c_uint64)), ("count", ctypes.c_size_t)]


class pms_options(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("chunk_work", ctypes.c_int), ("grab", ctypes.c_int),
                ("max_motifs", ctypes.c_size_t), ("count_work", ctypes.c_int), ("serve_wave_items", ctypes.c_int),
                ("serve_max_inflight", ctypes.c_int), ("smem_rows", ctypes.c_int), ("autotune", ctypes.c_int),
                ("seed_mode", ctypes.c_int), ("quorum", ctypes.c_int), ("partial_rows", ctypes.c_int),
                ("graph", ctypes.c_int), ("triple_rows", ctypes.c_int)]


class pms_tuning(ctypes.Structure):
    _fields_ = [("chunk_work", ctypes.c_int), ("prune_rows", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("grab", ctypes.c_int), ("partial_rows", ctypes.c_int), ("ms", ctypes.c_double)]


class pms_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_uint64), ("subsets", ctypes.c_uint64), ("subsets_pruned", ctypes.c_uint64),
                ("candidates_tested", ctypes.c_uint64), ("cmp_rows", ctypes.c_uint64), ("cmp_reduce", ctypes.c_uint64),
                ("cmp_verify", ctypes.c_uint64), ("seeds_infeasible", ctypes.c_uint64), ("ms_total", ctypes.c_double),
                ("ms_kernel", ctypes.c_double), ("ms_verify", ctypes.c_double),
                ("serve_waves", ctypes.c_uint64), ("serve_overlapped_waves", ctypes.c_uint64),
                ("serve_max_requests_per_wave", ctypes.c_uint64), ("graph_replays", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libpms.so (building it first if needed). Raises PMSError if that fails."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        try:
            path = _build.build() if build_if_missing else _build.LIB
            lib = ctypes.CDLL(path)
        except Exception as e:  # noqa: BLE001
            raise PMSError(PMS_ECUDA, f"the CUDA library could not be built or loaded: {e}") from e
        vp, sz, ci = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        u8p, u64p, u32p = ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
        sig = {
            "pms_create": (ci, [ctypes.POINTER(vp), ci, sz]),
            "pms_set_stream": (ci, [vp, vp]),
            "pms_set_allocator": (ci, [vp, ALLOC_FN, FREE_FN, vp]),
            "pms_set_options": (ci, [vp, ctypes.POINTER(pms_options)]),
            "pms_get_options": (ci, [vp, ctypes.POINTER(pms_options)]),
            "pms_solve": (ci, [vp, u8p, ci, ci, ci, ci, ctypes.POINTER(u64p), ctypes.POINTER(sz)]),
            "pms_solve_device": (ci, [vp, vp, ci, ci, ci, ci, vp, sz, vp]),
            "pms_solve_batch": (ci, [vp, ctypes.POINTER(pms_instance), ci, ctypes.POINTER(pms_result)]),
            "pms_submit": (ci, [vp, ctypes.POINTER(pms_instance), ctypes.POINTER(ctypes.c_uint64)]),
            "pms_wait": (ci, [vp, ctypes.c_uint64, ci, ctypes.POINTER(pms_result)]),
            "pms_release": (ci, [vp, ctypes.c_uint64]),
            "pms_get_stats": (ci, [vp, ctypes.POINTER(pms_stats)]),
            "pms_decode": (ci, [ctypes.c_uint64, ci, ctypes.c_char_p]),
            "pms_last_error": (ctypes.c_char_p, [vp]),
            "pms_probe_int_rate": (ci, [vp, ci, ctypes.POINTER(ctypes.c_double)]),
            "pms_destroy": (None, [vp]),
            "pms_solve_device_noalloc": (ci, [vp, ci, ci, ci, ci, vp, sz, vp, vp]),
            "pms_autotune": (ci, [vp, ci, ci, ci, ci, ctypes.c_void_p]),
            "pms_save_tuning": (ci, [vp, ctypes.c_char_p]),
            "pms_load_tuning": (ci, [vp, ctypes.c_char_p]),
            "pms_solve_sigma": (ci, [vp, u8p, ci, u8p, ci, ci, ci, ci, ci, ctypes.POINTER(u8p), ctypes.POINTER(sz)]),
            "pms_kernel_binary_version": (ci, [ci, ctypes.POINTER(ci)]),
            "pms_cancel": (ci, [vp, ctypes.c_uint64]),
            "pms_inject_fault": (ci, [vp, ci, ci, ci]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _as_seqs(seqs) -> np.ndarray:
    a = np.ascontiguousarray(seqs, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("seqs must be a 2-D (n, m) array of ASCII bytes")
    return a


# ---------------------------------------------------------------- C-named wrappers

def pms_decode(code: int, l: int) -> str:
    buf = ctypes.create_string_buffer(l + 1)
    rc = load().pms_decode(ctypes.c_uint64(int(code)), l, buf)
    if rc:
        raise PMSError(rc, "decode")
    return buf.value.decode()


def pms_create(device: int = 0, mem_budget_bytes: int = 0) -> "Context":
    return Context(device, mem_budget_bytes)


def pms_destroy(ctx: "Context") -> None:
    ctx.close()


def pms_solve(ctx: "Context", seqs, n: int, m: int, l: int, d: int) -> np.ndarray:
    return ctx.solve(np.asarray(seqs, dtype=np.uint8).reshape(n, m), l, d)


def pms_solve_device(ctx: "Context", d_seqs, n: int, m: int, l: int, d: int, d_motifs, capacity: int, d_status) -> None:
    ctx.solve_device(d_seqs, n, m, l, d, d_motifs, capacity, d_status)


def pms_solve_batch(ctx: "Context", instances) -> list:
    return ctx.solve_batch(instances)


def pms_submit(ctx: "Context", seqs, l: int, d: int) -> int:
    return ctx.submit(seqs, l, d)


def pms_wait(ctx: "Context", ticket: int, timeout_ms: int = -1):
    return ctx.wait(ticket, timeout_ms)


def pms_release(ctx: "Context", ticket: int) -> None:
    ctx.release(ticket)


def pms_set_stream(ctx: "Context", stream) -> None:
    ctx.set_stream(stream)


def pms_set_options(ctx: "Context", **kw) -> None:
    ctx.set_options(**kw)


def pms_get_options(ctx: "Context") -> dict:
    return ctx.get_options()


def pms_get_stats(ctx: "Context") -> dict:
    return ctx.stats()


def pms_last_error(ctx: "Context") -> str:
    return ctx.last_error()


def pms_probe_int_rate(ctx: "Context", kind: int) -> float:
    return ctx.probe_int_rate(kind)


def pms_set_allocator(ctx: "Context", alloc, free) -> None:
    ctx.set_allocator(alloc, free)


def pms_autotune(ctx: "Context", n: int, m: int, l: int, d: int) -> dict:
    return ctx.autotune(n, m, l, d)


def pms_save_tuning(ctx: "Context", path: str) -> None:
    ctx.save_tuning(path)


def pms_load_tuning(ctx: "Context", path: str) -> None:
    ctx.load_tuning(path)


def pms_kernel_binary_version(device: int = 0) -> int:
    """cudaFuncGetAttributes' binaryVersion of the library's device code on `device` (103: sm_103a)."""
    v = ctypes.c_int(0)
    rc = load().pms_kernel_binary_version(int(device), ctypes.byref(v))
    if rc:
        raise PMSError(rc, "pms_kernel_binary_version")
    return int(v.value)


def pms_cancel(ctx: "Context", ticket: int) -> None:
    ctx.cancel(ticket)


def pms_inject_fault(ctx: "Context", kind: int, after: int = 0, count: int = 1) -> None:
    ctx.inject_fault(kind, after, count)


def pms_solve_device_noalloc(d_seqs, n: int, m: int, l: int, d: int, d_motifs, capacity: int, d_status,
                             stream=None) -> None:
    """Allocation-free device solve (no context): every buffer comes from the library's fixed
    per-GPU scratch array. Arguments as for Context.solve_device, plus the stream to enqueue on.
    Calls that overlap on the GPU share that array and race; order them on one stream."""
    p = lambda t: ctypes.c_void_p(int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t))  # noqa: E731
    handle = getattr(stream, "cuda_stream", stream)
    rc = load().pms_solve_device_noalloc(p(d_seqs), int(n), int(m), int(l), int(d), p(d_motifs), int(capacity),
                                         p(d_status), ctypes.c_void_p(int(handle or 0)))
    if rc:
        raise PMSError(rc, "pms_solve_device_noalloc")


# ---------------------------------------------------------------- context object

class Context:
    """One library context (device memory, stream, options) on one CUDA device."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream=None, torch_allocator: bool = False):
        self._lib = load()
        self._h = ctypes.c_void_p()
        rc = self._lib.pms_create(ctypes.byref(self._h), int(device), int(mem_budget_bytes))
        if rc:
            raise PMSError(rc, f"pms_create(device={device}) failed")
        self.device = device
        self._keep = []
        if torch_allocator:
            self._use_torch_allocator()
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime
    def close(self) -> None:
        if self._h:
            self._lib.pms_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int, what: str) -> None:
        if rc:
            raise PMSError(rc, f"{what}: {self.last_error()}")

    def last_error(self) -> str:
        s = self._lib.pms_last_error(self._h)
        return s.decode() if s else ""

    # -- configuration
    def set_stream(self, stream) -> None:
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.pms_set_stream(self._h, ctypes.c_void_p(int(handle or 0))), "pms_set_stream")

    def set_allocator(self, alloc, free) -> None:
        a, f = ALLOC_FN(alloc), FREE_FN(free)
        self._keep += [a, f]
        self._check(self._lib.pms_set_allocator(self._h, a, f, None), "pms_set_allocator")

    def _use_torch_allocator(self) -> None:
        import torch

        dev = self.device

        def alloc(nbytes, _user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=dev))
            except Exception:  # noqa: BLE001
                return None

        def free(ptr, _user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.set_allocator(alloc, free)

    def get_options(self) -> dict:
        o = pms_options()
        self._check(self._lib.pms_get_options(self._h, ctypes.byref(o)), "pms_get_options")
        return {name: getattr(o, name) for name, _ in pms_options._fields_}

    def set_options(self, **kw) -> None:
        cur = self.get_options()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown options {sorted(unknown)}")
        cur.update(kw)
        o = pms_options(**cur)
        self._check(self._lib.pms_set_options(self._h, ctypes.byref(o)), "pms_set_options")

    def stats(self) -> dict:
        s = pms_stats()
        self._check(self._lib.pms_get_stats(self._h, ctypes.byref(s)), "pms_get_stats")
        return s.as_dict()

    def autotune(self, n: int, m: int, l: int, d: int) -> dict:
        t = pms_tuning()
        self._check(self._lib.pms_autotune(self._h, int(n), int(m), int(l), int(d),
                                           ctypes.cast(ctypes.byref(t), ctypes.c_void_p)), "pms_autotune")
        return {name: getattr(t, name) for name, _ in pms_tuning._fields_}

    def save_tuning(self, path: str) -> None:
        self._check(self._lib.pms_save_tuning(self._h, str(path).encode()), "pms_save_tuning")

    def load_tuning(self, path: str) -> None:
        self._check(self._lib.pms_load_tuning(self._h, str(path).encode()), "pms_load_tuning")

    def probe_int_rate(self, kind: int) -> float:
        v = ctypes.c_double()
        self._check(self._lib.pms_probe_int_rate(self._h, int(kind), ctypes.byref(v)), "pms_probe_int_rate")
        return v.value

    # -- solves
    def solve(self, seqs, l: int, d: int) -> np.ndarray:
        """Sorted unique motif codes of one instance given in host memory."""
        a = _as_seqs(seqs)
        n, m = a.shape
        out = ctypes.POINTER(ctypes.c_uint64)()
        cnt = ctypes.c_size_t()
        rc = self._lib.pms_solve(self._h, ctypes.cast(a.__array_interface__["data"][0], ctypes.POINTER(ctypes.c_uint8)),
                                 n, m, int(l), int(d), ctypes.byref(out), ctypes.byref(cnt))
        self._check(rc, "pms_solve")
        if cnt.value == 0:
            return np.zeros(0, dtype=np.uint64)
        return np.frombuffer(ctypes.string_at(out, cnt.value * 8), dtype=np.uint64).copy()

    def solve_sigma(self, seqs, l: int, d: int, alphabet=PROTEIN, q: int = 0) -> np.ndarray:
        """Motifs over a general alphabet (bytes, 2..32 distinct letters) as a (count, l) uint8 array of
        letters, rows in the alphabet's lexicographic order; q = 0: every sequence (PMS)."""
        a = _as_seqs(seqs)
        n, m = a.shape
        alpha = np.frombuffer(alphabet.encode() if isinstance(alphabet, str) else bytes(alphabet), dtype=np.uint8)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        out = u8p()
        cnt = ctypes.c_size_t()
        rc = self._lib.pms_solve_sigma(self._h, ctypes.cast(alpha.__array_interface__["data"][0], u8p), len(alpha),
                                       ctypes.cast(a.__array_interface__["data"][0], u8p), n, m, int(l), int(d),
                                       int(q), ctypes.byref(out), ctypes.byref(cnt))
        self._check(rc, "pms_solve_sigma")
        if cnt.value == 0:
            return np.zeros((0, int(l)), dtype=np.uint8)
        return np.frombuffer(ctypes.string_at(out, cnt.value * int(l)), dtype=np.uint8).reshape(-1, int(l)).copy()

    def solve_device(self, d_seqs, n: int, m: int, l: int, d: int, d_motifs, capacity: int, d_status) -> None:
        """Enqueues a solve on device buffers (torch tensors or raw pointers); does not wait."""
        p = lambda t: ctypes.c_void_p(int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t))  # noqa: E731
        rc = self._lib.pms_solve_device(self._h, p(d_seqs), int(n), int(m), int(l), int(d), p(d_motifs),
                                        int(capacity), p(d_status))
        self._check(rc, "pms_solve_device")

    def solve_batch(self, instances) -> list:
        """instances: list of (seqs (n, m) uint8, l, d). Returns a list of code arrays (or PMSError objects)."""
        arrays = [_as_seqs(s) for (s, _, _) in instances]
        k = len(instances)
        inst = (pms_instance * k)()
        for i, (a, (_, l, d)) in enumerate(zip(arrays, instances)):
            inst[i] = pms_instance(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), a.shape[0], a.shape[1], int(l), int(d))
        res = (pms_result * k)()
        self._check(self._lib.pms_solve_batch(self._h, inst, k, res), "pms_solve_batch")
        out = []
        for r in res:
            if r.status:
                out.append(PMSError(r.status, "instance failed"))
            elif r.count == 0:
                out.append(np.zeros(0, dtype=np.uint64))
            else:
                out.append(np.ctypeslib.as_array(r.motifs, shape=(r.count,)).copy())
        return out

    # -- served form
    def submit(self, seqs, l: int, d: int) -> int:
        a = _as_seqs(seqs)
        inst = pms_instance(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), a.shape[0], a.shape[1], int(l), int(d))
        t = ctypes.c_uint64()
        self._check(self._lib.pms_submit(self._h, ctypes.byref(inst), ctypes.byref(t)), "pms_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> np.ndarray:
        r = pms_result()
        rc = self._lib.pms_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r))
        self._check(rc, "pms_wait")
        if r.status:
            raise PMSError(r.status, "request failed")
        if r.count == 0:
            return np.zeros(0, dtype=np.uint64)
        return np.ctypeslib.as_array(r.motifs, shape=(r.count,)).copy()

    def release(self, ticket: int) -> None:
        self._check(self._lib.pms_release(self._h, ctypes.c_uint64(ticket)), "pms_release")

    def cancel(self, ticket: int) -> None:
        """Withdraws a queued served request (PMSError PMS_EBUSY once it is on the device)."""
        self._check(self._lib.pms_cancel(self._h, ctypes.c_uint64(ticket)), "pms_cancel")

    def inject_fault(self, kind: int, after: int = 0, count: int = 1) -> None:
        """Test hook: the next `count` operations of `kind` (PMS_FAULT_ALLOC, PMS_FAULT_UPLOAD) fail on
        the host after `after` more succeed; count 0 clears it."""
        self._check(self._lib.pms_inject_fault(self._h, int(kind), int(after), int(count)), "pms_inject_fault")


def decode_all(codes, l: int) -> list[str]:
    return [pms_decode(int(c), l) for c in codes]
