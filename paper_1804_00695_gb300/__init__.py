"""GB300 (sm_103a) CSR sparse matrix-matrix multiplication C = A*B.

Thin ctypes binding over the C ABI in ``include/spgemm.h``: it only marshals
torch tensors (device memory) and the current CUDA stream into the library's
calls.  Every step of the product runs in the library's CUDA kernels; there is
no CPU or PyTorch fallback.  The library must have been built
(``__graft_entry__.build()`` or ``python -m paper_1804_00695_gb300._build``);
calls raise ``RuntimeError`` when it is missing.

Method: Deveci et al., "Sparse Matrix-Matrix Multiplication on Multilevel
Memory Architectures" - two-phase (symbolic, numeric) row-wise product with
compressed column sets and hash-map accumulators (Section 2.1, Section 3.3),
and the chunking methods of Section 3.3.1 for operands in host memory.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libspgemm_gb300.so")

F32, F64 = 0, 1
NBINS = 8
OPT_F64_NATIVE, OPT_LANES_NUMERIC, OPT_LANES_SYMBOLIC, OPT_SMALL_CAP, OPT_SLOT_FACTOR = 1, 2, 3, 4, 5
OPT_NARROW, OPT_LANES_NARROW_SYMBOLIC, OPT_LANES_NARROW_NUMERIC, OPT_CHUNK_BUFFERS = 6, 7, 8, 9
OPT_WAIT_LIMIT_MS = 10
BIN_NARROW = 7
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_DIM", 3: "ERR_INDEX", 4: "ERR_NOMEM", 5: "ERR_BUDGET",
          6: "ERR_TIMEOUT", 7: "ERR_CUDA", 8: "ERR_NOT_SYMBOLIC", 9: "ERR_INTERNAL"}


class SpgemmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class TimingRec(C.Structure):
    _fields_ = [("label", C.c_char * 32), ("launches", C.c_int64), ("rows", C.c_int64),
                ("ms", C.c_double)]


class ChunkPlanRec(C.Structure):
    _fields_ = [("algorithm", C.c_int), ("branch", C.c_int), ("n_ac", C.c_int64), ("n_b", C.c_int64),
                ("size_a", C.c_int64), ("size_b", C.c_int64), ("size_c", C.c_int64),
                ("cost_chunk1", C.c_int64), ("cost_chunk2", C.c_int64),
                ("ac_cuts", C.c_void_p), ("b_cuts", C.c_void_p), ("cap_ac", C.c_int64),
                ("cap_b", C.c_int64)]


class ChunkStatsRec(C.Structure):
    _fields_ = [("algorithm", C.c_int), ("branch", C.c_int), ("n_ac", C.c_int64), ("n_b", C.c_int64),
                ("cost_chunk1", C.c_int64), ("cost_chunk2", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("skipped_b_parts", C.c_int64), ("device_bytes", C.c_int64),
                ("b_windows", C.c_int64)]


class CsrDesc(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("values", C.c_void_p)]


_lib = None

# int alloc(void *user, int64_t nnz, int32_t **col_idx, void **values)
ALLOC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p))


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    lib = C.CDLL(path)
    p, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    sig = {
        "spgemm_last_error": ([], C.c_char_p),
        "spgemm_version": ([], C.c_char_p),
        "spgemm_create": ([C.POINTER(p), i32], i32),
        "spgemm_destroy": ([p], i32),
        "spgemm_check": ([p, p], i32),
        "spgemm_symbolic": ([p, p, p, p, C.POINTER(i64), p], i32),
        "spgemm_numeric": ([p, i32, p, p, p, p], i32),
        "spgemm_row_flops": ([p, p, p, p, p], i32),
        "spgemm_compress": ([p, p, p, p, p], i32),
        "spgemm_bin_counts": ([p, p, p], i32),
        "spgemm_bin_of": ([i64, i64], i32),
        "spgemm_launch_count": ([p, C.POINTER(i64)], i32),
        "spgemm_set_timing": ([p, i32], i32),
        "spgemm_timings": ([p, p, i32, C.POINTER(i32)], i32),
        "spgemm_reset_timings": ([p], i32),
        "spgemm_set_option": ([p, i32, i64], i32),
        "spgemm_plan_chunks": ([p, i64, p, p, i64, i32, i64, p], i32),
        "spgemm_chunked_symbolic": ([p, p, p, p, C.POINTER(i64), C.c_size_t, p], i32),
        "spgemm_chunked_numeric": ([p, i32, p, p, p, C.c_size_t, p], i32),
        "spgemm_chunked_stats": ([p, p], i32),
        "spgemm_chunked": ([p, i32, p, p, p, ALLOC_FN, p, C.c_size_t, p], i32),
        "spgemm_host": ([p, i32, p, p, p, ALLOC_FN, p, i32, p], i32),
        "spgemm_triangles": ([p, p, C.POINTER(i64), p, p, p], i32),
        "spgemm_managed_alloc": ([C.c_size_t, C.POINTER(p)], i32),
        "spgemm_managed_free": ([p], i32),
        "spgemm_backward": ([p, i32, p, p, p, p, p, p], i32),
        "spgemm_batched_symbolic": ([p, i32, p, p, p, C.POINTER(i64), p, p], i32),
        "spgemm_batched_numeric": ([p, i32, i32, p, p, p, p], i32),
        "spgemm_batched_backward": ([p, i32, p, p, p, p], i32),
        "spgemm_autotune": ([p, i32, p, C.POINTER(C.c_float), p], i32),
        "spgemm_row_offsets_noalloc": ([p, i64, p], i32),
        "spgemm_row_offsets_noalloc_max_rows": ([], i64),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise SpgemmError(status, _lib.spgemm_last_error().decode())


def version() -> str:
    return load().spgemm_version().decode()


def _torch():
    import torch
    return torch


@dataclass
class Csr:
    """CSR matrix in device memory as torch tensors (int64 row_ptr, int32
    col, float32/float64 val)."""
    nrows: int
    ncols: int
    row_ptr: "object"
    col: "object"
    val: "object" = None

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    def desc(self) -> CsrDesc:
        return CsrDesc(self.nrows, self.ncols, self.nnz, self.row_ptr.data_ptr(),
                       self.col.data_ptr() if self.col.numel() else None,
                       self.val.data_ptr() if (self.val is not None and self.val.numel()) else None)

    def dev_desc(self) -> CsrDesc:
        """desc() for a device call: every array must be device, managed or
        pinned host memory (the kernels dereference it in place); pageable
        host memory is refused here rather than faulting on the device."""
        for t in (self.row_ptr, self.col, self.val):
            if t is not None and t.device.type == "cpu" and t.numel() and not t.is_pinned():
                raise ValueError("a device call needs device, managed or pinned host arrays; "
                                 "got pageable host memory (use Csr.placed or tensor.pin_memory())")
        return self.desc()

    @staticmethod
    def from_host(m, device="cuda", dtype=None) -> "Csr":
        """Copy an ``inputs.Csr`` (numpy) to the device."""
        torch = _torch()
        val = m.val if dtype is None else m.val.astype(dtype)
        return Csr(m.nrows, m.ncols, torch.from_numpy(m.row_ptr).to(device),
                   torch.from_numpy(m.col).to(device), torch.from_numpy(val).to(device))

    @staticmethod
    def placed(m, placement: str, dtype=None, device="cuda") -> "Csr":
        """An ``inputs.Csr`` in device, pinned host or managed memory (see
        placed_tensor); every device call takes it as it is."""
        val = m.val if dtype is None else m.val.astype(dtype)
        return Csr(m.nrows, m.ncols, *(placed_tensor(x, placement, device) for x in (m.row_ptr, m.col, val)))

    def dtype_code(self) -> int:
        torch = _torch()
        if self.val.dtype == torch.float64:
            return F64
        if self.val.dtype == torch.float32:
            return F32
        raise TypeError(f"unsupported value dtype {self.val.dtype}")


class ManagedBuffer:
    """Managed (UVM) memory from spgemm_managed_alloc, freed with the object;
    exposes __cuda_array_interface__ so torch can view it without a copy."""

    def __init__(self, nbytes: int, typestr: str, count: int):
        lib = load()
        self.ptr = C.c_void_p()
        _check(lib.spgemm_managed_alloc(max(nbytes, 1), C.byref(self.ptr)))
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (self.ptr.value or 0, False), "version": 3}

    def __del__(self):
        if _lib is not None and self.ptr:
            _lib.spgemm_managed_free(self.ptr)
            self.ptr = C.c_void_p()


def placed_tensor(x, placement: str, device="cuda"):
    """A copy of numpy array x in device memory ("device"), pinned host
    memory ("pinned": the device reads and writes it in place) or managed
    memory ("managed": written here by the host, so its pages start on the
    host and migrate when the device touches them)."""
    torch = _torch()
    t = torch.from_numpy(np.ascontiguousarray(x))
    if placement == "device":
        return t.to(device)
    if placement == "pinned":
        return t.pin_memory()
    if placement == "managed":
        buf = ManagedBuffer(t.numel() * t.element_size(), t.numpy().dtype.str, t.numel())
        if t.numel():
            C.memmove(buf.ptr.value, t.data_ptr(), t.numel() * t.element_size())
        out = torch.as_tensor(buf, device=device)
        out._managed_owner = buf   # keep the allocation alive with the view
        return out
    raise ValueError(f"unknown placement {placement!r}")


def placed_empty(n: int, dtype, placement: str, device="cuda"):
    """An uninitialised tensor of n elements with the given placement."""
    torch = _torch()
    if placement == "device":
        return torch.empty(n, dtype=dtype, device=device)
    if placement == "pinned":
        return torch.empty(n, dtype=dtype).pin_memory()
    if placement == "managed":
        z = np.empty(n, dtype={torch.int64: np.int64, torch.int32: np.int32, torch.float64: np.float64,
                               torch.float32: np.float32}[dtype])
        return placed_tensor(z, "managed", device)
    raise ValueError(f"unknown placement {placement!r}")


def _empty_like_placed(t):
    """An uninitialised tensor like t in t's placement (pinned stays pinned)."""
    torch = _torch()
    return torch.empty_like(t).pin_memory() if t.device.type == "cpu" else torch.empty_like(t)


@dataclass
class HostCsr(Csr):
    """CSR matrix in (pinned) host memory as torch CPU tensors."""

    @staticmethod
    def from_numpy(m, dtype=None, pin: bool = True) -> "HostCsr":
        torch = _torch()
        val = m.val if dtype is None else m.val.astype(dtype)
        t = [torch.from_numpy(x) for x in (m.row_ptr, m.col, val)]
        if pin:
            t = [x.pin_memory() for x in t]
        return HostCsr(m.nrows, m.ncols, *t)


def _stream(stream=None) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


class Handle:
    """Owns a library handle (device workspace and symbolic state)."""

    def __init__(self, device: int | None = None):
        torch = _torch()
        lib = load()
        self.device = torch.cuda.current_device() if device is None else device
        self._h = C.c_void_p()
        _check(lib.spgemm_create(C.byref(self._h), self.device))

    def close(self):
        if self._h:
            load().spgemm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self._h

    # -- two phases -----------------------------------------------------------
    def symbolic(self, A: Csr, B: Csr, stream=None, placement: str = "device", out=None):
        """Row offsets of C = A*B (int64 tensor in the given placement, or
        written into `out`, A.nrows + 1 int64 in any placement) and nnz(C)."""
        torch = _torch()
        if out is not None:
            if out.dtype != torch.int64 or out.numel() != A.nrows + 1:
                raise ValueError("out must hold A.nrows + 1 int64 offsets")
            if out.device.type == "cpu" and not out.is_pinned():
                raise ValueError("out must be device, managed or pinned host memory")
            rp = out
        else:
            rp = placed_empty(A.nrows + 1, torch.int64, placement, torch.device("cuda", self.device))
        nnz = C.c_int64()
        da, db = A.dev_desc(), B.dev_desc()
        _check(_lib.spgemm_symbolic(self._h, C.byref(da), C.byref(db), rp.data_ptr(), C.byref(nnz),
                                    _stream(stream)))
        return rp, int(nnz.value)

    def numeric(self, A: Csr, B: Csr, row_ptr, nnz: int, stream=None, placement: str = "device") -> Csr:
        """Columns (ascending per row) and values of C = A*B (in the given placement)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        col = placed_empty(nnz, torch.int32, placement, dev)
        val = placed_empty(nnz, A.val.dtype, placement, dev)
        c = Csr(A.nrows, B.ncols, row_ptr, col, val)
        self.numeric_into(A, B, c, stream)
        return c

    def numeric_into(self, A: Csr, B: Csr, Cm: Csr, stream=None):
        da, db, dc = A.dev_desc(), B.dev_desc(), Cm.dev_desc()
        _check(_lib.spgemm_numeric(self._h, A.dtype_code(), C.byref(da), C.byref(db), C.byref(dc),
                                   _stream(stream)))

    def spgemm(self, A: Csr, B: Csr, stream=None, placement: str = "device") -> Csr:
        """C = A*B; C in the given placement ("device", "pinned", "managed")."""
        rp, nnz = self.symbolic(A, B, stream, placement)
        return self.numeric(A, B, rp, nnz, stream, placement)

    def backward(self, A: Csr, B: Csr, Cm: Csr, dC, need_a: bool = True, need_b: bool = True,
                 stream=None):
        """(dA values on pattern(A), dB values on pattern(B)) for dC given on
        the pattern of C = A*B."""
        torch = _torch()
        da = _empty_like_placed(A.val) if need_a else None
        db = _empty_like_placed(B.val) if need_b else None
        dcm = Csr(Cm.nrows, Cm.ncols, Cm.row_ptr, Cm.col, dC.contiguous())
        d1, d2, d3 = A.dev_desc(), B.dev_desc(), dcm.dev_desc()
        _check(_lib.spgemm_backward(self._h, A.dtype_code(), C.byref(d1), C.byref(d2), C.byref(d3),
                                    da.data_ptr() if da is not None else None,
                                    db.data_ptr() if db is not None else None, _stream(stream)))
        return da, db

    # -- tuning -------------------------------------------------------------------
    def autotune(self, reps: int = 3, stream=None):
        """Time the last numeric call under every tunable setting; keep the
        fastest.  Returns ((lanes, small_cap, slot_factor), ms)."""
        ch = (C.c_int64 * 3)()
        ms = C.c_float()
        _check(_lib.spgemm_autotune(self._h, reps, ch, C.byref(ms), _stream(stream)))
        return (int(ch[0]), int(ch[1]), int(ch[2])), float(ms.value)

    def check(self, stream=None):
        _check(_lib.spgemm_check(self._h, _stream(stream)))

    # -- inspection ---------------------------------------------------------------
    def row_flops(self, A: Csr, B: Csr, stream=None):
        torch = _torch()
        out = torch.empty(A.nrows, dtype=torch.int64, device=A.row_ptr.device)
        da, db = A.dev_desc(), B.dev_desc()
        _check(_lib.spgemm_row_flops(self._h, C.byref(da), C.byref(db), out.data_ptr(), _stream(stream)))
        return out

    def compress(self, M: Csr, stream=None):
        """(count per row, pairs as an (nnz, 2) uint32-in-int32 tensor)."""
        torch = _torch()
        dev = M.row_ptr.device
        cnt = torch.empty(M.nrows, dtype=torch.int32, device=dev)
        pairs = torch.zeros((max(M.nnz, 1), 2), dtype=torch.int32, device=dev)
        dm = M.dev_desc()
        _check(_lib.spgemm_compress(self._h, C.byref(dm), cnt.data_ptr(), pairs.data_ptr(),
                                    _stream(stream)))
        return cnt, pairs

    # -- chunked product, operands in (pinned) host memory ----------------------
    def chunked_symbolic(self, A: "HostCsr", B: "HostCsr", budget: int, stream=None, out=None):
        """Row offsets of C (host int64 tensor, pinned; `out` if given) and nnz(C)."""
        torch = _torch()
        rp = out if out is not None else torch.empty(A.nrows + 1, dtype=torch.int64).pin_memory()
        if rp.dtype != torch.int64 or rp.numel() != A.nrows + 1 or rp.device.type != "cpu":
            raise ValueError("out must be a host int64 tensor of nrows(A) + 1 entries")
        nnz = C.c_int64()
        da, db = A.desc(), B.desc()
        _check(_lib.spgemm_chunked_symbolic(self._h, C.byref(da), C.byref(db), rp.data_ptr(),
                                            C.byref(nnz), budget, _stream(stream)))
        return rp, int(nnz.value)

    def chunked_numeric(self, A: "HostCsr", B: "HostCsr", row_ptr, nnz: int, budget: int,
                        stream=None) -> "HostCsr":
        """Columns and values of C into pinned host tensors (synchronised)."""
        torch = _torch()
        col = torch.empty(nnz, dtype=torch.int32).pin_memory()
        val = torch.empty(nnz, dtype=A.val.dtype).pin_memory()
        Cm = HostCsr(A.nrows, B.ncols, row_ptr, col, val)
        da, db, dc = A.desc(), B.desc(), Cm.desc()
        _check(_lib.spgemm_chunked_numeric(self._h, A.dtype_code(), C.byref(da), C.byref(db), C.byref(dc),
                                           budget, _stream(stream)))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        self.check(stream)
        return Cm

    def chunked_numeric_into(self, A: "HostCsr", B: "HostCsr", Cm: "HostCsr", budget: int, stream=None):
        """Fill the preallocated (pinned) Cm.col / Cm.val; synchronised."""
        da, db, dc = A.desc(), B.desc(), Cm.desc()
        _check(_lib.spgemm_chunked_numeric(self._h, A.dtype_code(), C.byref(da), C.byref(db), C.byref(dc),
                                           budget, _stream(stream)))
        torch = _torch()
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        self.check(stream)

    def chunked(self, A: "HostCsr", B: "HostCsr", budget: int, stream=None) -> "HostCsr":
        """Both chunked phases in one call (spgemm_chunked): the entries of C
        are allocated (pinned) by a callback once nnz(C) is known."""
        torch = _torch()
        rp = torch.empty(A.nrows + 1, dtype=torch.int64).pin_memory()
        held = {}

        def alloc(user, nnz, col_p, val_p):
            try:
                held["col"] = torch.empty(nnz, dtype=torch.int32).pin_memory()
                held["val"] = torch.empty(nnz, dtype=A.val.dtype).pin_memory()
            except Exception:
                return 1
            col_p[0] = held["col"].data_ptr()
            val_p[0] = held["val"].data_ptr()
            return 0

        cb = ALLOC_FN(alloc)
        dc = CsrDesc(A.nrows, B.ncols, 0, rp.data_ptr(), None, None)
        da, db = A.desc(), B.desc()
        _check(_lib.spgemm_chunked(self._h, A.dtype_code(), C.byref(da), C.byref(db), C.byref(dc), cb, None,
                                   budget, _stream(stream)))
        return HostCsr(A.nrows, B.ncols, rp, held["col"], held["val"])

    def host_product(self, A: "HostCsr", B: "Csr", keep_on_device: bool = False, stream=None) -> "Csr":
        """C = A*B with A in (pinned) host memory and B on the host or the
        device (spgemm_host): the library copies the operands in, runs both
        phases on the device and returns C on the host (pinned HostCsr), or
        on the device (Csr) with keep_on_device."""
        torch = _torch()
        b_dev = B.row_ptr.device.type == "cuda"
        dev = torch.device("cuda", self.device)
        if keep_on_device:
            rp = torch.empty(A.nrows + 1, dtype=torch.int64, device=dev)
        else:
            rp = torch.empty(A.nrows + 1, dtype=torch.int64).pin_memory()
        held = {}

        def alloc(user, nnz, col_p, val_p):
            try:
                if keep_on_device:
                    held["col"] = torch.empty(nnz, dtype=torch.int32, device=dev)
                    held["val"] = torch.empty(nnz, dtype=A.val.dtype, device=dev)
                else:
                    held["col"] = torch.empty(nnz, dtype=torch.int32).pin_memory()
                    held["val"] = torch.empty(nnz, dtype=A.val.dtype).pin_memory()
            except Exception:
                return 1
            col_p[0] = held["col"].data_ptr() if nnz else None
            val_p[0] = held["val"].data_ptr() if nnz else None
            return 0

        cb = ALLOC_FN(alloc)
        dc = CsrDesc(A.nrows, B.ncols, 0, rp.data_ptr(), None, None)
        da, db = A.desc(), B.desc()
        flags = (1 if b_dev else 0) | (2 if keep_on_device else 0)
        _check(_lib.spgemm_host(self._h, A.dtype_code(), C.byref(da), C.byref(db), C.byref(dc), cb, None, flags,
                                _stream(stream)))
        cls = Csr if keep_on_device else HostCsr
        return cls(A.nrows, B.ncols, rp, held["col"], held["val"])

    def triangles(self, G: "Csr", labels: bool = False, stream=None):
        """Triangles of the undirected graph with the symmetric pattern G
        (device) by the masked product L*L .* L (spgemm_triangles).  Returns
        the count, or with labels=True (count, labels of the vertices,
        per-vertex counts) as device int64 tensors."""
        torch = _torch()
        total = C.c_int64()
        perm = vc = None
        if labels:
            perm = torch.empty(G.nrows, dtype=torch.int64, device=G.row_ptr.device)
            vc = torch.empty(G.nrows, dtype=torch.int64, device=G.row_ptr.device)
        d = G.dev_desc()
        _check(_lib.spgemm_triangles(self._h, C.byref(d), C.byref(total), perm.data_ptr() if labels else None,
                                     vc.data_ptr() if labels else None, _stream(stream)))
        return (int(total.value), perm, vc) if labels else int(total.value)

    def chunked_stats(self) -> dict:
        r = ChunkStatsRec()
        _check(_lib.spgemm_chunked_stats(self._h, C.byref(r)))
        return {f: getattr(r, f) for f, _ in ChunkStatsRec._fields_}

    def set_option(self, option: int, value: int):
        _check(_lib.spgemm_set_option(self._h, option, value))

    def launch_count(self) -> int:
        n = C.c_int64()
        _check(_lib.spgemm_launch_count(self._h, C.byref(n)))
        return int(n.value)

    def set_timing(self, on=True):
        """True / 1: events around every kernel; 2: numeric-phase kernels only;
        False / 0: off."""
        _check(_lib.spgemm_set_timing(self._h, int(on)))

    def timings(self) -> dict:
        """{label: (launches, rows, ms)} accumulated since the last reset."""
        arr = (TimingRec * 64)()
        n = C.c_int()
        _check(_lib.spgemm_timings(self._h, arr, 64, C.byref(n)))
        return {arr[k].label.decode(): (int(arr[k].launches), int(arr[k].rows), float(arr[k].ms))
                for k in range(min(n.value, 64))}

    def reset_timings(self):
        _check(_lib.spgemm_reset_timings(self._h))

    def bin_counts(self):
        sym = (C.c_int64 * NBINS)()
        num = (C.c_int64 * NBINS)()
        _check(_lib.spgemm_bin_counts(self._h, sym, num))
        return list(sym), list(num)


_default = {}


def default_handle() -> Handle:
    torch = _torch()
    d = torch.cuda.current_device()
    if d not in _default:
        _default[d] = Handle(d)
    return _default[d]


def plan_chunks(a_row_ptr, c_row_ptr, b_row_ptr, value_bytes: int, fast_size: int) -> dict:
    """Algorithm 4 on host row offsets (numpy int64): algorithm, branch,
    part boundaries, sizes and the copy costs of Algorithms 2 and 3."""
    import numpy as np
    lib = load()
    a = np.ascontiguousarray(a_row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(c_row_ptr, dtype=np.int64)
    b = np.ascontiguousarray(b_row_ptr, dtype=np.int64)
    cap_ac, cap_b = len(a) + 1, len(b) + 1
    ac_cuts = np.zeros(cap_ac, dtype=np.int64)
    b_cuts = np.zeros(cap_b, dtype=np.int64)
    rec = ChunkPlanRec()
    rec.ac_cuts, rec.b_cuts = ac_cuts.ctypes.data, b_cuts.ctypes.data
    rec.cap_ac, rec.cap_b = cap_ac, cap_b
    _check(lib.spgemm_plan_chunks(a.ctypes.data, len(a) - 1, c.ctypes.data, b.ctypes.data, len(b) - 1,
                                  value_bytes, fast_size, C.byref(rec)))
    ac = ac_cuts[:rec.n_ac + 1]
    bb = b_cuts[:rec.n_b + 1]
    return {"algorithm": rec.algorithm, "branch": rec.branch,
            "p_ac": list(zip(ac[:-1].tolist(), ac[1:].tolist())),
            "p_b": list(zip(bb[:-1].tolist(), bb[1:].tolist())),
            "size_a": rec.size_a, "size_b": rec.size_b, "size_c": rec.size_c,
            "cost_chunk1": rec.cost_chunk1, "cost_chunk2": rec.cost_chunk2}


def bin_of(keys: int, flops: int) -> int:
    return int(load().spgemm_bin_of(keys, flops))


def spgemm(A: Csr, B: Csr, stream=None) -> Csr:
    """C = A*B with both phases on the current device's default handle."""
    return default_handle().spgemm(A, B, stream)


def _autograd_class():
    torch = _torch()

    class SpGEMMFunction(torch.autograd.Function):
        """C = A*B with a hand-written backward: dA = (dC B^T) on the pattern
        of A and dB = (A^T dC) on the pattern of B, computed by the
        library's backward kernel (no dense intermediates)."""

        @staticmethod
        def forward(ctx, a_val, b_val, a_rp, a_col, b_rp, b_col, shape, handle):
            m, k, n = shape
            A = Csr(m, k, a_rp, a_col, a_val.detach())
            B = Csr(k, n, b_rp, b_col, b_val.detach())
            Cm = handle.spgemm(A, B)
            ctx.save_for_backward(a_val, b_val, a_rp, a_col, b_rp, b_col, Cm.row_ptr, Cm.col)
            ctx.shape, ctx.handle = shape, handle
            ctx.mark_non_differentiable(Cm.row_ptr, Cm.col)
            return Cm.row_ptr, Cm.col, Cm.val

        @staticmethod
        def backward(ctx, g_rp, g_col, g_val):
            a_val, b_val, a_rp, a_col, b_rp, b_col, c_rp, c_col = ctx.saved_tensors
            m, k, n = ctx.shape
            A = Csr(m, k, a_rp, a_col, a_val.detach())
            B = Csr(k, n, b_rp, b_col, b_val.detach())
            Cm = Csr(m, n, c_rp, c_col, None)
            if g_val is None:
                return (None,) * 8
            da, db = ctx.handle.backward(A, B, Cm, g_val, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
            return da, db, None, None, None, None, None, None

    return SpGEMMFunction


_fn = None


def spgemm_autograd(A: Csr, B: Csr, handle: "Handle" = None) -> Csr:
    """Differentiable C = A*B: gradients flow to A.val and B.val."""
    global _fn
    if _fn is None:
        _fn = _autograd_class()
    h = handle or default_handle()
    rp, col, val = _fn.apply(A.val, B.val, A.row_ptr, A.col, B.row_ptr, B.col,
                             (A.nrows, A.ncols, B.ncols), h)
    return Csr(A.nrows, B.ncols, rp, col, val)


class Batch:
    """nbatch independent products A_i * B_i run as one product of
    block-diagonal operands (one launch per kernel for all instances).
    The result is stacked: rows of instance i after those of i-1, columns
    local to the instance."""

    def __init__(self, handle: "Handle", As, Bs):
        self.h = handle
        self.As, self.Bs = list(As), list(Bs)
        self.n = len(self.As)
        self._arrays()

    def _arrays(self):
        self.da = (CsrDesc * max(self.n, 1))(*[a.dev_desc() for a in self.As])
        self.db = (CsrDesc * max(self.n, 1))(*[b.dev_desc() for b in self.Bs])

    @property
    def rows(self):
        return sum(a.nrows for a in self.As)

    def symbolic(self, stream=None):
        torch = _torch()
        dev = self.As[0].row_ptr.device
        rp = torch.empty(self.rows + 1, dtype=torch.int64, device=dev)
        nnz = C.c_int64()
        per = (C.c_int64 * max(self.n, 1))()
        _check(_lib.spgemm_batched_symbolic(self.h.ptr, self.n, self.da, self.db, rp.data_ptr(), C.byref(nnz),
                                            per, _stream(stream)))
        self.row_ptr, self.nnz, self.inst_nnz = rp, int(nnz.value), [int(per[i]) for i in range(self.n)]
        return rp, self.nnz

    def alloc(self):
        torch = _torch()
        dev = self.As[0].row_ptr.device
        return Csr(self.rows, max(b.ncols for b in self.Bs), self.row_ptr,
                   torch.empty(self.nnz, dtype=torch.int32, device=dev),
                   torch.empty(self.nnz, dtype=self.As[0].val.dtype, device=dev))

    def numeric_into(self, Cm: Csr, stream=None):
        self._arrays()
        dc = Cm.dev_desc()
        _check(_lib.spgemm_batched_numeric(self.h.ptr, self.As[0].dtype_code(), self.n, self.da, self.db,
                                           C.byref(dc), _stream(stream)))

    def run(self, stream=None) -> Csr:
        self.symbolic(stream)
        Cm = self.alloc()
        self.numeric_into(Cm, stream)
        return Cm

    def split(self, Cm: Csr):
        """Per-instance views of the stacked result."""
        out, r0, p0 = [], 0, 0
        for a, b, nz in zip(self.As, self.Bs, self.inst_nnz):
            rp = Cm.row_ptr[r0:r0 + a.nrows + 1] - p0
            out.append(Csr(a.nrows, b.ncols, rp, Cm.col[p0:p0 + nz], Cm.val[p0:p0 + nz]))
            r0 += a.nrows
            p0 += nz
        return out

    def backward(self, Cm: Csr, dC, need_a: bool = True, need_b: bool = True, stream=None):
        """Stacked dA, dB for dC on the stacked pattern; split with split_grads."""
        torch = _torch()
        dev = dC.device
        na = sum(a.nnz for a in self.As)
        nb = sum(b.nnz for b in self.Bs)
        da = torch.empty(na, dtype=dC.dtype, device=dev) if need_a else None
        db = torch.empty(nb, dtype=dC.dtype, device=dev) if need_b else None
        dcm = Csr(Cm.nrows, Cm.ncols, Cm.row_ptr, Cm.col, dC.contiguous())
        d = dcm.dev_desc()
        _check(_lib.spgemm_batched_backward(self.h.ptr, self.As[0].dtype_code(), C.byref(d),
                                            da.data_ptr() if da is not None else None,
                                            db.data_ptr() if db is not None else None, _stream(stream)))
        return da, db

    def split_grads(self, da, db):
        ga, gb, pa, pb = [], [], 0, 0
        for a, b in zip(self.As, self.Bs):
            ga.append(da[pa:pa + a.nnz] if da is not None else None)
            gb.append(db[pb:pb + b.nnz] if db is not None else None)
            pa += a.nnz
            pb += b.nnz
        return ga, gb
