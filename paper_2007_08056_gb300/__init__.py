"""Irrep-aligned contraction of cyclic-group-symmetric tensors on GB300.

Thin Python binding over the C ABI of ``libsymctr.so`` (include/symctr.h):
argument marshalling only.  Every step of the contraction (alignment
transforms, the batched GEMM, the map back to the output's reduced form)
runs in the library's CUDA kernels.  PyTorch provides device memory and
streams.  There is no CPU fallback: if the library cannot be loaded, every
entry point raises.

    import paper_2007_08056_gb300 as sc
    plan = sc.Plan("abkl,klij->abij", moduli=[3],
                   sym_u=([1, 1, -1, -1], [0], [4, 4, 4, 4]),
                   sym_v=([1, 1, -1, -1], [0], [4, 4, 4, 4]),
                   precision="split_bf16")
    w = plan.contract(u, v)          # u, v: float64 CUDA tensors in reduced form
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import torch

from . import build as _build

MAX_ORDER = 8
MAX_MODULI = 4

PRECISIONS = {"fp64": 0, "split_bf16": 1, "tf32": 2}

STATUS = {
    0: "SYMCTR_OK", 1: "SYMCTR_ERR_EINSUM", 2: "SYMCTR_ERR_SIGNS", 3: "SYMCTR_ERR_SHAPE",
    4: "SYMCTR_ERR_CHARGE", 5: "SYMCTR_ERR_UNSUPPORTED", 6: "SYMCTR_ERR_NULLPTR",
    7: "SYMCTR_ERR_WORKSPACE", 8: "SYMCTR_ERR_CUDA", 9: "SYMCTR_ERR_DEVICE_TIMEOUT",
    10: "SYMCTR_ERR_OVERFLOW", 11: "SYMCTR_ERR_NONFINITE", 12: "SYMCTR_ERR_ARGUMENT",
}


class SymctrError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS.get(status, status)}: {detail}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("order_u", ctypes.c_int32), ("order_v", ctypes.c_int32), ("order_w", ctypes.c_int32),
        ("s", ctypes.c_int32), ("t", ctypes.c_int32), ("v", ctypes.c_int32),
        ("sigma", ctypes.c_int32), ("n_moduli", ctypes.c_int32),
        ("moduli", ctypes.c_int32 * MAX_MODULI), ("group_order", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("n_slices", ctypes.c_int32),
        ("signs_w", ctypes.c_int8 * MAX_ORDER), ("charge_w", ctypes.c_int32 * MAX_MODULI),
        ("dims_w", ctypes.c_int64 * MAX_ORDER),
        ("numel_u", ctypes.c_int64), ("numel_v", ctypes.c_int64), ("numel_w", ctypes.c_int64),
        ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
        ("n_q", ctypes.c_int32), ("q_single", ctypes.c_int32),
        ("aligned_numel_u", ctypes.c_int64), ("aligned_numel_v", ctypes.c_int64),
        ("aligned_numel_w", ctypes.c_int64),
        ("useful_flops", ctypes.c_double), ("transform_bytes", ctypes.c_double),
        ("workspace_bytes", ctypes.c_uint64), ("workspace_bytes_backward", ctypes.c_uint64),
        ("workspace_bytes_min", ctypes.c_uint64), ("table_bytes", ctypes.c_uint64),
        ("tensor_core", ctypes.c_int32), ("general", ctypes.c_int32),
        ("q_first", ctypes.c_int32), ("q_step", ctypes.c_int32),
        ("sectors_w", ctypes.c_int32 * MAX_ORDER), ("single_read_prep", ctypes.c_int32),
        ("chained", ctypes.c_int32), ("zero_fill_numel", ctypes.c_int64),
    ]


class Operand(ctypes.Structure):
    """symctr_operand: one operand in the general form of Eq. symtsr."""
    _fields_ = [
        ("signs", ctypes.POINTER(ctypes.c_int8)), ("charge", ctypes.POINTER(ctypes.c_int32)),
        ("dims", ctypes.POINTER(ctypes.c_int64)), ("sectors", ctypes.POINTER(ctypes.c_int32)),
        ("sector_dims", ctypes.POINTER(ctypes.c_int64)),
    ]


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsymctr.so (building it in-tree if absent).  Raises on failure."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError(f"libsymctr.so not built ({_build.LIB})")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    i8p, i32p, i64p = (ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int32),
                       ctypes.POINTER(ctypes.c_int64))
    lib.symctr_plan_create.argtypes = [ctypes.c_char_p, ctypes.c_int, i32p, i8p, i32p, i8p, i32p,
                                       i64p, i64p, i8p, i32p, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(P)]
    lib.symctr_plan_query.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.symctr_plan_create_general.argtypes = [ctypes.c_char_p, ctypes.c_int, i32p,
                                               ctypes.POINTER(Operand), ctypes.POINTER(Operand),
                                               i8p, i32p, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(P)]
    lib.symctr_align.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
    lib.symctr_contract.argtypes = [P, P, P, P, P, ctypes.c_size_t, P]
    lib.symctr_contract_backward.argtypes = [P, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.symctr_check_device_error.argtypes = [P, P, P]
    lib.symctr_status_string.argtypes = [ctypes.c_int]
    lib.symctr_status_string.restype = ctypes.c_char_p
    lib.symctr_last_error_detail.argtypes = []
    lib.symctr_last_error_detail.restype = ctypes.c_char_p
    lib.symctr_profile_enable.argtypes = [P, ctypes.c_int]
    lib.symctr_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int)]
    lib.symctr_contract_static_scratch.argtypes = [P, P, P, P, P]
    lib.symctr_selftest_bounded_wait.argtypes = [P, ctypes.c_size_t, ctypes.c_int64, P]
    lib.symctr_contract_complex.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                            ctypes.c_size_t, P]
    lib.symctr_plan_attach_tables.argtypes = [P, P, ctypes.c_size_t, P]
    lib.symctr_plan_chain.argtypes = [P, P, P, ctypes.c_int]
    lib.symctr_plan_destroy.argtypes = [P]
    lib.symctr_plan_destroy.restype = None
    for f in ("symctr_plan_create", "symctr_plan_create_general", "symctr_plan_query",
              "symctr_align", "symctr_contract",
              "symctr_contract_backward", "symctr_check_device_error", "symctr_profile_enable",
              "symctr_profile_read", "symctr_contract_static_scratch",
              "symctr_selftest_bounded_wait", "symctr_contract_complex",
              "symctr_plan_attach_tables", "symctr_plan_chain"):
        getattr(lib, f).restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(status: int):
    if status != 0:
        lib = load()
        raise SymctrError(status, lib.symctr_last_error_detail().decode())


def _arr(ctype, vals):
    vals = list(vals)
    return (ctype * max(len(vals), 1))(*vals)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass(frozen=True)
class SymSpec:
    """Conservation law of one operand: per-mode signs, remainder, block sizes;
    optionally (Eq. symtsr) the sector count H of each mode (coefficient
    sign * G / H; None: H = G) and the true size of each sector's block
    (non-uniform blocks padded to dims; None: uniform)."""
    signs: Tuple[int, ...]
    charge: Tuple[int, ...]
    dims: Tuple[int, ...]
    sectors: Optional[Tuple[int, ...]] = None
    sector_dims: Optional[Tuple[Tuple[int, ...], ...]] = None

    @property
    def general(self) -> bool:
        return self.sectors is not None or self.sector_dims is not None


def _spec(x) -> SymSpec:
    if isinstance(x, SymSpec):
        return x
    signs, charge, dims = x[:3]
    sectors = tuple(int(h) for h in x[3]) if len(x) > 3 and x[3] is not None else None
    sdims = (tuple(tuple(int(d) for d in m) for m in x[4])
             if len(x) > 4 and x[4] is not None else None)
    return SymSpec(tuple(int(s) for s in signs), tuple(int(c) for c in charge),
                   tuple(int(d) for d in dims), sectors, sdims)


def _operand(spec: SymSpec, keep: list) -> Operand:
    """symctr_operand for a spec (the arrays are kept alive in `keep`)."""
    arrs = [_arr(ctypes.c_int8, spec.signs), _arr(ctypes.c_int32, spec.charge),
            _arr(ctypes.c_int64, spec.dims),
            _arr(ctypes.c_int32, spec.sectors) if spec.sectors is not None else None,
            (_arr(ctypes.c_int64, [d for m in spec.sector_dims for d in m])
             if spec.sector_dims is not None else None)]
    keep.extend(a for a in arrs if a is not None)
    cast = lambda a, t: ctypes.cast(a, ctypes.POINTER(t)) if a is not None else None
    return Operand(cast(arrs[0], ctypes.c_int8), cast(arrs[1], ctypes.c_int32),
                   cast(arrs[2], ctypes.c_int64), cast(arrs[3], ctypes.c_int32),
                   cast(arrs[4], ctypes.c_int64))


class Plan:
    """A contraction plan W = einsum(spec, U, V) over Z_m1 x ... x Z_mr."""

    def __init__(self, einsum: str, moduli: Sequence[int], sym_u, sym_v, precision: str = "fp64",
                 n_slices: int = 0, sym_w=None):
        lib = load()
        self.einsum = einsum
        self.moduli = tuple(int(m) for m in moduli)
        self.sym_u, self.sym_v = _spec(sym_u), _spec(sym_v)
        self.precision = precision
        su, sv = self.sym_u, self.sym_v
        sw = _spec(sym_w) if sym_w is not None else None
        # the C ABI reads one entry per mode: check every spec against its operand
        lhs, lw_ = einsum.replace(" ", "").split("->") if "->" in einsum else (einsum, "")
        labels = lhs.split(",") + [lw_]
        for lab, sp, name in ((labels[0], su, "sym_u"), (labels[1] if len(labels) > 2 else "", sv, "sym_v"),
                              (labels[-1], sw, "sym_w")):
            if sp is None:
                continue
            if not (len(sp.signs) == len(sp.dims) == len(lab)) or len(sp.charge) != len(self.moduli):
                raise ValueError(f"{name}: {len(lab)} modes and {len(self.moduli)} moduli expected")
            if sp.sectors is not None and len(sp.sectors) != len(lab):
                raise ValueError(f"{name}: one sector count per mode expected")
            if sp.sector_dims is not None and len(sp.sector_dims) != len(lab):
                raise ValueError(f"{name}: one list of sector sizes per mode expected")
        handle = ctypes.c_void_p()
        if su.general or sv.general:
            keep = []
            ou, ov = _operand(su, keep), _operand(sv, keep)
            st = lib.symctr_plan_create_general(
                einsum.encode(), len(self.moduli), _arr(ctypes.c_int32, self.moduli),
                ctypes.byref(ou), ctypes.byref(ov),
                None if sw is None else _arr(ctypes.c_int8, sw.signs),
                None if sw is None else _arr(ctypes.c_int32, sw.charge),
                PRECISIONS[precision], int(n_slices), ctypes.byref(handle))
        else:
            st = lib.symctr_plan_create(
                einsum.encode(), len(self.moduli), _arr(ctypes.c_int32, self.moduli),
                _arr(ctypes.c_int8, su.signs), _arr(ctypes.c_int32, su.charge),
                _arr(ctypes.c_int8, sv.signs), _arr(ctypes.c_int32, sv.charge),
                _arr(ctypes.c_int64, su.dims), _arr(ctypes.c_int64, sv.dims),
                None if sw is None else _arr(ctypes.c_int8, sw.signs),
                None if sw is None else _arr(ctypes.c_int32, sw.charge),
                PRECISIONS[precision], int(n_slices), ctypes.byref(handle))
        _check(st)
        self._h = handle
        info = PlanInfo()
        _check(lib.symctr_plan_query(self._h, ctypes.byref(info)))
        self.info = info
        G = info.group_order
        general = bool(info.general)
        lhs, lw = einsum.replace(" ", "").split("->")
        lu, lv = lhs.split(",")

        def origin(c):   # the operand spec and mode a label of W comes from
            return (su, lu.index(c)) if c in lu else (sv, lv.index(c))
        sd_w = None
        if general and (su.sector_dims is not None or sv.sector_dims is not None):
            sd_w = tuple(tuple(sp.sector_dims[mu]) if sp.sector_dims is not None
                         else (sp.dims[mu],) * int(info.sectors_w[i])
                         for i, (sp, mu) in enumerate(origin(c) for c in lw))
        self.sym_w = SymSpec(tuple(info.signs_w[i] for i in range(info.order_w)),
                             tuple(info.charge_w[i] for i in range(info.n_moduli)),
                             tuple(info.dims_w[i] for i in range(info.order_w)),
                             tuple(info.sectors_w[i] for i in range(info.order_w)) if general else None,
                             sd_w)

        def shape(spec: SymSpec):
            n = len(spec.dims)
            hs = list(spec.sectors) if spec.sectors is not None else [G] * n
            return tuple(hs[:n - 1] + list(spec.dims)) if n else ()
        self.shape_u, self.shape_v, self.shape_w = shape(su), shape(sv), shape(self.sym_w)
        self._size_u, self._size_v, self._size_w = (torch.Size(self.shape_u), torch.Size(self.shape_v),
                                                     torch.Size(self.shape_w))
        self._ws = None
        self._tables = None
        self._tables_ready = info.table_bytes == 0
        self._lock = threading.Lock()
        # streams (other than the allocating one) on which the plan's device
        # buffers were used: the caching allocator waits for their work before
        # it reuses the memory of a freed buffer (Tensor.record_stream)
        self._seen = set()

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and _LIB is not None:
                # the device buffers (tables, workspace) are torch tensors whose
                # uses on other streams were recorded; nothing to wait for here
                _LIB.symctr_plan_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def _used_on(self, stream, *bufs):
        """Record that `bufs` (the plan's own buffers) are used on `stream`."""
        key = stream.cuda_stream
        if key in self._seen:
            return
        for b in bufs:
            if b is not None:
                b.record_stream(stream)
        self._seen.add(key)

    @staticmethod
    def _same_device(*ts):
        """All tensors on the current CUDA device (the library launches there)."""
        dev = torch.cuda.current_device()
        for t in ts:
            if t is not None and t.get_device() != dev:
                raise ValueError(f"tensor on cuda:{t.get_device()} but the current device is "
                                 f"cuda:{dev}; use torch.cuda.device(...) around the call")

    # -- contraction chains ------------------------------------------------
    def chain(self, u_from: "Optional[Plan]" = None, v_from: "Optional[Plan]" = None,
              w_aligned: bool = False) -> "Plan":
        """Keep intermediates aligned (symctr_plan_chain): with w_aligned the
        result is W_hat of shape (n_q, M, N), with no map back; u_from / v_from
        make U / V that plan's aligned result.  Call before the first
        contraction.  A chained plan has no backward."""
        _check(load().symctr_plan_chain(self._h, None if u_from is None else u_from._h,
                                        None if v_from is None else v_from._h, int(bool(w_aligned))))
        info = PlanInfo()
        _check(load().symctr_plan_query(self._h, ctypes.byref(info)))
        self.info = info
        aligned = lambda p: (int(p.info.n_q), int(p.info.M), int(p.info.N))
        if u_from is not None:
            self.shape_u = aligned(u_from)
        if v_from is not None:
            self.shape_v = aligned(v_from)
        if w_aligned:
            self.shape_w = aligned(self)
        self._size_u, self._size_v, self._size_w = (torch.Size(self.shape_u), torch.Size(self.shape_v),
                                                     torch.Size(self.shape_w))
        self._tables_ready = info.table_bytes == 0
        self._ws = None
        return self

    # -- device tables -------------------------------------------------------
    def attach_tables(self, device=None):
        """Give the plan a device copy of its offset tables (symctr_plan_attach_tables),
        so that its kernels read them from HBM instead of host memory.  The
        first contraction does this; the buffer lives as long as the plan."""
        with self._lock:
            if not self._tables_ready:
                buf = torch.empty(int(self.info.table_bytes), dtype=torch.uint8,
                                  device=device or "cuda")
                with torch.cuda.device(buf.device):
                    s = torch.cuda.current_stream(buf.device)
                    _check(load().symctr_plan_attach_tables(self._h, buf.data_ptr(), buf.numel(),
                                                            s.cuda_stream))
                    # contractions on other streams read the copy too
                    s.synchronize()
                self._tables = buf
                self._tables_ready = True
                self._seen = set()

    # -- workspace -----------------------------------------------------------
    def workspace(self, backward: bool = False, device=None) -> torch.Tensor:
        need = max(int(self.info.workspace_bytes), int(self.info.workspace_bytes_backward)
                   if backward else 0, 256)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=device or "cuda")
            self._seen = set()   # the new buffer's streams are recorded afresh
        return self._ws

    # -- checks --------------------------------------------------------------
    @staticmethod
    def _dev64(t: torch.Tensor, shape, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
            raise TypeError(f"{name} must be a float64 CUDA tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")

    # -- operations ------------------------------------------------------------
    def _ok64(self, t, size) -> bool:
        return (type(t) is torch.Tensor and t.dtype is torch.float64 and t.is_cuda
                and t.shape == size and t.is_contiguous())

    def contract(self, u: torch.Tensor, v: torch.Tensor, out: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        # one combined check on the common path; the detailed ones name the culprit
        if not (self._ok64(u, self._size_u) and self._ok64(v, self._size_v)):
            self._dev64(u, self.shape_u, "u")
            self._dev64(v, self.shape_v, "v")
        if out is None:
            out = torch.empty(self.shape_w, dtype=torch.float64, device=u.device)
        elif not self._ok64(out, self._size_w):
            self._dev64(out, self.shape_w, "out")
        self._same_device(u, v, out, workspace)
        if not self._tables_ready:
            self.attach_tables(u.device)
        ws = workspace if workspace is not None else self.workspace(device=u.device)
        cs = torch.cuda.current_stream()
        if cs.cuda_stream not in self._seen:
            self._used_on(cs, self._tables, self._ws)
        _check(_LIB.symctr_contract(self._h, u.data_ptr(), v.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                    ws.numel(), cs.cuda_stream))
        return out

    def contract_complex(self, u: torch.Tensor, v: torch.Tensor, out: Optional[torch.Tensor] = None,
                         conj_u: bool = False, conj_v: bool = False,
                         workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """W = einsum(op(U), op(V)) for complex128 reduced forms (op = conj where
        asked; the plan must carry the conjugated operand's negated law)."""
        for t, shape, name in ((u, self.shape_u, "u"), (v, self.shape_v, "v")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128):
                raise TypeError(f"{name} must be a complex128 CUDA tensor")
            if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}")
        if out is None:
            out = torch.empty(self.shape_w, dtype=torch.complex128, device=u.device)
        if out.dtype != torch.complex128 or tuple(out.shape) != tuple(self.shape_w) or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex128 tensor of the output shape")
        self._same_device(u, v, out, workspace)
        if not self._tables_ready:
            self.attach_tables(u.device)
        ws = workspace if workspace is not None else self.workspace(device=u.device)
        self._used_on(torch.cuda.current_stream(), self._tables, self._ws)
        _check(load().symctr_contract_complex(self._h, int(conj_u), int(conj_v), _ptr(u), _ptr(v),
                                              _ptr(out), _ptr(ws), ws.numel(), _stream()))
        return out

    def contract_static_scratch(self, u: torch.Tensor, v: torch.Tensor,
                                out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """contract() for callers that cannot allocate device scratch: the library
        uses its own static 64 MiB device array instead of a workspace.  Calls
        share that array, so they must not overlap on the GPU (use one stream).
        `out` must be preallocated by such callers (this convenience wrapper
        allocates it with torch only when it is omitted)."""
        self._dev64(u, self.shape_u, "u")
        self._dev64(v, self.shape_v, "v")
        if out is None:
            out = torch.empty(self.shape_w, dtype=torch.float64, device=u.device)
        self._dev64(out, self.shape_w, "out")
        # the library picks the static array of the current device: every
        # tensor must live there
        self._same_device(u, v, out)
        # no table buffer is attached here (that would allocate device memory);
        # tables attached by an earlier contract() are used
        if self._tables is not None:
            self._used_on(torch.cuda.current_stream(), self._tables)
        _check(load().symctr_contract_static_scratch(self._h, _ptr(u), _ptr(v), _ptr(out),
                                                     _stream()))
        return out

    def check_static_scratch_error(self):
        """Read and clear the device error word of contract_static_scratch's static
        array on the current device (synchronises the current stream)."""
        _check(load().symctr_check_device_error(self._h, None, _stream()))

    def backward(self, grad_w: torch.Tensor, u: torch.Tensor, v: torch.Tensor,
                 need_u: bool = True, need_v: bool = True,
                 workspace: Optional[torch.Tensor] = None):
        self._dev64(grad_w, self.shape_w, "grad_w")
        self._same_device(grad_w, u, v, workspace)
        gu = torch.empty(self.shape_u, dtype=torch.float64, device=u.device) if need_u else None
        gv = torch.empty(self.shape_v, dtype=torch.float64, device=u.device) if need_v else None
        if not self._tables_ready:
            self.attach_tables(u.device)
        ws = workspace if workspace is not None else self.workspace(True, u.device)
        self._used_on(torch.cuda.current_stream(), self._tables, self._ws)
        _check(load().symctr_contract_backward(self._h, _ptr(grad_w), _ptr(u), _ptr(v), _ptr(gu),
                                               _ptr(gv), _ptr(ws), ws.numel(), _stream()))
        return gu, gv

    def align(self, operand: int, direction: int, src: torch.Tensor) -> torch.Tensor:
        """Bit-exact alignment transforms (operand 0=U, 1=V, 2=W; direction +1 std->aligned)."""
        i = self.info
        red = [self.shape_u, self.shape_v, self.shape_w][operand]
        al = [(i.n_q, i.M, i.K), (i.n_q, i.N, i.K), (i.n_q, i.M, i.N)][operand]
        src_shape, dst_shape = (red, al) if direction > 0 else (al, red)
        self._dev64(src, src_shape, "src")
        self._same_device(src)
        dst = torch.empty(dst_shape, dtype=torch.float64, device=src.device)
        _check(load().symctr_align(self._h, operand, direction, _ptr(src), _ptr(dst), _stream()))
        return dst

    def check_device_error(self, workspace: Optional[torch.Tensor] = None):
        ws = workspace if workspace is not None else self._ws
        if ws is None:
            return
        _check(load().symctr_check_device_error(self._h, _ptr(ws), _stream()))

    def profile(self, enable: bool = True):
        """Record CUDA events around the operand preparation and the GEMM of
        each later contract() call (see phase_times)."""
        _check(load().symctr_profile_enable(self._h, int(enable)))

    def phase_times(self):
        """(prep_ms, gemm_ms, kernels launched) of the last contract() call."""
        a, b, n = ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
        _check(load().symctr_profile_read(self._h, ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(n)))
        return a.value, b.value, n.value

    @property
    def useful_flops(self) -> float:
        return float(self.info.useful_flops)

    def q_values(self):
        """The irrep of each batch of the aligned forms."""
        i = self.info
        if i.n_q == 0:
            return []
        if i.n_q == 1:
            return [i.q_single]
        return [(i.q_first + b * i.q_step) % i.group_order for b in range(i.n_q)]


class SymContract(torch.autograd.Function):
    """W = plan(U, V) with the hand-written adjoint: gU = gW.V and gV = U.gW
    as irrep-aligned contractions (aligned operands recomputed, never saved)."""

    @staticmethod
    def forward(ctx, plan: Plan, u: torch.Tensor, v: torch.Tensor):
        ctx.plan = plan
        ctx.save_for_backward(u, v)
        return plan.contract(u.contiguous(), v.contiguous())

    @staticmethod
    def backward(ctx, gw):
        u, v = ctx.saved_tensors
        plan = ctx.plan
        gu, gv = plan.backward(gw.contiguous(), u.contiguous(), v.contiguous(),
                               ctx.needs_input_grad[1], ctx.needs_input_grad[2])
        return None, gu, gv


def contract(plan: Plan, u: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """Differentiable contraction through the plan."""
    return SymContract.apply(plan, u, v)


def selftest_bounded_wait(workspace: torch.Tensor, wait_cycles: int = 2_000_000) -> None:
    """Launch the failure-detection self-test on the current stream: a kernel
    whose bounded wait on a barrier nothing completes gives up after
    `wait_cycles` cycles and records the timeout in `workspace`'s error word
    (read it with Plan.check_device_error)."""
    if not (isinstance(workspace, torch.Tensor) and workspace.is_cuda):
        raise TypeError("workspace must be a CUDA tensor")
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().symctr_selftest_bounded_wait(_ptr(workspace), nbytes, int(wait_cycles), _stream()))


def einsum(spec: str, u: torch.Tensor, v: torch.Tensor, moduli, sym_u, sym_v,
           precision: str = "fp64") -> torch.Tensor:
    """One-shot convenience: plan + differentiable contraction."""
    return contract(Plan(spec, moduli, sym_u, sym_v, precision), u, v)


__all__ = ["Plan", "PlanInfo", "SymSpec", "SymContract", "SymctrError", "contract", "einsum",
           "load", "library_path", "PRECISIONS", "selftest_bounded_wait"]
