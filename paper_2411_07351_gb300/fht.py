"""Python face of libfht.so.

PyTorch supplies device memory and streams; every step of the transform runs
in the library's CUDA kernels.  ``Plan`` owns one ``fht_plan_t``.
"""
from __future__ import annotations

import ctypes
import threading
from collections import OrderedDict

import torch

from . import _capi as C

DTYPES = {  # torch input dtype -> (fht_dtype, output dtype)
    torch.uint8: (C.FHT_U8_I32, torch.int32),
    torch.int32: (C.FHT_I32_I32, torch.int32),
    torch.float32: (C.FHT_F32_F32, torch.float32),
    torch.float64: (C.FHT_F64_F64, torch.float64),
}
BOUNDARY = {"cyclic": C.FHT_CYCLIC, "extended": C.FHT_EXTENDED}
SPLIT = {"T": C.FHT_SPLIT_T, "S": C.FHT_SPLIT_S}


def _stream_handle(device: torch.device, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


class Plan:
    """A transform plan for one (h, w, dtype, quadrants, boundary, split).

    ``device`` is a CUDA device index, or -1 for a host-only plan (sizes,
    tables and the byte model; cannot run).
    """

    def __init__(self, h: int, w: int, dtype=torch.float32, quads: int = C.FHT_QALL,
                 boundary: str = "cyclic", split: str = "T", device: int | None = None,
                 fused_rows: int = 0, tile_cols: int = 0, threads: int = 0, with_adjoint: bool = False,
                 tuning: str | None = None, rounding: str = "exact", spine_chunk: int = 0, generic_cols: int = 0):
        self._lib = C.load()
        if tuning == "auto" and not (tile_cols or threads):
            from .tune import lookup

            best = lookup(h, w, dtype, quads, boundary, split)
            if best:
                tile_cols, threads = int(best["tile_cols"]), int(best["threads"])
                if not fused_rows:
                    fused_rows = int(best.get("fused_rows", 0))
        if dtype not in DTYPES:
            raise ValueError(f"unsupported dtype {dtype}")
        self.h, self.w = int(h), int(w)
        self.in_dtype = dtype
        self.fht_dtype, self.out_dtype = DTYPES[dtype]
        self.quads = int(quads)
        self.boundary = boundary
        self.split = split
        if device is None:
            device = torch.cuda.current_device()
        self.device_index = int(device)
        if rounding not in ("exact", "float"):
            raise ValueError("rounding is 'exact' or 'float'")
        tun = C.fht_tuning_t(fused_rows, tile_cols, threads, int(with_adjoint), 1 if rounding == "float" else 0,
                             int(spine_chunk), int(generic_cols))
        handle = ctypes.c_void_p()
        args = (ctypes.byref(handle), self.h, self.w, self.fht_dtype, self.quads, BOUNDARY[boundary], SPLIT[split],
                self.device_index, ctypes.byref(tun))
        st = self._lib.fht_plan(*args)
        if st == C.FHT_ERR_NOMEM and self.device_index >= 0:
            # the plan's tables are allocated outside PyTorch: give back cached blocks once
            torch.cuda.empty_cache()
            st = self._lib.fht_plan(*args)
        C.check(st, "fht_plan")
        self._h = handle
        self._read_info()

    @classmethod
    def adopt(cls, handle, h: int, w: int, dtype, quads: int, boundary: str, split: str, device: int) -> "Plan":
        """Wrap a plan handle built elsewhere (``PlanBuilderPool``); the Plan owns it from now on."""
        self = cls.__new__(cls)
        self._lib = C.load()
        self.h, self.w = int(h), int(w)
        self.in_dtype = dtype
        self.fht_dtype, self.out_dtype = DTYPES[dtype]
        self.quads, self.boundary, self.split = int(quads), boundary, split
        self.device_index = int(device)
        self._h = handle
        self._read_info()
        return self

    def _read_info(self):
        info = C.fht_plan_info_t()
        C.check(self._lib.fht_plan_info(self._h, ctypes.byref(info)), "fht_plan_info")
        self.info = info
        self.out_elems = int(info.out_elems)
        self.workspace_bytes = int(info.workspace_bytes)
        self.adjoint_workspace_bytes = int(info.adjoint_workspace_bytes)
        self.shapes = [(int(info.rows[q]), int(info.cols[q])) for q in range(4) if self.quads & (1 << q)]
        self.offsets = [int(info.out_offset[q]) for q in range(4) if self.quads & (1 << q)]

    @property
    def device(self) -> torch.device:
        return torch.device("cuda", self.device_index)

    def check(self):
        C.check(self._lib.fht_plan_check(self._h), "fht_plan_check")

    def new_workspace(self, adjoint: bool = False) -> torch.Tensor:
        # 256-byte alignment: the caching allocator returns 512-byte aligned blocks
        nbytes = self.adjoint_workspace_bytes if adjoint else self.workspace_bytes
        return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)

    def new_output(self) -> torch.Tensor:
        return torch.empty(self.out_elems, dtype=self.out_dtype, device=self.device)

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        if x.dtype != self.in_dtype or x.dim() != 2 or tuple(x.shape) != (self.h, self.w):
            raise ValueError(f"expected a {self.h}x{self.w} {self.in_dtype} tensor, got {tuple(x.shape)} {x.dtype}")
        if not x.is_cuda or x.device.index != self.device_index:
            raise ValueError("input must live on the plan's CUDA device")
        if x.stride(1) != 1:
            x = x.contiguous()
        if out is None:
            out = self.new_output()
        if ws is None:
            ws = self.new_workspace()
        if out.numel() < self.out_elems or out.dtype != self.out_dtype or not out.is_contiguous():
            raise ValueError("output buffer has the wrong size, dtype or layout")
        C.check(self._lib.fht_forward(self._h, x.data_ptr(), x.stride(0), out.data_ptr(), ws.data_ptr(),
                                      ws.numel() * ws.element_size(), _stream_handle(x.device, stream)),
                "fht_forward")
        return out

    def _refresh_info(self):
        info = C.fht_plan_info_t()
        C.check(self._lib.fht_plan_info(self._h, ctypes.byref(info)), "fht_plan_info")
        self.info = info

    def adjoint(self, gout: torch.Tensor, gin: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        if gout.dtype != self.out_dtype or gout.numel() != self.out_elems or not gout.is_contiguous():
            raise ValueError("gout must be a contiguous tensor of out_elems elements of the output dtype")
        if gin is None:
            gin = torch.empty((self.h, self.w), dtype=self.out_dtype, device=self.device)
        if ws is None:
            ws = self.new_workspace(adjoint=True)
        C.check(self._lib.fht_adjoint(self._h, gout.data_ptr(), gin.data_ptr(), gin.stride(0), ws.data_ptr(),
                                      ws.numel() * ws.element_size(), _stream_handle(gout.device, stream)),
                "fht_adjoint")
        return gin

    def unpack(self, out: torch.Tensor) -> list[torch.Tensor]:
        return [out[o:o + n * c].view(n, c) for (n, c), o in zip(self.shapes, self.offsets)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fht_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipeline:
    """Transforms of images held in host memory (fht_pipe_*): every submit
    copies the image in, transforms it and copies the packed output back,
    overlapping with the neighbouring submits.  Host tensors should be
    pinned (``tensor.pin_memory()``) for the copies to run asynchronously;
    they must stay alive and unchanged until ``synchronize`` returns."""

    def __init__(self, plan: Plan, depth: int = 2, copy_streams: int = 2):
        self.plan = plan
        self._lib = plan._lib
        h = ctypes.c_void_p()
        st = self._lib.fht_pipe_create(ctypes.byref(h), plan._h, depth, copy_streams)
        if st == C.FHT_ERR_NOMEM:
            torch.cuda.empty_cache()  # the pipe allocates outside PyTorch
            st = self._lib.fht_pipe_create(ctypes.byref(h), plan._h, depth, copy_streams)
        C.check(st, "fht_pipe_create")
        self._h = h
        self._keep: list = []

    def submit(self, host_in: torch.Tensor, host_out: torch.Tensor):
        p = self.plan
        if host_in.is_cuda or host_out.is_cuda:
            raise ValueError("HostPipeline takes host tensors")
        if host_in.dtype != p.in_dtype or tuple(host_in.shape) != (p.h, p.w) or host_in.stride(1) != 1:
            raise ValueError(f"expected a {p.h}x{p.w} {p.in_dtype} host tensor with unit column stride")
        if host_out.dtype != p.out_dtype or host_out.numel() < p.out_elems or not host_out.is_contiguous():
            raise ValueError("host output has the wrong size, dtype or layout")
        C.check(self._lib.fht_pipe_submit(self._h, host_in.data_ptr(), host_in.stride(0), host_out.data_ptr()),
                "fht_pipe_submit")
        self._keep.append((host_in, host_out))

    def synchronize(self):
        C.check(self._lib.fht_pipe_sync(self._h), "fht_pipe_sync")
        self._keep.clear()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fht_pipe_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlanBuilderPool:
    """Plans built on the library's native worker threads (``fht_builder_*``):
    ``submit`` returns at once with a tag, ``poll`` returns the builds that
    have finished since, as (tag, Plan) or (tag, FHTError).  No interpreter
    thread takes part in building, so a serving loop keeps the interpreter
    lock to itself."""

    def __init__(self, threads: int = 8, poll_cap: int = 1024):
        self._lib = C.load()
        b = ctypes.c_void_p()
        C.check(self._lib.fht_builder_create(ctypes.byref(b), int(threads)), "fht_builder_create")
        self._b = b
        self._meta: dict = {}
        self._next = 1
        self._cap = poll_cap
        self._tags = (ctypes.c_uint64 * poll_cap)()
        self._plans = (ctypes.c_void_p * poll_cap)()
        self._status = (ctypes.c_int * poll_cap)()
        self._n = ctypes.c_int32()

    def submit(self, h: int, w: int, dtype, quads: int = C.FHT_QALL, boundary: str = "cyclic", split: str = "T",
               device: int | None = None, tile_cols: int = 0, threads: int = 0, generic_cols: int = 0) -> int:
        if device is None:
            device = torch.cuda.current_device()
        tag = self._next
        self._next += 1
        tun = C.fht_tuning_t(0, int(tile_cols), int(threads), 0, 0, 0, int(generic_cols))
        C.check(self._lib.fht_builder_submit(self._b, tag, int(h), int(w), DTYPES[dtype][0], int(quads),
                                             BOUNDARY[boundary], SPLIT[split], int(device), ctypes.byref(tun)),
                "fht_builder_submit")
        self._meta[tag] = (int(h), int(w), dtype, int(quads), boundary, split, int(device))
        return tag

    def poll(self) -> list:
        C.check(self._lib.fht_builder_poll(self._b, self._tags, self._plans, self._status, self._cap,
                                           ctypes.byref(self._n)), "fht_builder_poll")
        out = []
        for k in range(self._n.value):
            tag = int(self._tags[k])
            meta = self._meta.pop(tag)
            if self._status[k] == C.FHT_OK:
                out.append((tag, Plan.adopt(ctypes.c_void_p(self._plans[k]), *meta)))
            else:
                out.append((tag, C.FHTError(int(self._status[k]), f"plan build {meta[:2]}")))
        return out

    def pending(self) -> tuple[int, int]:
        q, f = ctypes.c_int32(), ctypes.c_int32()
        C.check(self._lib.fht_builder_pending(self._b, ctypes.byref(q), ctypes.byref(f)), "fht_builder_pending")
        return q.value, f.value

    def close(self):
        if getattr(self, "_b", None):
            self._lib.fht_builder_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlanCache:
    """Least-recently-used cache of plans keyed by their full configuration."""

    def __init__(self, capacity: int = 64):
        self.capacity = capacity
        self._d: OrderedDict = OrderedDict()
        self._lock = threading.Lock()

    def get(self, h, w, dtype, quads, boundary, split, device, tile_cols: int = 0, threads: int = 0,
            generic_cols: int = 0) -> Plan:
        key = (h, w, dtype, quads, boundary, split, device, tile_cols, threads, generic_cols)
        with self._lock:
            p = self._d.get(key)
            if p is not None:
                self._d.move_to_end(key)
                return p
        p = Plan(h, w, dtype, quads, boundary, split, device, tile_cols=tile_cols, threads=threads,
                 generic_cols=generic_cols)
        with self._lock:
            self._d[key] = p
            while len(self._d) > self.capacity:
                # dropped, not closed: autograd graphs may still hold the plan
                self._d.popitem(last=False)
        return p


_cache = PlanCache()


def forward(x: torch.Tensor, quads: int = C.FHT_QALL, boundary: str = "cyclic", split: str = "T") -> torch.Tensor:
    """FHT of one 2-D image tensor on its CUDA device; returns the packed quadrants."""
    plan = _cache.get(x.shape[0], x.shape[1], x.dtype, quads, boundary, split, x.device.index)
    return plan.forward(x)
