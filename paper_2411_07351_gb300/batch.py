"""Batched transforms through fht_submit: many images of uneven sizes in one
persistent launch.  PyTorch allocates the outputs and workspaces; the
persistent kernel does all the work."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _capi as C
from .fht import Plan, PlanCache


# Launch shape of plans made for batched launches: 64-column tiles keep the
# persistent kernel at 3 CTAs per SM (<= 64 KB of shared memory per CTA) and
# fit the small images batches are for.  (Plans with the register-tiled shape,
# tile 192 x 256 threads with 32-column generic tiles, also run in a batch;
# measured on the 4096-map batch they were slower: graph replay 26.2 vs
# 23.5 ms, a 192-column register tile costing the same however few of its
# columns a narrow image fills.)
BATCH_TILE_COLS = 64
BATCH_THREADS = 0
BATCH_GENERIC_COLS = 0

# numpy layout of fht_job (include/fht.h): 64 bytes, naturally aligned fields
_JOB_DTYPE = np.dtype([("plan", np.uint64), ("d_in", np.uint64), ("in_pitch", np.int64), ("d_out", np.uint64),
                       ("d_ws", np.uint64), ("ws_bytes", np.uint64), ("tag", np.uint64), ("flags", np.uint32),
                       ("reserved", np.uint32)])
assert _JOB_DTYPE.itemsize == ctypes.sizeof(C.fht_job)


class BatchQueue:
    """One fht_queue_t: device tables for up to max_jobs jobs / max_units units per submit."""

    def __init__(self, device: int | None = None, max_jobs: int = 8192, max_units: int = 1 << 22,
                 shape: tuple[int, int, int] | None = None):
        """`shape` = (tile_cols, threads, generic_cols) of the plans this queue
        makes (0 = default); None takes the batch defaults above (see
        ``tune.tune_batch`` for choosing one by measurement)."""
        self.shape = tuple(shape) if shape is not None else (BATCH_TILE_COLS, BATCH_THREADS, BATCH_GENERIC_COLS)
        self._lib = C.load()
        self.device_index = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        C.check(self._lib.fht_queue_create(ctypes.byref(h), self.device_index, max_jobs, max_units),
                "fht_queue_create")
        self._q = h
        self.plans = PlanCache(capacity=4096)
        self._keep = []  # buffers of the last submit

    def set_wait_limit(self, seconds: float):
        C.check(self._lib.fht_queue_set_wait_limit(self._q, int(seconds * 1e9)), "fht_queue_set_wait_limit")

    def plan_for(self, x: torch.Tensor, quads: int, boundary: str, split: str) -> Plan:
        tc, th, gc = self.shape
        return self.plans.get(x.shape[0], x.shape[1], x.dtype, quads, boundary, split, self.device_index,
                              tile_cols=tc, threads=th, generic_cols=gc)

    def submit(self, images, quads: int = C.FHT_QALL, boundary: str = "cyclic", split: str = "T",
               outs=None, workspaces=None, stream=None, flags=None, tags=None, plans=None):
        """Enqueue one persistent launch over `images` (2-D CUDA tensors of one dtype).

        `plans` may give each image's plan (made by the caller for that shape,
        quadrants, boundary and split); otherwise they come from this queue's cache.
        Returns (outputs, plans, workspaces); outputs are the packed quadrants of each image."""
        n = len(images)
        if plans is None:
            plans = [self.plan_for(x, quads, boundary, split) for x in images]
        if outs is None:
            outs = [p.new_output() for p in plans]
        if workspaces is None:
            workspaces = [p.new_workspace() for p in plans]
        if any(x.stride(1) != 1 for x in images):
            raise ValueError("images must have unit column stride")
        # the fht_job array, column by column (numpy view of the C struct layout)
        jobs = np.zeros(n, dtype=_JOB_DTYPE)
        jobs["plan"] = [p._h.value for p in plans]
        jobs["d_in"] = [x.data_ptr() for x in images]
        jobs["in_pitch"] = [x.stride(0) for x in images]
        jobs["d_out"] = [o.data_ptr() for o in outs]
        jobs["d_ws"] = [w.data_ptr() for w in workspaces]
        jobs["ws_bytes"] = [w.numel() * w.element_size() for w in workspaces]
        jobs["tag"] = np.arange(n) if tags is None else tags
        if flags is not None:
            jobs["flags"] = flags
        s = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", self.device_index))
        C.check(self._lib.fht_submit(self._q, n, jobs.ctypes.data_as(ctypes.POINTER(C.fht_job)), int(s.cuda_stream)),
                "fht_submit")
        self._keep = [images, outs, workspaces, plans]
        return outs, plans, workspaces

    def ready(self) -> bool:
        """True when a submit would not wait on the host for this queue's
        staging buffers (the previous submit's table copies have run)."""
        r = ctypes.c_int32()
        C.check(self._lib.fht_queue_ready(self._q, ctypes.byref(r)), "fht_queue_ready")
        return bool(r.value)

    def status(self, stream=None) -> int:
        s = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", self.device_index))
        return int(self._lib.fht_queue_status(self._q, int(s.cuda_stream)))

    def reset_status(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", self.device_index))
        C.check(self._lib.fht_queue_reset_status(self._q, int(s.cuda_stream)), "fht_queue_reset_status")

    def poll(self, cap: int = 4096) -> list[int]:
        buf = (ctypes.c_uint64 * cap)()
        n = ctypes.c_int32()
        C.check(self._lib.fht_queue_poll(self._q, buf, cap, ctypes.byref(n)), "fht_queue_poll")
        return [int(buf[i]) for i in range(n.value)]

    def close(self):
        if getattr(self, "_q", None):
            self._lib.fht_queue_destroy(self._q)
            self._q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
