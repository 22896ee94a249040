"""The paper's experiments, on the GPU.

* ``pattern_errors``: Section 5's accuracy experiment -- E_S(n), E_T(n) for a
  range of n, every pattern of Algorithm 2 generated (fht_pattern_errors).
* ``summary``: the aggregates Section 5 prints, recomputed from those errors
  (share of n where the Theorem 2 bound lies below E_S, the largest E_S/E_T
  and where, the E_S peak sizes).
* ``addition_counts``: Theorem 1's counts from the plan builder (host).
"""
from __future__ import annotations

import math

import torch

from . import _capi as C


def pattern_errors(n_lo: int, n_hi: int, split: str = "T", device: int | None = None) -> list[int]:
    """Exact numerators num(n) with E(n) = num(n) / (n - 1), for n in [n_lo, n_hi]."""
    lib = C.load()
    dev = torch.cuda.current_device() if device is None else device
    out = torch.empty(n_hi - n_lo + 1, dtype=torch.int64, device=f"cuda:{dev}")
    s = torch.cuda.current_stream(torch.device("cuda", dev))
    C.check(lib.fht_pattern_errors(n_lo, n_hi, C.FHT_SPLIT_S if split == "S" else C.FHT_SPLIT_T, out.data_ptr(),
                                   s.cuda_stream), "fht_pattern_errors")
    return [int(v) for v in out.cpu().tolist()]


def summary(num_s: list[int], num_t: list[int], n_lo: int = 1) -> dict:
    """Section 5's printed aggregates from the error numerators of n = n_lo, n_lo + 1, ..."""
    n = list(range(n_lo, n_lo + len(num_s)))
    es = [a / (k - 1) if k > 1 else 0.0 for a, k in zip(num_s, n)]
    et = [a / (k - 1) if k > 1 else 0.0 for a, k in zip(num_t, n)]
    bound = [math.floor(math.log2(k)) / 6 + 1 - 2.0 ** (-math.floor(math.log2(k))) for k in n]
    below = sum(1 for b, e in zip(bound, es) if b < e)
    ratios = [(s_ / t_, k) for s_, t_, k in zip(es, et, n) if t_ > 0]
    r, at = max(ratios)
    return {"share_bound_below_E_S_pct": 100.0 * below / len(n), "max_E_S_over_E_T": r, "at_n": at,
            "E_T_within_theorem2": all(e <= b + 1e-12 for e, b in zip(et, bound))}


def addition_counts(n: int, split: str = "T") -> int:
    """f(n) of Theorem 1 (one quadrant, cyclic, n x n) from the plan builder."""
    from .fht import Plan

    p = Plan(n, n, torch.float32, C.FHT_Q0, "cyclic", split, device=-1)
    adds = int(p.info.adds)
    p.close()
    return adds
