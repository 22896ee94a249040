"""Run the forward transform a few times on a seeded image, for profilers.

    python -m paper_2411_07351_gb300.profile_forward --h 2048 --w 2048 --reps 3

Each rep launches the plan's kernels once (fused pass, then the band pass and
the spine launches, or one pass per upper tree height); with --adjoint each
rep also runs the adjoint (one pass per upper tree height, highest first, the
fused subtrees in reverse, the sum of the quadrants' gradients).  Nothing is
timed here; use it under ncu.
"""
import argparse
import ctypes

import torch

import paper_2411_07351_gb300 as F
from paper_2411_07351_gb300 import inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--h", type=int, default=2048)
    ap.add_argument("--w", type=int, default=2048)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--dtype", choices=["f32", "u8"], default="f32")
    ap.add_argument("--boundary", choices=["cyclic", "extended"], default="extended")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--quads", type=int, default=15, help="quadrant mask (1 = Q0 ... 15 = all four)")
    ap.add_argument("--tile-cols", type=int, default=0, help="column tile (0: the library default)")
    ap.add_argument("--threads", type=int, default=0, help="CTA size of the fused pass (0: default)")
    a = ap.parse_args()
    if a.dtype == "f32":
        x = torch.from_numpy(inputs.normal_f32(2, a.h, a.w)).cuda()
    else:
        x = torch.from_numpy(inputs.uniform_u8(2, a.h, a.w)).cuda()
    p = F.Plan(a.h, a.w, x.dtype, a.quads, a.boundary, with_adjoint=a.adjoint, tile_cols=a.tile_cols,
               threads=a.threads)
    out, ws = p.new_output(), p.new_workspace(adjoint=a.adjoint)
    gin = torch.empty((a.h, a.w), dtype=p.out_dtype, device="cuda") if a.adjoint else None
    for _ in range(a.reps):
        p.forward(x, out, ws)
        if a.adjoint:
            p.adjoint(out, gin, ws)
    torch.cuda.synchronize()
    from paper_2411_07351_gb300 import _capi

    n = ctypes.c_int32()
    _capi.check(_capi.load().fht_plan_launches(p._h, ctypes.byref(n)), "fht_plan_launches")
    print(f"ok {a.h}x{a.w} {a.dtype} {a.boundary}: launches per forward = {n.value}, "
          f"model bytes = {p.info.model_bytes}")


if __name__ == "__main__":
    main()
