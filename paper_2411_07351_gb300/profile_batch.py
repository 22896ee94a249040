"""Run batched submits of seeded binary edge maps (h, w ~ U{17..511}), for profilers.

    python -m paper_2411_07351_gb300.profile_batch --images 256 --reps 3
"""
import argparse

import torch

import paper_2411_07351_gb300 as F
from paper_2411_07351_gb300 import inputs
from paper_2411_07351_gb300.batch import BatchQueue


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--images", type=int, default=256)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    xs = [torch.from_numpy(im).cuda() for im in inputs.c3_batch(count=a.images)]
    q = BatchQueue(max_jobs=a.images, max_units=1 << 22)
    plans = [q.plan_for(x, F.FHT_QALL, "cyclic", "T") for x in xs]
    outs = [p.new_output() for p in plans]
    wss = [p.new_workspace() for p in plans]
    for _ in range(a.reps):
        q.submit(xs, F.FHT_QALL, "cyclic", "T", outs=outs, workspaces=wss)
    torch.cuda.synchronize()
    assert q.status() == 0
    print(f"ok {a.images} images, {sum(x.numel() for x in xs) / 1e6:.1f} Mpix")
    q.close()


if __name__ == "__main__":
    main()
