"""GPU tests of the host-memory pipeline (fht_pipe_*): every submit's output,
copied back to host memory, equals the oracle's transform of its image."""
import numpy as np
import pytest
import torch

from paper_2411_07351_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07351_gb300 import build as B

    B.build()
    import paper_2411_07351_gb300 as F

    return F


@pytest.mark.parametrize("depth,copies", [(1, 1), (2, 2), (3, 4)])
def test_pipeline_outputs_match_oracle(F, orc, depth, copies):
    h, w = 300, 211
    p = F.Plan(h, w, torch.uint8, 15, "extended")
    pipe = F.HostPipeline(p, depth=depth, copy_streams=copies)
    imgs = [inputs.uniform_u8(50 + i, h, w) for i in range(7)]
    ins = [torch.from_numpy(im).pin_memory() for im in imgs]
    outs = [torch.full((p.out_elems,), -1, dtype=torch.int32).pin_memory() for _ in imgs]
    for a, b in zip(ins, outs):
        pipe.submit(a, b)
    pipe.synchronize()
    for im, o in zip(imgs, outs):
        assert np.array_equal(o.numpy().astype(np.int64), orc.fht(im.astype(np.int64), 15, orc.EXTENDED))
    pipe.close()


def test_pipeline_pitched_and_pageable(F, orc):
    # a pitched host view, pageable output memory
    h, w = 129, 77
    img = inputs.normal_f32(9, h, w)
    big = torch.zeros((h, 96), dtype=torch.float32)
    big[:, :w] = torch.from_numpy(img)
    view = big[:, :w]
    p = F.Plan(h, w, torch.float32, 15, "cyclic")
    pipe = F.HostPipeline(p)
    out = torch.zeros(p.out_elems, dtype=torch.float32)
    pipe.submit(view, out)
    pipe.synchronize()
    ref = p.forward(torch.from_numpy(img).cuda()).cpu()
    assert torch.equal(out, ref)
    pipe.close()


def test_pipeline_rejects_bad_arguments(F):
    p = F.Plan(16, 16, torch.uint8, 1, "cyclic")
    pipe = F.HostPipeline(p)
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros((16, 16), dtype=torch.float32), torch.zeros(p.out_elems, dtype=torch.int32))
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros((16, 16), dtype=torch.uint8).cuda(), torch.zeros(p.out_elems, dtype=torch.int32))
    pipe.close()
