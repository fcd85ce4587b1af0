"""Pipelined end-to-end rendering (Renderer.render_sequence_to_host): every view's image must
reach the host intact although the copy of view i overlaps the rendering of view i + 1 and two
device and host buffers are reused in turn.  Each host image is compared bit for bit with a
separate single-view render of the same pose."""
import numpy as np
import pytest

import synth
from gpu_helpers import lib_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


@pytest.mark.parametrize("n", [1, 2, 5])
def test_sequence_to_host_matches_single_renders(abi, n):
    import torch
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    rd = Renderer(sc, mlp, cams[0].W, cams[0].H, sel_cap=200_000, pair_cap=4_000_000,
                  precision="bf16")
    poses = [(17 * i + 3) % len(cams) for i in range(n)]
    hosts = [torch.empty(3, rd.H, rd.W, pin_memory=True) for _ in range(2)]
    got = {}
    rd.render_sequence_to_host([cams[p] for p in poses], hosts,
                               on_frame=lambda i, h: got.__setitem__(i, h.numpy().copy()))
    assert sorted(got) == list(range(n))
    for i, p in enumerate(poses):
        c = rd.render(cams[p])
        assert c.overflow == 0 and c.timeout == 0
        assert np.array_equal(got[i], rd.img.cpu().numpy()), i
