"""End-to-end rendering into pinned host memory: Renderer.render_sequence_to_host, pipelined
either by writing each image straight into its host buffer from the blend (zero copy) or by
copying view i while view i + 1 renders (consecutive views on two compute streams with two
sets of per-view buffers), two host buffers reused in turn; and the single-view
render_to_host in both forms.  Each host image is compared bit for bit with a separate
single-view render of the same pose on the device."""
import numpy as np
import pytest

import synth
from gpu_helpers import lib_ready

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


@pytest.mark.parametrize("zero_copy", [True, False])
@pytest.mark.parametrize("n", [1, 2, 5])
def test_sequence_to_host_matches_single_renders(abi, n, zero_copy):
    import torch
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    rd = Renderer(sc, mlp, cams[0].W, cams[0].H, sel_cap=200_000, pair_cap=4_000_000,
                  precision="bf16")
    poses = [(17 * i + 3) % len(cams) for i in range(n)]
    hosts = [torch.empty(3, rd.H, rd.W, pin_memory=True) for _ in range(2)]
    got = {}
    rd.render_sequence_to_host([cams[p] for p in poses], hosts,
                               on_frame=lambda i, h: got.__setitem__(i, h.numpy().copy()),
                               zero_copy=zero_copy)
    assert sorted(got) == list(range(n))
    c = rd.counts()                    # both buffer sets of the pipelined form
    assert c.overflow == 0 and c.timeout == 0
    for i, p in enumerate(poses):
        c = rd.render(cams[p])
        assert c.overflow == 0 and c.timeout == 0
        assert np.array_equal(got[i], rd.img.cpu().numpy()), i


@pytest.mark.parametrize("zero_copy", [True, False])
def test_render_to_host_matches_device_render(abi, zero_copy):
    import torch
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    rd = Renderer(sc, mlp, cams[0].W, cams[0].H, sel_cap=200_000, pair_cap=4_000_000,
                  precision="bf16")
    host = torch.full((3, rd.H, rd.W), -1.0, pin_memory=True)
    for p in (5, 61):
        rd.render_to_host(cams[p], host, zero_copy=zero_copy)
        got = host.numpy().copy()
        rd.render(cams[p])
        assert np.array_equal(got, rd.img.cpu().numpy()), p
