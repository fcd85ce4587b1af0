"""Fused BF16 decode + projection (ogs_decode_project_bf16) against the two-call path it
replaces (ogs_decode_bf16, then ogs_project_bin): the Gaussians, screen records, depth keys,
rectangles, tile counts and per-tile pair counts must be identical bit for bit.  Each of the
two calls is pinned to the FP64 oracle by its own tests (test_gpu_bf16, test_gpu_parity), and
whole fused frames against the oracle by test_bf16_frame_error_vs_oracle; this file checks
the composition, on a small scene (single and ragged tiles) and on the 2M-anchor city (about
100k anchors: many tiles per persistent CTA)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import cuda, lib_ready

pytestmark = pytest.mark.gpu

NAMES = ("w1", "b1", "w2_op", "b2_op", "w2_col", "b2_col", "w2_cov", "b2_cov")


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


def _bufs(torch, G, gx, gy):
    return {"means": torch.zeros(G, 3, device="cuda"), "scales": torch.zeros(G, 3, device="cuda"),
            "quats": torch.zeros(G, 4, device="cuda"), "opac": torch.zeros(G, device="cuda"),
            "colors": torch.zeros(G, 3, device="cuda"),
            "rec": torch.full((G, 12), -7.0, device="cuda"),
            "dk": torch.full((G,), 5, dtype=torch.int32, device="cuda"),
            "rect": torch.full((G, 2), 3, dtype=torch.int32, device="cuda"),
            "tiles": torch.full((G,), 9, dtype=torch.int32, device="cuda"),
            "tc": torch.full((gx * gy,), 11, dtype=torch.int32, device="cuda")}


def _run(abi, sc, mlp, cam, sel, w, fused, with_out=True):
    import torch
    M = len(sel)
    cap = max(M, 1)
    G = cap * 10
    gx, gy = (cam.W + 15) // 16, (cam.H + 15) // 16
    b = _bufs(torch, G, gx, gy)
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, M * 10
    ct = cuda(counts.view(np.int32))
    mt = {n: cuda(a) for n, a in zip(NAMES, mlp.arrays())}
    s = cuda(np.resize(sel, cap).astype(np.int32))
    ww = cuda(np.resize(np.asarray(w, np.float32), cap))
    g = {k: b[k] for k in ("means", "scales", "quats", "opac", "colors")}
    args = (cuda(sc.pos), cuda(sc.feat), cuda(sc.offs), cuda(sc.lv), sc.N, mt, cam, s, ww, cap, ct)
    if fused:
        scr = torch.empty(abi.decode_project_scratch_bytes(), dtype=torch.uint8, device="cuda")
        abi.decode_project_bf16(*args, b["rec"], b["dk"], b["rect"], b["tiles"], scr,
                                out=g if with_out else None, tile_count=b["tc"])
    else:
        abi.decode_bf16(*args, g)
        abi.project_bin(g, G, 1, cam, b["rec"], b["dk"], b["rect"], b["tiles"], ct,
                        tile_count=b["tc"])
    torch.cuda.synchronize()
    assert ct.cpu().numpy().view(np.uint32)[6] == 0          # no bounded wait expired
    out = {k: v.cpu().numpy() for k, v in b.items()}
    return out, M * 10


def _same(a, b, G, keys):
    for k in keys:
        x, y = a[k][:G], b[k][:G]
        assert x.tobytes() == y.tobytes(), f"{k} differs ({np.count_nonzero(x != y)} entries)"


GAUSS = ("means", "scales", "quats", "opac", "colors")
PROJ = ("rec", "dk", "rect", "tiles")


@pytest.mark.parametrize("M", [1, 127, 128, 777, 3000])
def test_fused_equals_two_calls_small(abi, M):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    rng = np.random.default_rng(100 + M)
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=M)
    ref, G = _run(abi, sc, mlp, cam, sel, w, fused=False)
    got, _ = _run(abi, sc, mlp, cam, sel, w, fused=True)
    _same(ref, got, G, GAUSS + PROJ)
    assert np.array_equal(ref["tc"], got["tc"])
    assert to_np_u32_sum(got["tc"]) == int(got["tiles"][:G].astype(np.int64).sum())
    # records only: the Gaussian buffers stay untouched, the records are the same
    rec_only, _ = _run(abi, sc, mlp, cam, sel, w, fused=True, with_out=False)
    _same(ref, rec_only, G, PROJ)
    assert not rec_only["opac"].any()
    assert np.array_equal(ref["tc"], rec_only["tc"])


def to_np_u32_sum(a):
    return int(a.view(np.uint32).astype(np.int64).sum())


@pytest.mark.parametrize("pose", [40, 100])
def test_fused_equals_two_calls_city(abi, pose):
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    cam = cams[pose]
    sel, w, _ = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cam, True)
    ref, G = _run(abi, sc, mlp, cam, sel, w, fused=False)
    got, _ = _run(abi, sc, mlp, cam, sel, w, fused=True)
    print(f"city pose {pose}: {len(sel)} anchors, {G} Gaussians, "
          f"{to_np_u32_sum(got['tc'])} pairs")
    _same(ref, got, G, GAUSS + PROJ)
    assert np.array_equal(ref["tc"], got["tc"])


def test_fused_empty_selection(abi):
    """M = 0: the tile counts are zeroed and no record is written."""
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    got, _ = _run(abi, sc, mlp, cams[0], np.zeros(0, np.int64), np.zeros(0), fused=True)
    assert not got["tc"].any()
    assert (got["rec"] == -7.0).all() and (got["dk"] == 5).all()


def test_fused_frame_equals_two_call_frame(abi):
    """Whole frames through the renderer with and without the fused call: same images."""
    import torch
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    rd = Renderer(sc, mlp, cams[0].W, cams[0].H, sel_cap=200_000, pair_cap=4_000_000,
                  precision="bf16")
    for pose in (14, 97):
        rd.fuse_decode_project = False
        rd.render(cams[pose])
        a = (rd.img.clone(), rd.T.clone(), rd.n_last.clone())
        rd.fuse_decode_project = True
        c = rd.render(cams[pose])
        assert c.overflow == 0 and c.timeout == 0
        for x, y in zip(a, (rd.img, rd.T, rd.n_last)):
            assert torch.equal(x, y)
