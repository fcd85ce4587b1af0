"""BF16 tensor-core decoding against the FP64 oracle.

Tolerances follow from the arithmetic: inputs and hidden activations are rounded to BF16
(relative 2^-9), so an output logit built from ~36 + 32 products of O(0.1-1) terms carries an
absolute error of a few 1e-3; after tanh / sigmoid / normalisation that stays below 1e-2.
Positions do not pass through the GEMMs and keep FP32 accuracy.  The measured errors per
output are printed (pytest -s) and bounded here."""
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


def _decode_gpu(abi, sc, mlp, cam, sel, w, fn):
    import torch
    M = len(sel)
    G = M * 10
    counts = np.zeros(8, np.uint32)
    counts[0], counts[1] = M, G
    out = {"means": torch.zeros(G, 3, device="cuda"), "scales": torch.zeros(G, 3, device="cuda"),
           "quats": torch.zeros(G, 4, device="cuda"), "opac": torch.zeros(G, device="cuda"),
           "colors": torch.zeros(G, 3, device="cuda")}
    mt = {n: cuda(a) for n, a in zip(NAMES, mlp.arrays())}
    ct = cuda(counts.view(np.int32))
    fn(cuda(sc.pos), cuda(sc.feat), cuda(sc.offs), cuda(sc.lv), sc.N, mt, cam,
       cuda(sel.astype(np.int32)), cuda(w.astype(np.float32)), M, ct, out)
    torch.cuda.synchronize()
    assert ct.cpu().numpy().view(np.uint32)[6] == 0      # no bounded wait expired
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


def _errors(got, ref, cam):
    rel_means = ref["means"] - cam.campos.astype(np.float64)
    return {"opac": np.abs(got["opac"] - ref["opac"]).max(),
            "colors": np.abs(got["colors"] - ref["colors"]).max(),
            "quats": np.abs(got["quats"] - ref["quats"]).max(),
            "scales_rel": (np.abs(got["scales"] - ref["scales"]) / ref["scales"]).max(),
            "means": np.abs(got["means"] - rel_means).max()}


@pytest.mark.parametrize("M", [1, 127, 128, 777, 3000])
def test_decode_bf16_matches_oracle(abi, M):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    rng = np.random.default_rng(M)
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=M)
    ref = oracle.decode(sel, w, sc, mlp, cam)
    got = _decode_gpu(abi, sc, mlp, cam, sel, w, abi.decode_bf16)
    e = _errors(got, ref, cam)
    print("bf16 decode max errors", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["opac"] <= 1e-2 and e["colors"] <= 1e-2 and e["quats"] <= 2e-2
    assert e["scales_rel"] <= 2e-2 and e["means"] <= 2e-5


def test_decode_bf16_city_scale(abi):
    """100k selected anchors of the 2M-anchor city: many tiles per CTA (grid-stride)."""
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    cam = cams[40]
    sel, w, _ = oracle.lod_select(sc.pos, sc.level, sc.dL, sc.NL, cam, True)
    assert len(sel) > 50_000
    ref = oracle.decode(sel, w, sc, mlp, cam)
    got = _decode_gpu(abi, sc, mlp, cam, sel, w, abi.decode_bf16)
    e = _errors(got, ref, cam)
    print("bf16 decode (city) max errors", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["opac"] <= 1e-2 and e["colors"] <= 1e-2 and e["quats"] <= 2e-2
    assert e["scales_rel"] <= 2e-2
    # positions are FP32 camera-relative: error grows with distance, still sub-millimetre
    assert e["means"] <= 1e-3


def test_bf16_frame_error_vs_oracle(abi):
    """Whole frame with BF16 decoding: per-pixel error against the FP64 oracle (stated)."""
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    cam = cams[0]
    rd = Renderer(sc, mlp, 128, 128, precision="bf16")
    c = rd.render(cam)
    assert c.overflow == 0 and c.timeout == 0
    fr = oracle.render(sc, mlp, cam)
    err = np.abs(rd.img.cpu().numpy() - fr.out["img"])
    print(f"bf16 frame error: max {err.max():.3e} mean {err.mean():.3e}")
    assert err.mean() <= 3e-3 and err.max() <= 0.1
