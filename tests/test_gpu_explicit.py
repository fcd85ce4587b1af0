"""GPU parity of the explicit-Gaussian variant (Our-3D-GS): per-Gaussian attributes and
their backward against the FP64 oracle, and a whole frame through the shared projection,
lists and blending."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import PIXEL_TOL, SEL_MARGIN, cuda, knife_pixel_mask, lib_ready, to_np_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


def _attr_tensors(attr):
    return {n: cuda(attr[n].astype(np.float32)) for n in ("log_scale", "quat", "opacity",
                                                         "color_dc")}


def _setup(M, seed):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    attr = synth.explicit_attributes(sc, seed=seed)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(sc.N, size=M, replace=False)).astype(np.int64)
    w = rng.uniform(0.05, 1.0, size=M).astype(np.float32)
    return sc, attr, cams[0], sel, w


@pytest.mark.parametrize("M", [1, 1000, 4096])
def test_explicit_gaussians_match_oracle(abi, M):
    import torch
    sc, attr, cam, sel, w = _setup(M, 3)
    ref = oracle.explicit_gaussians(sel, w, sc, attr)
    G = M * sc.k
    out = {"means": torch.zeros(G, 3, device="cuda"), "scales": torch.zeros(G, 3, device="cuda"),
           "quats": torch.zeros(G, 4, device="cuda"), "opac": torch.zeros(G, device="cuda"),
           "colors": torch.zeros(G, 3, device="cuda")}
    counts = np.zeros(8, np.uint32)
    counts[0] = M
    abi.explicit_gaussians(cuda(sc.pos), cuda(sc.offs), cuda(sc.lv), sc.N, sc.k,
                           _attr_tensors(attr), cam, cuda(sel.astype(np.int32)), cuda(w), M,
                           cuda(counts.view(np.int32)), out)
    torch.cuda.synchronize()
    means = out["means"].cpu().numpy() + cam.campos.astype(np.float64)   # camera-relative
    np.testing.assert_allclose(means, ref["means"], atol=5e-6)
    np.testing.assert_allclose(out["scales"].cpu().numpy(), ref["scales"], rtol=2e-6)
    np.testing.assert_allclose(out["quats"].cpu().numpy(), ref["quats"], atol=2e-7)
    np.testing.assert_allclose(out["opac"].cpu().numpy(), ref["opac"], atol=2e-7)
    np.testing.assert_allclose(out["colors"].cpu().numpy(), ref["colors"], atol=2e-7)


def test_explicit_backward_matches_oracle(abi):
    import torch
    M = 1500
    sc, attr, cam, sel, w = _setup(M, 5)
    G = M * sc.k
    rng = np.random.default_rng(6)
    up = {k: rng.normal(size=s).astype(np.float32) for k, s in
          (("dmeans", (G, 3)), ("dscales", (G, 3)), ("dquats", (G, 4)), ("dopac", (G,)),
           ("dcolors", (G, 3)))}
    ref = oracle.explicit_gaussians_bwd(sel, w, sc, attr, up)
    drec = np.zeros((G, 9), np.float32)
    drec[:, 5], drec[:, 6:9] = up["dopac"], up["dcolors"]
    grad = {n: torch.zeros_like(t) for n, t in _attr_tensors(attr).items()}
    doffs = torch.zeros(sc.N, sc.k, 3, device="cuda")
    dlv = torch.zeros(sc.N, 3, device="cuda")
    counts = np.zeros(8, np.uint32)
    counts[0] = M
    abi.explicit_gaussians_bwd(cuda(sc.pos), cuda(sc.offs), cuda(sc.lv), sc.N, sc.k,
                               _attr_tensors(attr), cam, cuda(sel.astype(np.int32)), cuda(w), M,
                               cuda(counts.view(np.int32)), cuda(up["dmeans"]),
                               cuda(up["dscales"]), cuda(up["dquats"]), cuda(drec), grad, doffs,
                               dlv)
    torch.cuda.synchronize()
    for name, got in (("dlog_scale", grad["log_scale"]), ("dquat", grad["quat"]),
                      ("dopacity", grad["opacity"]), ("dcolor_dc", grad["color_dc"]),
                      ("doffs", doffs), ("dlv", dlv)):
        a, b = got.cpu().numpy(), ref[name]
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), name


def test_explicit_frame_matches_oracle(abi):
    import torch
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    attr = synth.explicit_attributes(sc, seed=7)
    cam = cams[0]
    bg = (0.05, 0.1, 0.15)
    fr = oracle.render_explicit(sc, attr, cam, infer=True, bg=bg)
    rd = Renderer(sc, None, cam.W, cam.H, explicit=attr)
    c = rd.render(cam, infer=True, bg=bg)
    assert c.overflow == 0 and c.n_selected > 1000
    knife = np.nonzero(fr.sel_margin < SEL_MARGIN)[0]
    sel_g = to_np_u32(rd.sel_idx)[:c.n_selected]
    assert np.array_equal(np.setdiff1d(sel_g, knife), np.setdiff1d(fr.sel_idx, knife))
    ok = ~knife_pixel_mask(fr, cam.W, cam.H)
    assert ok.mean() > 0.5, ok.mean()
    err = np.abs(rd.img.cpu().numpy() - fr.out["img"])
    assert err[:, ok].max() <= PIXEL_TOL, err[:, ok].max()
    assert np.abs(rd.T.cpu().numpy() - fr.out["T"])[ok].max() <= 1e-5
