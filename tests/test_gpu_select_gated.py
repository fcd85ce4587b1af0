"""Gated selection in one pass (ogs_lod_select_gated) against the two calls it replaces
(ogs_lod_select, then ogs_proposal_gate_bf16): the same anchors in the same order with the
same weights, and the same counts.  Both compute the gate with the same tensor-core network
code, so the keep decisions must agree exactly, including at p*.  The two calls are pinned to
the FP64 oracle by test_gpu_parity and test_gpu_proposal.  Cases: full 2048-anchor tiles read
by bulk copies (4096-anchor cube, 2M-anchor city), a ragged last tile, arrays that are not
16-byte aligned (plain loads), several networks and thresholds, and an empty view; the fused
call starts from stale counters, which it must reset."""
import numpy as np
import pytest

import synth
from gpu_helpers import cuda, lib_ready, to_np_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    return lib_ready()


def _net(seed):
    from paper_2403_17898_gb300 import proposal
    return proposal.ProposalNet(synth.proposal_mlp(seed=seed)).w


def _two_calls(abi, arrs, N, NL, cam, net, p_star, cap):
    import torch
    pos, level, dL, feat = arrs
    sel = torch.zeros(cap, dtype=torch.int32, device="cuda")
    w = torch.zeros(cap, device="cuda")
    so = torch.zeros(cap, dtype=torch.int32, device="cuda")
    wo = torch.zeros(cap, device="cuda")
    ct = torch.zeros(8, dtype=torch.int32, device="cuda")
    s1 = torch.empty(abi.lod_select_scratch_bytes(N), dtype=torch.uint8, device="cuda")
    s2 = torch.empty(abi.proposal_gate_scratch_bytes(cap), dtype=torch.uint8, device="cuda")
    abi.lod_select(pos, level, dL, N, NL, 10, cam, True, sel, w, cap, ct, s1)
    abi.proposal_gate(pos, level, feat, N, NL, 10, cam, net, p_star, sel, w, cap, ct, so, wo,
                      None, s2, bf16=True)
    torch.cuda.synchronize()
    c = to_np_u32(ct)
    M = int(c[0])
    return to_np_u32(so)[:M].copy(), wo.cpu().numpy()[:M].copy(), c


def _fused(abi, arrs, N, NL, cam, net, p_star, cap):
    import torch
    pos, level, dL, feat = arrs
    sel = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    w = torch.zeros(cap, device="cuda")
    # stale counters from an earlier frame: the call resets every field itself
    ct = torch.full((8,), 0x5A5A, dtype=torch.int32, device="cuda")
    scr = torch.empty(abi.lod_select_gated_scratch_bytes(N), dtype=torch.uint8, device="cuda")
    abi.lod_select_gated(pos, level, dL, feat, N, NL, 10, cam, True, net, p_star, sel, w, cap,
                         ct, scr)
    torch.cuda.synchronize()
    c = to_np_u32(ct)
    M = int(c[0])
    return to_np_u32(sel)[:M].copy(), w.cpu().numpy()[:M].copy(), c


def _compare(abi, arrs, N, NL, cam, net, p_star, cap):
    a_idx, a_w, a_c = _two_calls(abi, arrs, N, NL, cam, net, p_star, cap)
    b_idx, b_w, b_c = _fused(abi, arrs, N, NL, cam, net, p_star, cap)
    assert a_c[6] == 0 and b_c[6] == 0                       # no bounded wait expired
    assert a_c[3] == 0 and b_c[3] == 0                       # no overflow
    assert np.array_equal(a_idx, b_idx)
    assert a_w.tobytes() == b_w.tobytes()
    assert a_c[0] == b_c[0] and a_c[1] == b_c[1]
    return len(b_idx)


def _arrays(sc, lo=0, hi=None, shift=False):
    """Device copies of the anchor arrays [lo, hi); shift=True stores them one element past a
    16-byte boundary (selection falls back to plain loads; features stay aligned)."""
    import torch
    hi = sc.N if hi is None else hi

    def dev(a, dtype):
        a = np.ascontiguousarray(a[lo:hi])
        if not shift:
            return cuda(a)
        flat = torch.zeros(a.size + 4, dtype=dtype, device="cuda")
        v = flat[1:1 + a.size].view(a.shape)
        v.copy_(torch.from_numpy(a).to("cuda"))
        return v

    return (dev(sc.pos.astype(np.float32), torch.float32), dev(sc.level.astype(np.uint8), torch.uint8),
            dev(sc.dL.astype(np.float32), torch.float32), cuda(np.ascontiguousarray(sc.feat[lo:hi])))


@pytest.mark.parametrize("seed,p_star", [(0, 0.5), (1, 0.3), (2, 0.7)])
def test_gated_select_cube(abi, seed, p_star):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    side = synth.look_at_camera(np.array([6.0, 3.0, 2.5]), np.zeros(3), 128, 128, d_max=30.0)
    for cam in (cams[0], side):
        n = _compare(abi, _arrays(sc), sc.N, sc.NL, cam, _net(seed), p_star, sc.N)
        print(f"cube seed {seed} p* {p_star}: {n} kept")


def test_gated_select_ragged_and_unaligned(abi):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    N = 3001                                                  # one full tile + a ragged one
    for shift in (False, True):
        _compare(abi, _arrays(sc, 0, N, shift), N, sc.NL, cams[0], _net(3), 0.5, N)


@pytest.mark.parametrize("pose", [14, 60, 119])
def test_gated_select_city(abi, pose):
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    n = _compare(abi, _arrays(sc), sc.N, sc.NL, cams[pose], _net(0), 0.5, 400_000)
    print(f"city pose {pose}: {n} kept")


def test_gated_select_empty_view(abi):
    sc, mlp, cams = synth.CONFIGS["cube4k_128"]()
    away = synth.look_at_camera(cams[0].campos, 2 * cams[0].campos, 128, 128, d_max=30.0)
    assert _compare(abi, _arrays(sc), sc.N, sc.NL, away, _net(0), 0.5, sc.N) == 0


def test_gated_frame_equals_two_call_frame(abi):
    """Whole gated frames through the renderer, fused and two-call: the same image."""
    import torch
    from paper_2403_17898_gb300.render import Renderer
    sc, mlp, cams = synth.CONFIGS["city2M_1080p"]()
    rd = Renderer(sc, mlp, cams[0].W, cams[0].H, sel_cap=200_000, pair_cap=4_000_000,
                  precision="bf16")
    gate = (_net(0), 0.5)
    for pose in (14, 97):
        rd.fuse_gate = False
        c0 = rd.render(cams[pose], gate=gate)
        a = (rd.img.clone(), rd.T.clone(), rd.n_last.clone())
        rd.fuse_gate = True
        c1 = rd.render(cams[pose], gate=gate)
        assert c1.overflow == 0 and c1.timeout == 0 and c1.n_selected == c0.n_selected
        for x, y in zip(a, (rd.img, rd.T, rd.n_last)):
            assert torch.equal(x, y)
