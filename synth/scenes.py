"""Seeded synthetic scenes, decoder weights and cameras (inputs only, no renderer arithmetic).

Stand-ins for the paper's captured datasets (MatrixCity, BungeeNeRF, Mip-NeRF360 are not
available here).  Shapes follow the paper's workloads: anchors sit on voxel centres of
nested grids whose cell size halves per level (Sec. 4.1.2, Eq. for V_L), each anchor carries
a 32-dim feature, k=10 learnable offsets, a scaling vector and a LOD bias (Sec. 4.1.1, 4.2.1),
and camera paths zoom out from street level to aerial altitude (Tab. matrix_traj, Fig. traj,
BungeeNeRF scales in Tab. bungeenerf).

Conventions shared by every consumer:
  * world frame is z-up; camera frame is x right, y down, z forward (looking direction);
  * ``R`` maps world vectors to the camera frame, ``campos`` is the camera centre, so a world
    point p has camera coordinates R @ (p - campos);
  * pixel (i, j) has its centre at integer coordinates (i, j); ``cx, cy`` is the principal
    point in those coordinates, so an image of width W centred on the axis has cx = (W-1)/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "DecoderMLP", "Camera", "ProposalMLP",
    "cube_scene", "city_scene", "decoder_mlp", "proposal_mlp",
    "look_at_camera", "zoom_out_path", "trajectory_d_max", "proposal_poses",
    "random_gaussians", "random_records", "random_rects_depths", "random_sort_keys",
    "explicit_attributes", "with_appearance", "APP_DIM", "CONFIGS", "voxel_sizes",
]

F_DIM = 32      # anchor feature width (all configs)
HIDDEN = 32     # decoder hidden width (all configs)
K_GAUSS = 10    # neural Gaussians per anchor (all configs)


@dataclass
class Scene:
    """Structure-of-arrays anchor set (float32 / uint8, C-contiguous)."""
    pos: np.ndarray        # f32[N,3]  anchor centre x_v (voxel centre)
    level: np.ndarray      # u8[N]     octree level L_j, 0 = coarsest
    dL: np.ndarray         # f32[N]    learnable LOD bias Delta L_j
    feat: np.ndarray       # f32[N,F]  anchor feature f_v
    offs: np.ndarray       # f32[N,k,3] offsets O_i
    lv: np.ndarray         # f32[N,3]  scaling l_v (positive)
    NL: int                # number of levels
    k: int = K_GAUSS
    meta: dict = field(default_factory=dict)
    app: np.ndarray = None  # f32[N,A] per-anchor appearance codes (Sec. 4.4), or None

    @property
    def N(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class DecoderMLP:
    """Three 2-layer decoders (opacity, colour, covariance) sharing the input
    z = [f_v (F), viewing direction (3), viewing distance (1)].

    Layer-1 weights are stacked: w1[m] is [HIDDEN, F+4] for m = 0 opacity, 1 colour, 2 cov.
    Layer-2 weights: w2_op [k, H], w2_col [3k, H], w2_cov [7k, H]; output rows per Gaussian i
    are contiguous (colour rows 3i..3i+2; covariance rows 7i..7i+6 = 3 scale + 4 quaternion).
    """
    w1: np.ndarray      # f32[3, H, Din]
    b1: np.ndarray      # f32[3, H]
    w2_op: np.ndarray   # f32[k, H]
    b2_op: np.ndarray   # f32[k]
    w2_col: np.ndarray  # f32[3k, H]
    b2_col: np.ndarray  # f32[3k]
    w2_cov: np.ndarray  # f32[7k, H]
    b2_cov: np.ndarray  # f32[7k]
    w1_app: np.ndarray = None  # f32[H, A] colour decoder's weights of the appearance code

    def arrays(self):
        return [self.w1, self.b1, self.w2_op, self.b2_op, self.w2_col, self.b2_col,
                self.w2_cov, self.b2_cov]


@dataclass
class ProposalMLP:
    """3-layer anchor-visibility proposal network: Din -> 64 -> 64 -> 1."""
    w1: np.ndarray  # f32[64, Din]
    b1: np.ndarray  # f32[64]
    w2: np.ndarray  # f32[64, 64]
    b2: np.ndarray  # f32[64]
    w3: np.ndarray  # f32[1, 64]
    b3: np.ndarray  # f32[1]

    def arrays(self):
        return [self.w1, self.b1, self.w2, self.b2, self.w3, self.b3]


@dataclass
class Camera:
    R: np.ndarray        # f32[3,3] world -> camera rotation (rows: right, down, forward)
    campos: np.ndarray   # f32[3]   camera centre, world
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    znear: float = 0.2
    d_max: float = 1.0   # reference distance of the LOD rule (Eq. for L_hat)
    s: float = 1.0       # focal scale factor

    def as_floats(self) -> np.ndarray:
        """Flat 22-float layout used by both the oracle and the C-ABI:
        R[9], campos[3], fx, fy, cx, cy, W, H, znear, d_max, s, pad."""
        return np.concatenate([
            self.R.astype(np.float32).reshape(9), self.campos.astype(np.float32).reshape(3),
            np.array([self.fx, self.fy, self.cx, self.cy, self.W, self.H, self.znear,
                      self.d_max, self.s, 0.0], dtype=np.float32)]).astype(np.float32)


# --------------------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------------------

def look_at_camera(eye, target, W, H, fovx_deg=60.0, up=(0.0, 0.0, 1.0), znear=0.2,
                   d_max=1.0, s=1.0) -> Camera:
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(np.float32)
    fx = (W / 2.0) / math.tan(math.radians(fovx_deg) / 2.0)
    return Camera(R=R, campos=eye.astype(np.float32), fx=float(np.float32(fx)),
                  fy=float(np.float32(fx)), cx=(W - 1) / 2.0, cy=(H - 1) / 2.0,
                  W=int(W), H=int(H), znear=float(znear), d_max=float(np.float32(d_max)),
                  s=float(s))


def zoom_out_path(n, h0, h1, centre, W, H, pitch_deg=45.0, azimuth_deg=30.0,
                  yaw_jitter_deg=0.0, seed=None, fovx_deg=60.0, d_max=1.0):
    """Cameras at altitude h_i = h0 (h1/h0)^(i/(n-1)) looking at ``centre`` with a fixed
    pitch; optional per-pose azimuth jitter (uniform, degrees)."""
    rng = np.random.default_rng(seed)
    cams = []
    c = np.asarray(centre, np.float64)
    for i in range(n):
        h = h0 * (h1 / h0) ** (i / max(n - 1, 1))
        az = math.radians(azimuth_deg + (rng.uniform(-yaw_jitter_deg, yaw_jitter_deg)
                                         if yaw_jitter_deg > 0 else 0.0))
        horiz = h / math.tan(math.radians(pitch_deg))
        eye = c + np.array([-horiz * math.cos(az), -horiz * math.sin(az), h])
        cams.append(look_at_camera(eye, c, W, H, fovx_deg=fovx_deg, d_max=d_max))
    return cams


def trajectory_d_max(scene: Scene, cams, q=0.999, sample=200_000, seed=0):
    """Robust largest / smallest camera-anchor distance over a set of poses (the r_d
    quantiles of Sec. 4.1.2), estimated on a seeded anchor subsample."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(scene.N, size=min(sample, scene.N), replace=False)
    p = scene.pos[idx].astype(np.float64)
    ds = [np.linalg.norm(p - c.campos.astype(np.float64), axis=1) for c in cams]
    d = np.concatenate(ds)
    return float(np.quantile(d, q)), float(np.quantile(d, 1.0 - q))


# --------------------------------------------------------------------------------------
# anchor attributes and decoder weights
# --------------------------------------------------------------------------------------

def _anchor_attrs(rng, pos, level, cell, k=K_GAUSS, F=F_DIM):
    N = pos.shape[0]
    feat = rng.normal(0.0, 0.1, size=(N, F)).astype(np.float32)
    dL = (np.round(rng.uniform(0.0, 0.3, size=N) / 0.01) * 0.01).astype(np.float32)
    offs = rng.normal(0.0, 0.5, size=(N, k, 3)).astype(np.float32)
    lv = np.repeat(cell[level][:, None], 3, axis=1).astype(np.float32)
    return feat, dL, offs, lv


def decoder_mlp(seed=0, k=K_GAUSS, F=F_DIM, H=HIDDEN, dist_scale=1.0, opacity_bias=0.5):
    """PyTorch-default-style uniform init (bound 1/sqrt(fan_in)).  The distance input column
    is scaled by ``dist_scale`` (1/d_max) so a random decoder sees O(1) inputs; the opacity
    output bias is raised by ``opacity_bias`` so that tanh gives alpha ~ 0.4-0.6 instead of
    ~0 (a random-init decoder would otherwise render an empty image)."""
    rng = np.random.default_rng(seed)
    Din = F + 4
    b_in = 1.0 / math.sqrt(Din)
    b_h = 1.0 / math.sqrt(H)
    w1 = rng.uniform(-b_in, b_in, size=(3, H, Din)).astype(np.float32)
    w1[:, :, Din - 1] *= np.float32(dist_scale)
    b1 = rng.uniform(-b_in, b_in, size=(3, H)).astype(np.float32)
    w2_op = rng.uniform(-b_h, b_h, size=(k, H)).astype(np.float32)
    b2_op = (rng.uniform(-b_h, b_h, size=k) + opacity_bias).astype(np.float32)
    w2_col = rng.uniform(-b_h, b_h, size=(3 * k, H)).astype(np.float32)
    b2_col = rng.uniform(-1.5, 1.5, size=3 * k).astype(np.float32)
    w2_cov = rng.uniform(-b_h, b_h, size=(7 * k, H)).astype(np.float32)
    b2_cov = rng.uniform(-b_h, b_h, size=7 * k).astype(np.float32)
    b2_cov.reshape(k, 7)[:, :3] += rng.uniform(-1.0, 1.0, size=(k, 3)).astype(np.float32)
    b2_cov.reshape(k, 7)[:, 3:] += rng.normal(0.0, 1.0, size=(k, 4)).astype(np.float32)
    return DecoderMLP(w1, b1, w2_op, b2_op, w2_col, b2_col, w2_cov, b2_cov)


def proposal_mlp(seed=0, Din=F_DIM + 5, H=64):
    rng = np.random.default_rng(seed)
    b0 = 1.0 / math.sqrt(Din)
    bh = 1.0 / math.sqrt(H)
    return ProposalMLP(
        w1=rng.uniform(-b0, b0, size=(H, Din)).astype(np.float32),
        b1=rng.uniform(-b0, b0, size=H).astype(np.float32),
        w2=rng.uniform(-bh, bh, size=(H, H)).astype(np.float32),
        b2=rng.uniform(-bh, bh, size=H).astype(np.float32),
        w3=rng.uniform(-bh, bh, size=(1, H)).astype(np.float32),
        b3=np.zeros(1, np.float32))


# --------------------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------------------

def cube_scene(seed=0, N=4096, NL=3, extent=10.0, k=K_GAUSS, F=F_DIM) -> Scene:
    """Anchors at distinct random voxel centres of NL nested grids filling a cube of side
    ``extent`` centred on the origin; level-L cells are extent/2^(L+3); per-level counts are
    proportional to 4^L (surface-like growth of detail)."""
    rng = np.random.default_rng(seed)
    w = 4.0 ** np.arange(NL)
    counts = np.floor(N * w / w.sum()).astype(np.int64)
    counts[-1] += N - counts.sum()
    cell = np.array([extent / 2 ** (L + 3) for L in range(NL)], np.float64)
    pos, lev = [], []
    for L in range(NL):
        n_side = 2 ** (L + 3)
        flat = rng.choice(n_side ** 3, size=int(counts[L]), replace=False)
        ijk = np.stack(np.unravel_index(flat, (n_side,) * 3), axis=1).astype(np.float64)
        pos.append((ijk + 0.5) * cell[L] - extent / 2)
        lev.append(np.full(counts[L], L, np.uint8))
    pos = np.concatenate(pos).astype(np.float32)
    level = np.concatenate(lev)
    perm = rng.permutation(N)
    pos, level = pos[perm], level[perm]
    feat, dL, offs, lv = _anchor_attrs(rng, pos, level, cell, k, F)
    return Scene(pos=np.ascontiguousarray(pos), level=level, dL=dL, feat=feat, offs=offs,
                 lv=lv, NL=NL, k=k, meta={"kind": "cube", "extent": extent,
                                           "cell": cell.tolist(), "counts": counts.tolist()})


def _city_boxes(rng, extent, block=100.0, street=20.0, plaza=40.0):
    """Boxes (x0, y0, x1, y1, h) on a street grid centred on the origin, 1-4 per 100 m block
    (footprint and height U[10, 60] m); a plaza of radius ``plaza`` around the centre is kept
    free of buildings.  Also returns a [nb, nb, 4] table of each block's box indices (-1 =
    none) for fast point-in-footprint queries."""
    pitch = block + street
    nb = int(math.ceil(extent / pitch))
    boxes = []
    table = -np.ones((nb, nb, 4), np.int64)
    for bi in range(nb):
        for bj in range(nb):
            bx0 = -extent / 2 + bi * pitch + street / 2
            by0 = -extent / 2 + bj * pitch + street / 2
            slot = 0
            for _ in range(int(rng.integers(1, 5))):
                wx, wy, h = rng.uniform(10.0, 60.0, size=3)
                x0 = bx0 + rng.uniform(0.0, block - wx)
                y0 = by0 + rng.uniform(0.0, block - wy)
                cxb, cyb = x0 + wx / 2, y0 + wy / 2
                if math.hypot(cxb, cyb) < plaza + max(wx, wy) / 2:
                    continue
                table[bi, bj, slot] = len(boxes)
                slot += 1
                boxes.append((x0, y0, x0 + wx, y0 + wy, h))
    return np.asarray(boxes, np.float64).reshape(-1, 5), table, pitch


def _sample_surface(rng, city, extent, half, n):
    """n points uniformly (by area) on the ground square [-half, half]^2 (outside box
    footprints) and on the top and side faces of the boxes, restricted to |x|,|y| <= half."""
    boxes, table, pitch = city
    x0, y0, x1, y1, h = boxes.T
    wx, wy = x1 - x0, y1 - y0
    # only boxes that reach into the square can receive samples
    near = (x1 >= -half) & (x0 <= half) & (y1 >= -half) & (y0 <= half)
    bidx = np.nonzero(near)[0]
    nbx = len(bidx)
    # faces: ground, then per nearby box: top, -x, +x, -y, +y
    areas = np.concatenate([[4 * half * half], (wx * wy)[bidx], (wy * h)[bidx], (wy * h)[bidx],
                            (wx * h)[bidx], (wx * h)[bidx]])
    prob = areas / areas.sum()
    out = []
    have = 0
    while have < n:
        m = int((n - have) * 1.3) + 64
        face = rng.choice(len(areas), size=m, p=prob)
        u, v = rng.uniform(size=m), rng.uniform(size=m)
        P = np.zeros((m, 3))
        g = face == 0
        P[g, 0] = (u[g] * 2 - 1) * half
        P[g, 1] = (v[g] * 2 - 1) * half
        fb = face - 1
        for kind in range(5):
            sel = (fb >= kind * nbx) & (fb < (kind + 1) * nbx) & ~g
            b = bidx[fb[sel] - kind * nbx]
            uu, vv = u[sel], v[sel]
            if kind == 0:
                P[sel] = np.stack([x0[b] + uu * wx[b], y0[b] + vv * wy[b], h[b]], 1)
            elif kind == 1:
                P[sel] = np.stack([x0[b], y0[b] + uu * wy[b], vv * h[b]], 1)
            elif kind == 2:
                P[sel] = np.stack([x1[b], y0[b] + uu * wy[b], vv * h[b]], 1)
            elif kind == 3:
                P[sel] = np.stack([x0[b] + uu * wx[b], y0[b], vv * h[b]], 1)
            else:
                P[sel] = np.stack([x0[b] + uu * wx[b], y1[b], vv * h[b]], 1)
        keep = (np.abs(P[:, 0]) <= half) & (np.abs(P[:, 1]) <= half)
        if len(boxes):
            # ground points under a footprint are hidden: drop them (block-table lookup)
            gi = np.nonzero(g)[0]
            nbk = table.shape[0]
            bi = np.clip(((P[gi, 0] + extent / 2) // pitch).astype(np.int64), 0, nbk - 1)
            bj = np.clip(((P[gi, 1] + extent / 2) // pitch).astype(np.int64), 0, nbk - 1)
            inside = np.zeros(len(gi), bool)
            for slot in range(4):
                k = table[bi, bj, slot]
                has = k >= 0
                kk = np.where(has, k, 0)
                inside |= has & (P[gi, 0] >= x0[kk]) & (P[gi, 0] <= x1[kk]) & \
                    (P[gi, 1] >= y0[kk]) & (P[gi, 1] <= y1[kk])
            keep[gi[inside]] = False
        P = P[keep]
        out.append(P)
        have += len(P)
    return np.concatenate(out)[:n]


def city_scene(seed=0, N=2_000_000, NL=8, extent=2000.0, c0=4.0, gamma=0.55,
               k=K_GAUSS, F=F_DIM) -> Scene:
    """Street-grid city of side ``extent`` (blocks 100 m, streets 20 m, 1-4 boxes per block
    with footprint and height U[10, 60] m) plus ground.  Level-L anchors are voxel centres
    (cell c0/2^L, Eq. for V_L) of surface samples inside a centred square of half-width
    (extent/2)·2^(-gamma·L): fine levels concentrate where a zoom-out path starts, as in
    multi-scale captures.  Per-level counts follow the number of cells that square holds,
    (2^((1-gamma)·L))^2, scaled to N; duplicates within a level are removed."""
    rng = np.random.default_rng(seed)
    city = _city_boxes(rng, extent)
    w = np.array([4.0 ** ((1.0 - gamma) * L) for L in range(NL)])
    counts = np.floor(N * w / w.sum()).astype(np.int64)
    counts[-1] += N - counts.sum()
    cell = np.array([c0 / 2 ** L for L in range(NL)], np.float64)
    pos, lev = [], []
    for L in range(NL):
        half = (extent / 2) * 2.0 ** (-gamma * L)
        need = int(counts[L])
        keys = np.empty(0, np.int64)
        V_all = np.empty((0, 3))
        batch = int(need * 1.5) + 64
        for _ in range(40):
            P = _sample_surface(rng, city, extent, half, batch)
            V = np.round(P / cell[L])
            key = ((V[:, 0].astype(np.int64) + (1 << 20)) << 42) | \
                  ((V[:, 1].astype(np.int64) + (1 << 20)) << 21) | \
                  (V[:, 2].astype(np.int64) + (1 << 20))
            keys = np.concatenate([keys, key])
            V_all = np.concatenate([V_all, V])
            _, first = np.unique(keys, return_index=True)
            if len(first) >= need:
                break
            batch = int((need - len(first)) * 3) + 64
        else:
            raise RuntimeError(f"level {L}: only {len(first)} of {need} free cells")
        first = np.sort(first)[:need]
        pos.append(V_all[first] * cell[L])
        lev.append(np.full(need, L, np.uint8))
    pos = np.concatenate(pos).astype(np.float32)
    level = np.concatenate(lev)
    perm = rng.permutation(pos.shape[0])
    pos, level = pos[perm], level[perm]
    feat, dL, offs, lv = _anchor_attrs(rng, pos, level, cell, k, F)
    return Scene(pos=np.ascontiguousarray(pos), level=level, dL=dL, feat=feat, offs=offs,
                 lv=lv, NL=NL, k=k, meta={"kind": "city", "extent": extent, "c0": c0,
                                           "gamma": gamma, "counts": counts.tolist(),
                                           "n_boxes": int(len(city[0]))})


# --------------------------------------------------------------------------------------
# stage-test inputs
# --------------------------------------------------------------------------------------

def random_gaussians(seed, G, cam: Camera, depth=(2.0, 30.0), scale=(0.05, 0.8),
                     spread=1.2, frac_behind=0.05):
    """Random world-space Gaussians (means, scales, unit quaternions w-first, opacity,
    colour) mostly inside the view of ``cam``; a fraction lies behind the camera."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(*depth, size=G)
    tanx = cam.W / (2 * cam.fx)
    tany = cam.H / (2 * cam.fy)
    x = rng.uniform(-spread, spread, size=G) * tanx * z
    y = rng.uniform(-spread, spread, size=G) * tany * z
    behind = rng.uniform(size=G) < frac_behind
    z = np.where(behind, -z, z)
    pc = np.stack([x, y, z], 1)
    means = (pc @ cam.R.astype(np.float64)) + cam.campos.astype(np.float64)
    scales = np.exp(rng.uniform(np.log(scale[0]), np.log(scale[1]), size=(G, 3)))
    q = rng.normal(size=(G, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.uniform(0.05, 0.95, size=G)
    col = rng.uniform(0.0, 1.0, size=(G, 3))
    f = np.float32
    return dict(means=means.astype(f), scales=scales.astype(f), quats=q.astype(f),
                opac=opac.astype(f), colors=col.astype(f))


def random_records(seed, G, W, H, sigma=(0.6, 12.0), opac=(0.05, 0.99)):
    """Random screen-space Gaussians: centre (u, v), 2x2 covariance from random axes and its
    inverse (conic), opacity, colour and a strictly positive depth, spread over a W x H image
    (with a margin)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-0.1 * W, 1.1 * W, size=G)
    v = rng.uniform(-0.1 * H, 1.1 * H, size=G)
    s1 = np.exp(rng.uniform(np.log(sigma[0]), np.log(sigma[1]), size=G))
    s2 = np.exp(rng.uniform(np.log(sigma[0]), np.log(sigma[1]), size=G))
    th = rng.uniform(0, np.pi, size=G)
    c, s = np.cos(th), np.sin(th)
    a = c * c * s1 * s1 + s * s * s2 * s2
    b = c * s * (s1 * s1 - s2 * s2)
    d = s * s * s1 * s1 + c * c * s2 * s2
    o = rng.uniform(*opac, size=G)
    col = rng.uniform(0, 1, size=(G, 3))
    depth = rng.uniform(1.0, 50.0, size=G)
    # inverse of [[a, b], [b, d]] from the same axes: R diag(1/s1^2, 1/s2^2) R^T
    ia = c * c / (s1 * s1) + s * s / (s2 * s2)
    ib = c * s * (1 / (s1 * s1) - 1 / (s2 * s2))
    idd = s * s / (s1 * s1) + c * c / (s2 * s2)
    f = np.float32
    return dict(u=u.astype(f), v=v.astype(f), cov=np.stack([a, b, d], 1).astype(f),
                conic=np.stack([ia, ib, idd], 1).astype(f), opac=o.astype(f),
                colors=col.astype(f), depth=depth.astype(f))


def random_rects_depths(seed, G, gx, gy, max_span=6, equal_depth_frac=0.05):
    """Random tile rectangles [x0,x1)x[y0,y1) inside a gx x gy grid (some empty) and positive
    depths, a fraction of which repeat exactly (ties)."""
    rng = np.random.default_rng(seed)
    x0 = rng.integers(0, gx, size=G)
    y0 = rng.integers(0, gy, size=G)
    x1 = np.minimum(gx, x0 + rng.integers(0, max_span + 1, size=G))
    y1 = np.minimum(gy, y0 + rng.integers(0, max_span + 1, size=G))
    depth = rng.uniform(0.3, 100.0, size=G).astype(np.float32)
    tie = rng.uniform(size=G) < equal_depth_frac
    if G > 1:
        depth[tie] = depth[rng.integers(0, G, size=int(tie.sum()))]
    rect = np.stack([x0, y0, x1, y1], 1).astype(np.int32)
    return rect, depth


def random_sort_keys(seed, n, bits=32, dup_frac=0.2):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
    dup = rng.uniform(size=n) < dup_frac
    if n > 1:
        keys[dup] = keys[rng.integers(0, n, size=int(dup.sum()))]
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


# --------------------------------------------------------------------------------------
# the five workloads (scene, decoder, cameras)
# --------------------------------------------------------------------------------------

def _cfg1():
    """4,096 anchors, 3 levels, 10 m cube, one camera 12 m from the centre, 128x128."""
    sc = cube_scene(seed=0)
    d_max = 30.0
    cam = look_at_camera(np.array([3.0, -4.0, 10.5]) * (12.0 / np.linalg.norm([3.0, -4.0, 10.5])),
                         np.zeros(3), 128, 128, d_max=d_max)
    mlp = decoder_mlp(seed=0, dist_scale=1.0 / d_max)
    return sc, mlp, [cam]


def _city_cfg(N, NL, extent, c0, n_poses, h0, h1, W, H, seed=0, yaw_jitter=0.0, pose_seed=None):
    sc = city_scene(seed=seed, N=N, NL=NL, extent=extent, c0=c0)
    cams = zoom_out_path(n_poses, h0, h1, (0.0, 0.0, 0.0), W, H, yaw_jitter_deg=yaw_jitter,
                         seed=pose_seed)
    d_max, d_min = trajectory_d_max(sc, cams)
    for c in cams:
        c.d_max = float(np.float32(d_max))
    sc.meta.update(d_max=d_max, d_min=d_min, NL_eqK=int(round(math.log2(d_max / d_min))) + 1)
    mlp = decoder_mlp(seed=seed, dist_scale=1.0 / d_max)
    return sc, mlp, cams


def _cfg2():
    """500k anchors, 6 levels, 600 m street grid, 30-pose zoom-out 8 m -> 250 m, 1600x900."""
    return _city_cfg(500_000, 6, 600.0, 2.0, 30, 8.0, 250.0, 1600, 900)


def _cfg3():
    """2M anchors, 8 levels, 2 km city grid, 120-pose zoom-out 10 m -> 2 km, 1920x1080."""
    return _city_cfg(2_000_000, 8, 2000.0, 4.0, 120, 10.0, 2000.0, 1920, 1080)


def proposal_poses(main_cams, n, seed, h0=10.0, h1=2000.0, yaw_jitter=40.0):
    """Zoom-out poses with random azimuth jitter for training / evaluating the anchor
    visibility proposal; they share the LOD reference distance of the main path."""
    c0 = main_cams[0]
    return zoom_out_path(n, h0, h1, (0.0, 0.0, 0.0), c0.W, c0.H, yaw_jitter_deg=yaw_jitter,
                         seed=seed, d_max=c0.d_max)


def _cfg3_train_poses():
    """Config-3 scene with 200 zoom-out poses with yaw jitter (proposal-net training views)."""
    return _city_cfg(2_000_000, 8, 2000.0, 4.0, 200, 10.0, 2000.0, 1920, 1080,
                     yaw_jitter=40.0, pose_seed=2)


def _cfg3_heldout_poses():
    """Config-3 scene with 60 held-out zoom-out poses (different yaw jitter seed)."""
    return _city_cfg(2_000_000, 8, 2000.0, 4.0, 60, 10.0, 2000.0, 1920, 1080,
                     yaw_jitter=40.0, pose_seed=3)


def _cfg5():
    """8M anchors, 10 levels, 4 km city grid, zoom-out 8 m -> 4 km (16 views per step), 1080p."""
    return _city_cfg(8_000_000, 10, 4000.0, 6.0, 64, 8.0, 4000.0, 1920, 1080)


CONFIGS = {
    "cube4k_128": _cfg1,
    "street500k_1600x900": _cfg2,
    "city2M_1080p": _cfg3,
    "city2M_1080p_train200": _cfg3_train_poses,
    "city2M_1080p_heldout60": _cfg3_heldout_poses,
    "city8M_1080p": _cfg5,
}


APP_DIM = 8   # appearance code width (Sec. 4.4 gives none; 8 fills the decoders' K padding)


def voxel_sizes(scene):
    """Voxel size of every level of a generated scene (float32[NL]): the cube's cells, or the
    city's base cell c0 halved per level."""
    if "cell" in scene.meta:
        return np.asarray(scene.meta["cell"], np.float32)
    return np.asarray([scene.meta["c0"] / 2 ** L for L in range(scene.NL)], np.float32)


def with_appearance(scene, mlp, seed=0, A=APP_DIM, scale=0.5):
    """Copies of (scene, mlp) with a seeded appearance code per anchor, N(0, scale), and the
    colour decoder's first-layer weights for it, U(+-1/sqrt(F + 4 + A))."""
    import copy
    rng = np.random.default_rng(seed + 777)
    sc = copy.copy(scene)
    sc.app = rng.normal(0.0, scale, size=(scene.N, A)).astype(np.float32)
    m = copy.copy(mlp)
    H = mlp.w1.shape[1]
    b = 1.0 / math.sqrt(mlp.w1.shape[2] + A)
    m.w1_app = rng.uniform(-b, b, size=(H, A)).astype(np.float32)
    return sc, m


def explicit_attributes(scene, seed=0):
    """Seeded per-Gaussian attributes for the explicit-Gaussian variant: log-scales around
    20-80 % of the anchor's cell (l_v), random quaternions, opacity logits N(0.5, 1) and
    degree-0 colour coefficients N(0, 1.5)."""
    rng = np.random.default_rng(seed)
    N, k = scene.N, scene.k
    frac = rng.uniform(0.2, 0.8, size=(N, k, 3))
    return dict(
        log_scale=np.log(scene.lv[:, None, :].astype(np.float64) * frac).astype(np.float32),
        quat=rng.normal(size=(N, k, 4)).astype(np.float32),
        opacity=rng.normal(0.5, 1.0, size=(N, k)).astype(np.float32),
        color_dc=rng.normal(0.0, 1.5, size=(N, k, 3)).astype(np.float32),
    )
