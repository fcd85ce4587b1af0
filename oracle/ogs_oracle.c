/*
 * FP64 CPU oracle for the Octree-GS LOD renderer hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg load this library.  It shares no code, header, table or helper with the CUDA
 * path; both receive the same seeded inputs.
 *
 * Plain, slow, obviously-correct restatements, in double precision, in the paper's order:
 *   orc_lod_select   Sec. 4.1.3, Eq. for L_hat (cumulative LOD + LOD bias), and the opacity
 *                    blending of the next level during inference (same section).
 *   orc_decode       Sec. 3.2, Eq. offsets (mu_i = x_v + O_i * l_v) and Eq. mlp (attributes
 *                    decoded by small MLPs from feature, viewing distance and direction).
 *   orc_project      Sec. 3.1, Eq. 1: Sigma = R S S^T R^T, EWA projection to a 2D Gaussian,
 *                    with the conventions of the tile rasterizer that Sec. 3.1 cites.
 *   orc_tile_lists   Sec. 3.1: each 16x16 tile's Gaussians in front-to-back depth order.
 *   orc_blend        Sec. 3.1, Eq. 2: C = sum_i T_i c_i sigma_i, T_i = prod_{j<i}(1 - sigma_j).
 *   orc_*_bwd        hand-derived analytic gradients of the above (training path).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - L* = clamp(log2(d_max / (d s)) + dL, 0, NL-1): the clamp bounds the fractional level;
 *   - visibility = anchor centre in front of the near plane and within 1.3x the half-fov;
 *   - decoder input z = [f_v, (x_v - c)/|x_v - c|, |x_v - c|]; opacity tanh, kept if > 0;
 *     colour sigmoid; scale l_v * sigmoid; quaternion (w,x,y,z) normalised;
 *   - opacity of a next-level (transitional) anchor is multiplied by L* - floor(L*); a
 *     next-level anchor whose weight would be exactly 0 is not selected (it could only emit
 *     zero-opacity Gaussians, which the alpha > 0 rule drops anyway);
 *   - 2D covariance gets +0.3 px^2 on its diagonal; extent radius r = 3 sqrt(lambda_max) with
 *     lambda_max = mid + sqrt(max(0.1, mid^2 - det)); a tile is covered if it holds a pixel
 *     centre inside [u-r, u+r] x [v-r, v+r];
 *   - alpha = min(0.99, o exp(power)); skip power > 0 or alpha < 1/255; stop before
 *     blending a Gaussian that would bring T below 1e-4; C += T bg at the end;
 *   - depth ties are broken by Gaussian id (= anchor rank in the selection * k + i).
 *
 * Every discrete decision also reports a margin (distance to its threshold) so that tests can
 * tell a decision that is fixed by the inputs from one that rounding could flip.
 *
 * Camera layout (22 doubles): R[9] (world->camera, row-major), campos[3], fx, fy, cx, cy,
 * W, H, znear, d_max, s, pad.  Camera coordinates of world point p: R (p - campos).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_ALPHA_MAX 0.99
#define ORC_T_MIN 1e-4
#define ORC_LOWPASS 0.3
#define ORC_FRUSTUM 1.3

typedef struct {
    double R[9], c[3], fx, fy, cx, cy;
    int W, H;
    double znear, d_max, s;
} cam_t;

static cam_t read_cam(const double* p) {
    cam_t k;
    for (int i = 0; i < 9; ++i) k.R[i] = p[i];
    for (int i = 0; i < 3; ++i) k.c[i] = p[9 + i];
    k.fx = p[12]; k.fy = p[13]; k.cx = p[14]; k.cy = p[15];
    k.W = (int)p[16]; k.H = (int)p[17];
    k.znear = p[18]; k.d_max = p[19]; k.s = p[20];
    return k;
}

static void to_cam(const cam_t* k, const double* p, double* out) {
    double d[3] = {p[0] - k->c[0], p[1] - k->c[1], p[2] - k->c[2]};
    for (int r = 0; r < 3; ++r)
        out[r] = k->R[3 * r] * d[0] + k->R[3 * r + 1] * d[1] + k->R[3 * r + 2] * d[2];
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------------------------- */
/* Sec. 4.1.3: anchor selection                                                           */
/* ------------------------------------------------------------------------------------- */

/* Returns M, the number of selected anchors, in anchor-index order.  sel_w is 1 for anchors
 * with L_j <= L_hat and L* - L_hat for next-level anchors (infer != 0 only).  margin[j] is the
 * smallest of: |Lraw - t| over the level thresholds t that decide anchor j, and the relative
 * distances of the visibility tests to their bounds. */
long orc_lod_select(long N, const double* pos, const int32_t* level, const double* dL, int NL,
                    const double* camp, int infer, int64_t* sel_idx, double* sel_w,
                    double* margin) {
    cam_t k = read_cam(camp);
    double tanx = k.W / (2.0 * k.fx), tany = k.H / (2.0 * k.fy);
    long M = 0;
    for (long j = 0; j < N; ++j) {
        const double* p = pos + 3 * j;
        double dv[3] = {p[0] - k.c[0], p[1] - k.c[1], p[2] - k.c[2]};
        double d = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double pc[3];
        to_cam(&k, p, pc);
        /* visibility of the anchor centre */
        double bx = ORC_FRUSTUM * tanx * pc[2], by = ORC_FRUSTUM * tany * pc[2];
        int visible = pc[2] > k.znear && fabs(pc[0]) <= bx && fabs(pc[1]) <= by;
        double m = fabs(pc[2] - k.znear) / dmax(d, 1e-300);
        m = dmin(m, fabs(bx - fabs(pc[0])) / dmax(d, 1e-300));
        m = dmin(m, fabs(by - fabs(pc[1])) / dmax(d, 1e-300));
        /* Eq. for L_hat: fractional level from distance plus LOD bias, clamped */
        double Lraw = log2(k.d_max / (d * k.s)) + dL[j];
        double Lstar = dmin(dmax(Lraw, 0.0), (double)(NL - 1));
        double Lhat = floor(Lstar);
        int L = level[j];
        if (L >= 1) m = dmin(m, fabs(Lraw - L));
        if (L >= 2) m = dmin(m, fabs(Lraw - (L - 1)));
        if (margin) margin[j] = m;
        if (!visible) continue;
        if ((double)L <= Lhat) {
            sel_idx[M] = j;
            sel_w[M] = 1.0;
            ++M;
        } else if (infer && (double)L == Lhat + 1.0 && Lstar > Lhat) {
            sel_idx[M] = j;
            sel_w[M] = Lstar - Lhat;
            ++M;
        }
    }
    return M;
}

/* ------------------------------------------------------------------------------------- */
/* Sec. 3.2: neural Gaussians of the selected anchors                                     */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    const double *w1, *b1, *w2op, *b2op, *w2col, *b2col, *w2cov, *b2cov;
    int F, Hd, k;
    const double* w1app;   /* colour decoder's weights of the appearance code [Hd][A], or NULL */
    int A;                 /* appearance code width (0: none) */
} mlp_t;

/* z = [f_v, dir, dist]; hidden[m][h] = relu(W1[m] z + b1[m]); pre-activation kept too.  The
 * colour decoder (m = 1) also sees the anchor's appearance code a (Sec. 4.4):
 * + W1app[h] . a. */
static void mlp_hidden(const mlp_t* W, const double* z, const double* app, double* hid,
                       double* pre) {
    int Din = W->F + 4;
    for (int m = 0; m < 3; ++m)
        for (int h = 0; h < W->Hd; ++h) {
            const double* row = W->w1 + ((long)m * W->Hd + h) * Din;
            double a = W->b1[m * W->Hd + h];
            for (int i = 0; i < Din; ++i) a += row[i] * z[i];
            if (m == 1 && W->A > 0)
                for (int c = 0; c < W->A; ++c) a += W->w1app[(long)h * W->A + c] * app[c];
            pre[m * W->Hd + h] = a;
            hid[m * W->Hd + h] = a > 0 ? a : 0;
        }
}

static double mlp_out(const double* w2, const double* b2, int row, const double* hid, int Hd,
                      double* absum) {
    double a = b2[row], s = fabs(b2[row]);
    for (int h = 0; h < Hd; ++h) {
        a += w2[(long)row * Hd + h] * hid[h];
        s += fabs(w2[(long)row * Hd + h] * hid[h]);
    }
    if (absum) *absum = s;
    return a;
}

static void anchor_input(const cam_t* k, const double* p, const double* f, int F, double* z) {
    double dv[3] = {p[0] - k->c[0], p[1] - k->c[1], p[2] - k->c[2]};
    double d = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int i = 0; i < F; ++i) z[i] = f[i];
    z[F] = dv[0] / d; z[F + 1] = dv[1] / d; z[F + 2] = dv[2] / d; z[F + 3] = d;
}

/* Gaussian g = r*k + i of selected anchor r.  opac <= 0 marks a dropped Gaussian.
 * means are world coordinates.  op_margin[g] = |raw| / (sum of |terms| of raw). */
void orc_decode(long M, const int64_t* sel_idx, const double* sel_w, const double* pos,
                const double* feat, int F, const double* offs, const double* lv, int k,
                const double* w1, const double* b1, int Hd, const double* w2op,
                const double* b2op, const double* w2col, const double* b2col,
                const double* w2cov, const double* b2cov, const double* camp, double* means,
                double* scales, double* quats, double* opac, double* colors,
                double* op_margin, const double* app, int A, const double* w1app) {
    cam_t cam = read_cam(camp);
    mlp_t W = {w1, b1, w2op, b2op, w2col, b2col, w2cov, b2cov, F, Hd, k, w1app, A};
    double* z = malloc(sizeof(double) * (F + 4));
    double* hid = malloc(sizeof(double) * 3 * Hd);
    double* pre = malloc(sizeof(double) * 3 * Hd);
    for (long r = 0; r < M; ++r) {
        long j = sel_idx[r];
        anchor_input(&cam, pos + 3 * j, feat + (long)j * F, F, z);
        mlp_hidden(&W, z, A > 0 ? app + (long)j * A : NULL, hid, pre);
        const double* hop = hid;
        const double* hcol = hid + Hd;
        const double* hcov = hid + 2 * Hd;
        const double* l = lv + 3 * j;
        for (int i = 0; i < k; ++i) {
            long g = r * k + i;
            double s_abs;
            double raw = mlp_out(w2op, b2op, i, hop, Hd, &s_abs);
            opac[g] = sel_w[r] * tanh(raw);
            if (op_margin) op_margin[g] = fabs(raw) / dmax(s_abs, 1e-300);
            for (int c = 0; c < 3; ++c)
                colors[3 * g + c] = sigmoid(mlp_out(w2col, b2col, 3 * i + c, hcol, Hd, NULL));
            for (int c = 0; c < 3; ++c)
                scales[3 * g + c] = l[c] * sigmoid(mlp_out(w2cov, b2cov, 7 * i + c, hcov, Hd, NULL));
            double q[4], qn = 0;
            for (int c = 0; c < 4; ++c) {
                q[c] = mlp_out(w2cov, b2cov, 7 * i + 3 + c, hcov, Hd, NULL);
                qn += q[c] * q[c];
            }
            qn = sqrt(qn);
            for (int c = 0; c < 4; ++c) quats[4 * g + c] = q[c] / qn;
            const double* O = offs + ((long)j * k + i) * 3;
            for (int c = 0; c < 3; ++c) means[3 * g + c] = pos[3 * j + c] + O[c] * l[c];
        }
    }
    free(z); free(hid); free(pre);
}

/* ------------------------------------------------------------------------------------- */
/* Sec. 3.1: EWA projection and tile extent                                               */
/* ------------------------------------------------------------------------------------- */

static void quat_to_rot(const double* q, double* R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* distance from e to the nearest value 16m + off */
static double grid_dist(double e, double off) {
    double t = (e - off) / ORC_TILE;
    return fabs(t - floor(t + 0.5)) * ORC_TILE;
}

static double floor_div16(double pix) { return floor(pix / ORC_TILE); }

typedef struct {
    double pc[3], Sigma[9], T[6], cov2[3], J[6];
    int clampx, clampy;
} proj_tmp;

/* Forward projection of one Gaussian; returns 0 when culled by the near plane. */
static int project_one(const cam_t* k, const double* mu, const double* s, const double* q,
                       proj_tmp* t) {
    to_cam(k, mu, t->pc);
    if (!(t->pc[2] > k->znear)) return 0;
    double Rq[9], Mm[9];
    quat_to_rot(q, Rq);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Mm[3 * r + c] = Rq[3 * r + c] * s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double a = 0;
            for (int i = 0; i < 3; ++i) a += Mm[3 * r + i] * Mm[3 * c + i];
            t->Sigma[3 * r + c] = a;
        }
    double z = t->pc[2];
    double limx = ORC_FRUSTUM * k->W / (2.0 * k->fx), limy = ORC_FRUSTUM * k->H / (2.0 * k->fy);
    double xz = t->pc[0] / z, yz = t->pc[1] / z;
    t->clampx = xz < -limx || xz > limx;
    t->clampy = yz < -limy || yz > limy;
    double tx = dmin(dmax(xz, -limx), limx) * z, ty = dmin(dmax(yz, -limy), limy) * z;
    double J[6] = {k->fx / z, 0, -k->fx * tx / (z * z), 0, k->fy / z, -k->fy * ty / (z * z)};
    memcpy(t->J, J, sizeof J);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double a = 0;
            for (int i = 0; i < 3; ++i) a += J[3 * r + i] * k->R[3 * i + c];
            t->T[3 * r + c] = a;
        }
    double TS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double a = 0;
            for (int i = 0; i < 3; ++i) a += t->T[3 * r + i] * t->Sigma[3 * i + c];
            TS[3 * r + c] = a;
        }
    double C[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double a = 0;
            for (int i = 0; i < 3; ++i) a += TS[3 * r + i] * t->T[3 * c + i];
            C[2 * r + c] = a;
        }
    t->cov2[0] = C[0]; t->cov2[1] = 0.5 * (C[1] + C[2]); t->cov2[2] = C[3];
    return 1;
}

/* uv: pixel coordinates of the centre; conic = inverse 2D covariance (a, b, c); rect =
 * [x0, y0, x1, y1) tiles, all zero when culled (uv and radius are still reported when only
 * the rectangle is empty).  mz: relative margin of the near-plane test,
 * mpx: pixel distance of the four extent edges to a value that changes the tile rectangle. */
void orc_project(long G, const double* means, const double* scales, const double* quats,
                 const double* opac, const double* camp, double* uv, double* conic,
                 double* depth, double* radius, int32_t* rect, double* mz, double* mpx) {
    cam_t k = read_cam(camp);
    int gx = (k.W + ORC_TILE - 1) / ORC_TILE, gy = (k.H + ORC_TILE - 1) / ORC_TILE;
    for (long g = 0; g < G; ++g) {
        proj_tmp t;
        int32_t* rc = rect + 4 * g;
        rc[0] = rc[1] = rc[2] = rc[3] = 0;
        uv[2 * g] = uv[2 * g + 1] = 0;
        conic[3 * g] = conic[3 * g + 1] = conic[3 * g + 2] = 0;
        depth[g] = 0; radius[g] = 0;
        if (mz) mz[g] = INFINITY;
        if (mpx) mpx[g] = INFINITY;
        if (!(opac[g] > 0)) continue;
        int front = project_one(&k, means + 3 * g, scales + 3 * g, quats + 4 * g, &t);
        double nrm = sqrt(t.pc[0] * t.pc[0] + t.pc[1] * t.pc[1] + t.pc[2] * t.pc[2]);
        if (mz) mz[g] = fabs(t.pc[2] - k.znear) / dmax(nrm, 1e-300);
        if (!front) continue;
        double a = t.cov2[0] + ORC_LOWPASS, b = t.cov2[1], c = t.cov2[2] + ORC_LOWPASS;
        double det = a * c - b * b;
        if (!(det > 0)) continue;
        double mid = 0.5 * (a + c);
        double lam = mid + sqrt(dmax(0.1, mid * mid - det));
        double r = 3.0 * sqrt(lam);
        double u = k.fx * t.pc[0] / t.pc[2] + k.cx;
        double v = k.fy * t.pc[1] / t.pc[2] + k.cy;
        /* tiles holding a pixel centre inside the 3-sigma square */
        double x0 = dmax(floor_div16(ceil(u - r)), 0), x1 = dmin(floor_div16(floor(u + r)) + 1, gx);
        double y0 = dmax(floor_div16(ceil(v - r)), 0), y1 = dmin(floor_div16(floor(v + r)) + 1, gy);
        if (mpx) {
            double m = grid_dist(u - r, -1.0);
            m = dmin(m, grid_dist(u + r, 0.0));
            m = dmin(m, grid_dist(v - r, -1.0));
            m = dmin(m, grid_dist(v + r, 0.0));
            mpx[g] = m;
        }
        /* centre and extent are reported even when the rectangle is empty */
        uv[2 * g] = u; uv[2 * g + 1] = v;
        radius[g] = r;
        if (x0 >= x1 || y0 >= y1) continue;
        conic[3 * g] = c / det; conic[3 * g + 1] = -b / det; conic[3 * g + 2] = a / det;
        depth[g] = t.pc[2];
        rc[0] = (int32_t)x0; rc[1] = (int32_t)y0; rc[2] = (int32_t)x1; rc[3] = (int32_t)y1;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Sec. 3.1: per-tile front-to-back lists                                                 */
/* ------------------------------------------------------------------------------------- */

static const double* g_sort_depth;
static int cmp_depth_id(const void* A, const void* B) {
    int64_t a = *(const int64_t*)A, b = *(const int64_t*)B;
    double da = g_sort_depth[a], db = g_sort_depth[b];
    if (da < db) return -1;
    if (da > db) return 1;
    return (a > b) - (a < b);
}

/* tile_start[gx*gy + 1]; list[P] (Gaussian ids).  Returns P, or -P if cap is too small (lists
 * not written).  tie[t] = smallest relative depth gap between neighbours in tile t's list. */
long orc_tile_lists(long G, const int32_t* rect, const double* depth, int gx, int gy,
                    int64_t* tile_start, int64_t* list, long cap, double* tie) {
    long T = (long)gx * gy;
    for (long t = 0; t <= T; ++t) tile_start[t] = 0;
    for (long g = 0; g < G; ++g) {
        const int32_t* r = rect + 4 * g;
        for (int y = r[1]; y < r[3]; ++y)
            for (int x = r[0]; x < r[2]; ++x) tile_start[(long)y * gx + x + 1]++;
    }
    for (long t = 0; t < T; ++t) tile_start[t + 1] += tile_start[t];
    long P = tile_start[T];
    if (P > cap) return -P;
    long* fill = calloc(T, sizeof(long));
    for (long g = 0; g < G; ++g) {
        const int32_t* r = rect + 4 * g;
        for (int y = r[1]; y < r[3]; ++y)
            for (int x = r[0]; x < r[2]; ++x) {
                long t = (long)y * gx + x;
                list[tile_start[t] + fill[t]++] = g;
            }
    }
    free(fill);
    g_sort_depth = depth;
    for (long t = 0; t < T; ++t) {
        long n = tile_start[t + 1] - tile_start[t];
        qsort(list + tile_start[t], n, sizeof(int64_t), cmp_depth_id);
        if (tie) {
            double m = INFINITY;
            for (long i = tile_start[t] + 1; i < tile_start[t + 1]; ++i) {
                double a = depth[list[i - 1]], b = depth[list[i]];
                m = dmin(m, fabs(b - a) / dmax(fabs(a), 1e-300));
            }
            tie[t] = m;
        }
    }
    return P;
}

/* ------------------------------------------------------------------------------------- */
/* Sec. 3.1, Eq. 2: front-to-back alpha blending                                          */
/* ------------------------------------------------------------------------------------- */

/* Gaussian id g of tile-list entry -> its falloff-weighted opacity at pixel (px, py) */
static double eval_alpha(const double* uv, const double* conic, const double* opac, long g,
                         int px, int py, double* power_out, double* raw_out) {
    double dx = uv[2 * g] - px, dy = uv[2 * g + 1] - py;
    const double* q = conic + 3 * g;
    double power = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy;
    *power_out = power;
    double raw = opac[g] * exp(power);
    *raw_out = raw;
    return dmin(ORC_ALPHA_MAX, raw);
}

/* img[3][H][W], Tfinal[H][W], last[H][W] = number of list entries up to and including the
 * last blended one.  px_margin: smallest relative distance of an alpha-skip or stop test to
 * its threshold at that pixel.  If anchor_of and maxc are given, maxc[anchor] is raised to
 * the largest T_i alpha_i of any blended Gaussian of that anchor.  If depth and px_tie are
 * given, px_tie is the smallest relative depth gap between consecutive Gaussians that take
 * part at the pixel (blended ones and the one that stops it): only such pairs change the
 * pixel when their order flips. */
void orc_blend(int W, int H, const int64_t* tile_start, const int64_t* list, const double* uv,
               const double* conic, const double* opac, const double* colors, const double* bg,
               double* img, double* Tfinal, int32_t* last, double* px_margin,
               const int64_t* anchor_of, double* maxc, const double* depth, double* px_tie) {
    int gx = (W + ORC_TILE - 1) / ORC_TILE;
#pragma omp parallel for schedule(dynamic, 64)
    for (long pix = 0; pix < (long)W * H; ++pix) {
        int px = (int)(pix % W), py = (int)(pix / W);
        long t = (long)(py / ORC_TILE) * gx + px / ORC_TILE;
        double T = 1.0, C[3] = {0, 0, 0}, m = INFINITY, tie = INFINITY, prev_z = -1.0;
        int32_t n_last = 0;
        for (int64_t e = tile_start[t]; e < tile_start[t + 1]; ++e) {
            long g = list[e];
            double power, raw;
            double alpha = eval_alpha(uv, conic, opac, g, px, py, &power, &raw);
            if (power > 0) continue;
            if (raw < ORC_ALPHA_MAX) m = dmin(m, fabs(raw - ORC_ALPHA_MIN) / ORC_ALPHA_MIN);
            if (alpha < ORC_ALPHA_MIN) continue;
            if (depth) {
                if (prev_z >= 0) tie = dmin(tie, fabs(depth[g] - prev_z) / dmax(prev_z, 1e-300));
                prev_z = depth[g];
            }
            double Tn = T * (1.0 - alpha);
            m = dmin(m, fabs(Tn - ORC_T_MIN) / ORC_T_MIN);
            if (Tn < ORC_T_MIN) break;
            for (int c = 0; c < 3; ++c) C[c] += colors[3 * g + c] * alpha * T;
            if (anchor_of && maxc) {
                double contrib = alpha * T;
                long a = anchor_of[g];
#pragma omp critical
                if (contrib > maxc[a]) maxc[a] = contrib;
            }
            T = Tn;
            n_last = (int32_t)(e - tile_start[t] + 1);
        }
        for (int c = 0; c < 3; ++c) img[(long)c * W * H + pix] = C[c] + T * bg[c];
        Tfinal[pix] = T;
        last[pix] = n_last;
        if (px_margin) px_margin[pix] = m;
        if (px_tie) px_tie[pix] = tie;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Backward of Eq. 2 (per-pixel replay, back to front)                                    */
/* ------------------------------------------------------------------------------------- */

/* dimg[3][H][W] = dL/dC.  Accumulates dL/d(uv, conic, opacity, colour) per Gaussian (arrays
 * must be zeroed by the caller).  Derivation: C = sum_i c_i a_i T_i + T_{n+1} bg, so
 * dC/dc_i = a_i T_i and dC/da_i = T_i (c_i - S_i) with S_n = bg, S_{i-1} = a_i c_i +
 * (1 - a_i) S_i; a_i = min(0.99, o G), G = exp(power) (zero derivative where clamped). */
void orc_blend_bwd(int W, int H, const int64_t* tile_start, const int64_t* list,
                   const double* uv, const double* conic, const double* opac,
                   const double* colors, const double* bg, const double* dimg, double* duv,
                   double* dconic, double* dopac, double* dcolors) {
    int gx = (W + ORC_TILE - 1) / ORC_TILE;
    long maxlen = 0;
    for (long t = 0; t < (long)gx * ((H + ORC_TILE - 1) / ORC_TILE); ++t)
        if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
#pragma omp parallel
    {
        long* ids = malloc(sizeof(long) * (maxlen + 1));
        double* al = malloc(sizeof(double) * (maxlen + 1));
        double* Ts = malloc(sizeof(double) * (maxlen + 1));
        int* clamped = malloc(sizeof(int) * (maxlen + 1));
#pragma omp for schedule(dynamic, 64)
        for (long pix = 0; pix < (long)W * H; ++pix) {
            int px = (int)(pix % W), py = (int)(pix / W);
            long t = (long)(py / ORC_TILE) * gx + px / ORC_TILE;
            double T = 1.0;
            long n = 0;
            for (int64_t e = tile_start[t]; e < tile_start[t + 1]; ++e) {
                long g = list[e];
                double power, raw;
                double alpha = eval_alpha(uv, conic, opac, g, px, py, &power, &raw);
                if (power > 0 || alpha < ORC_ALPHA_MIN) continue;
                double Tn = T * (1.0 - alpha);
                if (Tn < ORC_T_MIN) break;
                ids[n] = g; al[n] = alpha; Ts[n] = T; clamped[n] = raw >= ORC_ALPHA_MAX;
                ++n;
                T = Tn;
            }
            double dC[3], S[3];
            for (int c = 0; c < 3; ++c) {
                dC[c] = dimg[(long)c * W * H + pix];
                S[c] = bg[c];
            }
            for (long i = n - 1; i >= 0; --i) {
                long g = ids[i];
                double a = al[i], Ti = Ts[i];
                double dalpha = 0;
                for (int c = 0; c < 3; ++c) {
                    dalpha += dC[c] * Ti * (colors[3 * g + c] - S[c]);
                    double dcol = dC[c] * a * Ti;
#pragma omp atomic
                    dcolors[3 * g + c] += dcol;
                }
                for (int c = 0; c < 3; ++c) S[c] = a * colors[3 * g + c] + (1 - a) * S[c];
                if (clamped[i]) continue;
                double dx = uv[2 * g] - px, dy = uv[2 * g + 1] - py;
                const double* q = conic + 3 * g;
                double G = a / opac[g];
                double dpow = dalpha * a;     /* d(o G)/dpower = o G = a */
                double dop = dalpha * G;
#pragma omp atomic
                dopac[g] += dop;
                double du = dpow * (-(q[0] * dx + q[1] * dy));
                double dv = dpow * (-(q[2] * dy + q[1] * dx));
#pragma omp atomic
                duv[2 * g] += du;
#pragma omp atomic
                duv[2 * g + 1] += dv;
                double da = dpow * (-0.5 * dx * dx), db = dpow * (-dx * dy), dc = dpow * (-0.5 * dy * dy);
#pragma omp atomic
                dconic[3 * g] += da;
#pragma omp atomic
                dconic[3 * g + 1] += db;
#pragma omp atomic
                dconic[3 * g + 2] += dc;
            }
        }
        free(ids); free(al); free(Ts); free(clamped);
    }
}

/* ------------------------------------------------------------------------------------- */
/* Backward of the EWA projection                                                         */
/* ------------------------------------------------------------------------------------- */

/* dmeans/dscales/dquats: gradients w.r.t. world means, scales and the unit quaternion that
 * builds R(q) (accumulated; caller zeroes).  Culled Gaussians (rect empty) get nothing. */
void orc_project_bwd(long G, const double* means, const double* scales, const double* quats,
                     const int32_t* rect, const double* camp, const double* duv,
                     const double* dconic, double* dmeans, double* dscales, double* dquats) {
    cam_t k = read_cam(camp);
    for (long g = 0; g < G; ++g) {
        const int32_t* rc = rect + 4 * g;
        if (rc[0] >= rc[2] || rc[1] >= rc[3]) continue;
        proj_tmp t;
        project_one(&k, means + 3 * g, scales + 3 * g, quats + 4 * g, &t);
        double A = t.cov2[0] + ORC_LOWPASS, B = t.cov2[1], C = t.cov2[2] + ORC_LOWPASS;
        double det = A * C - B * B;
        double K[4] = {C / det, -B / det, -B / det, A / det};
        /* conic parameter gradients -> symmetric matrix gradient of K */
        double gK[4] = {dconic[3 * g], 0.5 * dconic[3 * g + 1], 0.5 * dconic[3 * g + 1],
                        dconic[3 * g + 2]};
        /* dL/dM = -K gK K for M = cov2 + 0.3 I */
        double tmp[4], gM[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                tmp[2 * r + c] = gK[2 * r] * K[c] + gK[2 * r + 1] * K[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                gM[2 * r + c] = -(K[2 * r] * tmp[c] + K[2 * r + 1] * tmp[2 + c]);
        /* cov2 = T Sigma T^T:  dL/dSigma = T^T gM T,  dL/dT = 2 gM T Sigma */
        double gS[9], gT[6], TS[6];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double a = 0;
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) a += t.T[3 * i + r] * gM[2 * i + j] * t.T[3 * j + c];
                gS[3 * r + c] = a;
            }
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double a = 0;
                for (int i = 0; i < 3; ++i) a += t.T[3 * r + i] * t.Sigma[3 * i + c];
                TS[3 * r + c] = a;
            }
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                gT[3 * r + c] = 2.0 * (gM[2 * r] * TS[c] + gM[2 * r + 1] * TS[3 + c]);
        /* T = J W: dL/dJ = gT W^T */
        double gJ[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double a = 0;
                for (int i = 0; i < 3; ++i) a += gT[3 * r + i] * k.R[3 * c + i];
                gJ[3 * r + c] = a;
            }
        double x = t.pc[0], y = t.pc[1], z = t.pc[2];
        double limx = ORC_FRUSTUM * k.W / (2.0 * k.fx), limy = ORC_FRUSTUM * k.H / (2.0 * k.fy);
        double gp[3] = {0, 0, 0};
        /* J00 = fx/z, J02 = -fx tx/z^2 with tx = x (unclamped) or lim_signed z (clamped) */
        gp[2] += gJ[0] * (-k.fx / (z * z)) + gJ[4] * (-k.fy / (z * z));
        if (!t.clampx) {
            gp[0] += gJ[2] * (-k.fx / (z * z));
            gp[2] += gJ[2] * (2.0 * k.fx * x / (z * z * z));
        } else {
            double ls = (x / z < 0 ? -limx : limx);
            gp[2] += gJ[2] * (k.fx * ls / (z * z));
        }
        if (!t.clampy) {
            gp[1] += gJ[5] * (-k.fy / (z * z));
            gp[2] += gJ[5] * (2.0 * k.fy * y / (z * z * z));
        } else {
            double ls = (y / z < 0 ? -limy : limy);
            gp[2] += gJ[5] * (k.fy * ls / (z * z));
        }
        /* u = fx x/z + cx, v = fy y/z + cy */
        gp[0] += duv[2 * g] * k.fx / z;
        gp[2] += duv[2 * g] * (-k.fx * x / (z * z));
        gp[1] += duv[2 * g + 1] * k.fy / z;
        gp[2] += duv[2 * g + 1] * (-k.fy * y / (z * z));
        /* pc = W (mu - c): dL/dmu = W^T gp */
        for (int c = 0; c < 3; ++c)
            dmeans[3 * g + c] += k.R[c] * gp[0] + k.R[3 + c] * gp[1] + k.R[6 + c] * gp[2];
        /* Sigma = M M^T, M = R(q) S: dL/dM = 2 gS M */
        double Rq[9], Mm[9], gMm[9];
        quat_to_rot(quats + 4 * g, Rq);
        const double* s = scales + 3 * g;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Mm[3 * r + c] = Rq[3 * r + c] * s[c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double a = 0;
                for (int i = 0; i < 3; ++i) a += gS[3 * r + i] * Mm[3 * i + c];
                gMm[3 * r + c] = 2.0 * a;
            }
        double gR[9];
        for (int c = 0; c < 3; ++c) {
            double a = 0;
            for (int r = 0; r < 3; ++r) {
                a += gMm[3 * r + c] * Rq[3 * r + c];
                gR[3 * r + c] = gMm[3 * r + c] * s[c];
            }
            dscales[3 * g + c] += a;
        }
        const double* q = quats + 4 * g;
        double w = q[0], qx = q[1], qy = q[2], qz = q[3];
        dquats[4 * g + 0] += 2 * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
        dquats[4 * g + 1] += 2 * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2 * qx * gR[4] - w * gR[5] +
                                  qz * gR[6] + w * gR[7] - 2 * qx * gR[8]);
        dquats[4 * g + 2] += 2 * (-2 * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] -
                                  w * gR[6] + qz * gR[7] - 2 * qy * gR[8]);
        dquats[4 * g + 3] += 2 * (-2 * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2 * qz * gR[4] +
                                  qy * gR[5] + qx * gR[6] + qy * gR[7]);
    }
}

/* ------------------------------------------------------------------------------------- */
/* Backward of the decoders (Eq. offsets, Eq. mlp)                                        */
/* ------------------------------------------------------------------------------------- */

/* Per-Gaussian gradients (dmeans, dscales, dquats w.r.t. the unit quaternion, dopac, dcolors)
 * -> anchor feature / offset / scaling gradients and decoder weight gradients (all
 * accumulated; caller zeroes).  Anchor positions, LOD bias and selection are constants. */
void orc_decode_bwd(long M, const int64_t* sel_idx, const double* sel_w, const double* pos,
                    const double* feat, int F, const double* offs, const double* lv, int k,
                    const double* w1, const double* b1, int Hd, const double* w2op,
                    const double* b2op, const double* w2col, const double* b2col,
                    const double* w2cov, const double* b2cov, const double* camp,
                    const double* dmeans, const double* dscales, const double* dquats,
                    const double* dopac, const double* dcolors, double* dfeat, double* doffs,
                    double* dlv, double* dw1, double* db1, double* dw2op, double* db2op,
                    double* dw2col, double* db2col, double* dw2cov, double* db2cov,
                    const double* app, int A, const double* w1app, double* dapp,
                    double* dw1app) {
    cam_t cam = read_cam(camp);
    mlp_t W = {w1, b1, w2op, b2op, w2col, b2col, w2cov, b2cov, F, Hd, k, w1app, A};
    int Din = F + 4;
    double* z = malloc(sizeof(double) * Din);
    double* hid = malloc(sizeof(double) * 3 * Hd);
    double* pre = malloc(sizeof(double) * 3 * Hd);
    double* dhid = malloc(sizeof(double) * 3 * Hd);
    for (long r = 0; r < M; ++r) {
        long j = sel_idx[r];
        const double* aj = A > 0 ? app + (long)j * A : NULL;
        anchor_input(&cam, pos + 3 * j, feat + (long)j * F, F, z);
        mlp_hidden(&W, z, aj, hid, pre);
        for (int h = 0; h < 3 * Hd; ++h) dhid[h] = 0;
        const double* l = lv + 3 * j;
        for (int i = 0; i < k; ++i) {
            long g = r * k + i;
            /* opacity: o = w tanh(raw), Gaussian dropped if o <= 0 */
            double raw = mlp_out(w2op, b2op, i, hid, Hd, NULL);
            double o = sel_w[r] * tanh(raw);
            if (o > 0) {
                double th = tanh(raw);
                double draw = dopac[g] * sel_w[r] * (1 - th * th);
                db2op[i] += draw;
                for (int h = 0; h < Hd; ++h) {
                    dw2op[(long)i * Hd + h] += draw * hid[h];
                    dhid[h] += draw * w2op[(long)i * Hd + h];
                }
            }
            /* colour: sigmoid */
            for (int c = 0; c < 3; ++c) {
                int row = 3 * i + c;
                double sg = sigmoid(mlp_out(w2col, b2col, row, hid + Hd, Hd, NULL));
                double draw = dcolors[3 * g + c] * sg * (1 - sg);
                db2col[row] += draw;
                for (int h = 0; h < Hd; ++h) {
                    dw2col[(long)row * Hd + h] += draw * hid[Hd + h];
                    dhid[Hd + h] += draw * w2col[(long)row * Hd + h];
                }
            }
            /* scale = l_v * sigmoid(raw) */
            for (int c = 0; c < 3; ++c) {
                int row = 7 * i + c;
                double sg = sigmoid(mlp_out(w2cov, b2cov, row, hid + 2 * Hd, Hd, NULL));
                dlv[3 * j + c] += dscales[3 * g + c] * sg;
                double draw = dscales[3 * g + c] * l[c] * sg * (1 - sg);
                db2cov[row] += draw;
                for (int h = 0; h < Hd; ++h) {
                    dw2cov[(long)row * Hd + h] += draw * hid[2 * Hd + h];
                    dhid[2 * Hd + h] += draw * w2cov[(long)row * Hd + h];
                }
            }
            /* quaternion = raw / |raw|: d raw = (dq - q (q . dq)) / |raw| */
            double q[4], qn = 0;
            for (int c = 0; c < 4; ++c) {
                q[c] = mlp_out(w2cov, b2cov, 7 * i + 3 + c, hid + 2 * Hd, Hd, NULL);
                qn += q[c] * q[c];
            }
            qn = sqrt(qn);
            double qdot = 0;
            for (int c = 0; c < 4; ++c) {
                q[c] /= qn;
                qdot += q[c] * dquats[4 * g + c];
            }
            for (int c = 0; c < 4; ++c) {
                int row = 7 * i + 3 + c;
                double draw = (dquats[4 * g + c] - q[c] * qdot) / qn;
                db2cov[row] += draw;
                for (int h = 0; h < Hd; ++h) {
                    dw2cov[(long)row * Hd + h] += draw * hid[2 * Hd + h];
                    dhid[2 * Hd + h] += draw * w2cov[(long)row * Hd + h];
                }
            }
            /* mu = x_v + O * l_v */
            const double* O = offs + ((long)j * k + i) * 3;
            for (int c = 0; c < 3; ++c) {
                doffs[((long)j * k + i) * 3 + c] += dmeans[3 * g + c] * l[c];
                dlv[3 * j + c] += dmeans[3 * g + c] * O[c];
            }
        }
        /* hidden layers: relu, then W1 */
        for (int m = 0; m < 3; ++m)
            for (int h = 0; h < Hd; ++h) {
                int idx = m * Hd + h;
                if (!(pre[idx] > 0)) continue;
                double dp = dhid[idx];
                db1[idx] += dp;
                for (int i = 0; i < Din; ++i) dw1[(long)idx * Din + i] += dp * z[i];
                for (int i = 0; i < F; ++i) dfeat[(long)j * F + i] += dp * w1[(long)idx * Din + i];
                if (m == 1 && A > 0)                  /* appearance code of the colour MLP */
                    for (int c = 0; c < A; ++c) {
                        dw1app[(long)h * A + c] += dp * aj[c];
                        dapp[(long)j * A + c] += dp * w1app[(long)h * A + c];
                    }
            }
    }
    free(z); free(hid); free(pre); free(dhid);
}
