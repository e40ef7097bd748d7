// DQO-MAP hot-path oracle: a plain, slow FP64 CPU restatement of what the GPU path
// computes.  TEST INFRASTRUCTURE ONLY: it is linked by the tests, the smoke check and
// the bench's CPU-baseline leg, never by the library.  It shares no code, header,
// table or constant generator with the CUDA path.
//
// What it follows (DQO-MAP, arXiv 2503.02223):
//   * Sec. III-A Eq. 1-3: dual quadric Q* of an ellipsoid (centre, rotation, semi-axes).
//   * Sec. III-B Eq. 4: image dual conic C* = P Q* P^T (the printed P^T Q* P is
//     dimensionally impossible for a 3x4 P; the 3x3 reading is used).
//   * Sec. III-D Eq. 12: bbox loss over the frames observing an object, read as
//     sum (1 - IoU(BBox(C*), BBox_obs)).
//   * Sec. III-D Eq. 7-10, 15: colour, depth and instance losses of the Gaussian-splatting
//     render; ins = sum of blend weights of the pixel's own object's opaque Gaussians.
//   * Sec. IV (impl.): rasterization and its backward pass run as CUDA kernels -- the
//     rasterizer is the 3D Gaussian Splatting one the paper builds on (Sec. I, II-B);
//     its unstated constants are the settings struct below.
//
// Conventions (readings where the paper is silent):
//   pixel (u,v) centre at integer (u,v); u = fx x/z + cx.
//   Gaussian: p_c = R_view mean + t_view; Sigma = R(q) diag(exp(2 s)) R(q)^T (q normalised);
//   Sigma' = J W Sigma W^T J^T + lowpass I; conic = Sigma'^-1; radius = ceil(k sqrt(lmax)).
//   Tile membership: tile contains a pixel centre inside [x-hx, x+hx] x [y-hy, y+hy], the
//   3-sigma square (hx = hy = r) narrowed, when alpha_min > 0, to the bounding box of the
//   ellipse q <= T' outside of which no pixel can blend the Gaussian: alpha <= o G, so a
//   blended pixel has q <= T = 2 ln(o / alpha_min).  T' = T (1 + 2^-10) + 2^-14 (a + c)
//   R^2 + 2^-10 (a, c the conic's diagonal, R = r + max(tile_w, tile_h)) widens it by more
//   than the single-precision evaluation of G can move q within the square's tiles;
//   hx = min(r, sqrt(T' Sigma'_xx)), hy = min(r, sqrt(T' Sigma'_yy)); T' <= 0 culls.  The rule
//   removes only (tile, Gaussian) pairs whose pixels all skip the Gaussian, so no pixel
//   value depends on it (pinned by brute force in tests/).
//   Per pixel: tile's Gaussians sorted by (float bit pattern of z, index), the 3DGS depth
//   key; alpha = min(clamp, o exp(power));
//   skip alpha < alpha_min; stop before the Gaussian that would make T(1-alpha) < t_stop.
//   C = sum w c + T_final bg; D = sum w z; A = sum w; ins = sum over Gaussians of the
//   pixel's labelled object (opaque ones if og_filter) of w; id = argmax_k W_k.
//   Losses (mean over H*W pixels, labelled pixels only): L1 colour, L1 depth (where the
//   target depth > 0), L1 of (ins - 1); total = rgb + depth + lambda * ins.
//   The derivative of |x| is sign(x) with sign(0) = 0.
//
// Quadric: params (centre xyz, log a b c, rotation vector); Q* = Z diag(a^2,b^2,c^2,-1) Z^T,
//   Z = [R t; 0 1].  BBox(C*) from the vertical / horizontal tangent lines l with
//   l^T C* l = 0.  A pair is valid iff c33 < 0, the centre is in front and both
//   discriminants are positive; invalid pairs are left out of the loss.
//   Gradients of the quadric loss are computed by forward-mode dual numbers run through
//   the same forward code (an exact derivative, no hand-derived adjoint).
//
// Parity pins live in tests/: closed-form single Gaussian, sphere-quadric radius,
// silhouette brute force, invariants, tiled vs per-pixel brute force, finite
// differences of every gradient.

#include <algorithm>
#include <array>
#define _USE_MATH_DEFINES
#include <cmath>
#include <map>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

struct OSettings {
    int32_t tile_w, tile_h;
    double alpha_clamp;   // alpha = min(alpha_clamp, o G)
    double alpha_min;     // skip if alpha < alpha_min
    double t_stop;        // stop before T (1 - alpha) < t_stop
    double znear;         // cull if z < znear
    double lowpass;       // added to the 2D covariance diagonal (px^2)
    double radius_sigma;  // radius = ceil(radius_sigma * sqrt(lambda_max))
    double lambda_ins;    // weight of the instance loss (Eq. 10)
    double bg[3];         // background colour
    int32_t og_filter;    // 1: only opaque (flag bit0) Gaussians count toward ins (Eq. 15)
    int32_t num_objects;  // object ids outside [0, num_objects) carry no object
    double amb_rel;       // relative margin for flagging threshold decisions
    double amb_px;        // pixel margin for flagging tile-membership decisions
    double theta_alpha, theta_d, theta_c;  // Eq. 11 thresholds
};

struct OCamera {
    double fx, fy, cx, cy;
    int32_t width, height;
    double viewmat[12];  // row-major [R | t], world -> camera
};

}  // extern "C"

namespace {

// ------------------------------------------------------------------ projection (per Gaussian)

struct Proj {
    bool visible = false;
    bool ambiguous = false;    // a discrete decision is within the flagging margin
    double pc[3] = {0, 0, 0};  // camera-space mean
    double xy[2] = {0, 0};
    double cov2[3] = {0, 0, 0};   // Sigma' entries (A, B, C)
    double conic[3] = {0, 0, 0};  // Sigma'^-1 entries (a, b, c)
    double opac = 0;
    double lmax = 0;
    int radius = 0;
    int rect[4] = {0, 0, 0, 0};   // tx0, ty0, tx1, ty1 (exclusive); empty if invisible
    int urect[4] = {0, 0, 0, 0};  // union of rects over the flagging perturbations
    int irect[4] = {0, 0, 0, 0};  // their intersection (empty if any of them is empty)
    double S3[3][3];              // world-space 3D covariance
    double Rq[3][3];              // rotation from the normalised quaternion
    double qn[4];                 // normalised quaternion
    double qnorm = 1;
    double s[3];                  // exp(log_scales)
    double T2[2][3];              // J W
    double J[2][3];
};

void quat_to_rot(const double q[4], double R[3][3]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

// Tiles containing a pixel centre inside the box [x-hx, x+hx] x [y-hy, y+hy].
bool tile_rect(double x, double y, double hx, double hy, const OSettings& st, const OCamera& cam, int rect[4]) {
    double ulo = std::ceil(x - hx), uhi = std::floor(x + hx);
    double vlo = std::ceil(y - hy), vhi = std::floor(y + hy);
    if (ulo < 0) ulo = 0;
    if (vlo < 0) vlo = 0;
    if (uhi > cam.width - 1) uhi = cam.width - 1;
    if (vhi > cam.height - 1) vhi = cam.height - 1;
    if (ulo > uhi || vlo > vhi) { rect[0] = rect[1] = rect[2] = rect[3] = 0; return false; }
    rect[0] = (int)ulo / st.tile_w;
    rect[1] = (int)vlo / st.tile_h;
    rect[2] = (int)uhi / st.tile_w + 1;
    rect[3] = (int)vhi / st.tile_h + 1;
    return true;
}

Proj project_gaussian(const OSettings& st, const OCamera& cam, const double* mean,
                      const double* log_scale, const double* quat, double opacity_logit) {
    Proj P;
    const double* V = cam.viewmat;
    for (int i = 0; i < 3; ++i)
        P.pc[i] = V[4 * i + 0] * mean[0] + V[4 * i + 1] * mean[1] + V[4 * i + 2] * mean[2] + V[4 * i + 3];
    const double x = P.pc[0], y = P.pc[1], z = P.pc[2];
    if (!(z >= st.znear)) {
        P.ambiguous = std::fabs(z - st.znear) <= st.amb_rel * st.znear;
        return P;
    }
    // 3D covariance from the normalised quaternion and exponentiated scales
    double qq = 0;
    for (int i = 0; i < 4; ++i) qq += quat[i] * quat[i];
    P.qnorm = std::sqrt(qq);
    for (int i = 0; i < 4; ++i) P.qn[i] = quat[i] / P.qnorm;
    quat_to_rot(P.qn, P.Rq);
    for (int i = 0; i < 3; ++i) P.s[i] = std::exp(log_scale[i]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += P.Rq[i][k] * P.s[k] * P.s[k] * P.Rq[j][k];
            P.S3[i][j] = acc;
        }
    // EWA: Jacobian of (fx x/z + cx, fy y/z + cy) at the camera-space mean
    P.J[0][0] = cam.fx / z; P.J[0][1] = 0;           P.J[0][2] = -cam.fx * x / (z * z);
    P.J[1][0] = 0;          P.J[1][1] = cam.fy / z;  P.J[1][2] = -cam.fy * y / (z * z);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += P.J[i][k] * V[4 * k + j];
            P.T2[i][j] = acc;
        }
    double C2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += P.T2[i][k] * P.S3[k][l] * P.T2[j][l];
            C2[i][j] = acc;
        }
    P.cov2[0] = C2[0][0] + st.lowpass;
    P.cov2[1] = 0.5 * (C2[0][1] + C2[1][0]);
    P.cov2[2] = C2[1][1] + st.lowpass;
    const double det = P.cov2[0] * P.cov2[2] - P.cov2[1] * P.cov2[1];
    if (!(det > 0)) return P;
    P.conic[0] = P.cov2[2] / det;
    P.conic[1] = -P.cov2[1] / det;
    P.conic[2] = P.cov2[0] / det;
    const double mid = 0.5 * (P.cov2[0] + P.cov2[2]);
    P.lmax = mid + std::sqrt(std::max(0.0, mid * mid - det));
    const double rr = st.radius_sigma * std::sqrt(P.lmax);
    P.radius = (int)std::ceil(rr);
    P.xy[0] = cam.fx * x / z + cam.cx;
    P.xy[1] = cam.fy * y / z + cam.cy;
    P.opac = 1.0 / (1.0 + std::exp(-opacity_logit));
    // the alpha_min ellipse's half-widths (infinite when alpha_min = 0: no narrowing)
    double ex = INFINITY, ey = INFINITY, Tm = 1.0, Tscale = 0.0;
    if (st.alpha_min > 0) {
        const double T = 2.0 * std::log(P.opac / st.alpha_min);
        const double R = P.radius + (double)std::max(st.tile_w, st.tile_h);
        Tm = T * (1.0 + std::ldexp(1.0, -10)) + std::ldexp(1.0, -14) * (P.conic[0] + P.conic[2]) * R * R +
             std::ldexp(1.0, -10);
        Tscale = std::fabs(T) + 1.0;
        if (Tm > 0) {
            ex = std::sqrt(Tm * P.cov2[0]);
            ey = std::sqrt(Tm * P.cov2[2]);
        }
    }
    P.visible = Tm > 0 && tile_rect(P.xy[0], P.xy[1], std::min((double)P.radius, ex),
                                    std::min((double)P.radius, ey), st, cam, P.rect);
    if (!P.visible) P.rect[0] = P.rect[1] = P.rect[2] = P.rect[3] = 0;

    // Flag decisions that single precision may take the other way: the radius rounding,
    // the sign of T', the ellipse's half-widths (relative amb_rel), and the tile rect under
    // a shift of the centre by amb_px.  The rect grows with r, hx and hy, so the low and the
    // high perturbations of all three bound every mix of them.
    int rlo = (int)std::ceil(rr * (1 - st.amb_rel)), rhi = (int)std::ceil(rr * (1 + st.amb_rel));
    bool amb = (rlo != P.radius) || (rhi != P.radius) ||
               std::fabs(z - st.znear) <= st.amb_rel * st.znear || std::fabs(Tm) <= st.amb_rel * Tscale;
    int u[4] = {P.rect[0], P.rect[1], P.rect[2], P.rect[3]};
    int in4[4] = {P.rect[0], P.rect[1], P.rect[2], P.rect[3]};
    bool all = P.visible;
    bool any = P.visible;
    for (int side : {-1, 1}) {
        const int rad = side < 0 ? rlo : rhi;
        const double f = 1.0 + side * st.amb_rel;
        const bool vis_t = Tm + side * st.amb_rel * Tscale > 0;
        for (int dxs = -1; dxs <= 1; ++dxs)
            for (int dys = -1; dys <= 1; ++dys) {
                int r2[4];
                bool v2 = vis_t && tile_rect(P.xy[0] + dxs * st.amb_px, P.xy[1] + dys * st.amb_px,
                                             std::min((double)rad, ex * f), std::min((double)rad, ey * f), st,
                                             cam, r2);
                if (v2 != P.visible || (v2 && (r2[0] != P.rect[0] || r2[1] != P.rect[1] ||
                                               r2[2] != P.rect[2] || r2[3] != P.rect[3])))
                    amb = true;
                if (v2) {
                    if (!any) { for (int k = 0; k < 4; ++k) u[k] = r2[k]; any = true; }
                    u[0] = std::min(u[0], r2[0]); u[1] = std::min(u[1], r2[1]);
                    u[2] = std::max(u[2], r2[2]); u[3] = std::max(u[3], r2[3]);
                    in4[0] = std::max(in4[0], r2[0]); in4[1] = std::max(in4[1], r2[1]);
                    in4[2] = std::min(in4[2], r2[2]); in4[3] = std::min(in4[3], r2[3]);
                } else {
                    all = false;
                }
            }
    }
    P.ambiguous = amb;
    for (int k = 0; k < 4; ++k) P.urect[k] = any ? u[k] : 0;
    for (int k = 0; k < 4; ++k) P.irect[k] = all ? in4[k] : 0;
    return P;
}

struct Inputs {
    int64_t n;
    const double *means, *log_scales, *quats, *opacity_logit, *rgb;
    const int32_t* obj_id;
    const uint8_t* flags;
};

std::vector<Proj> project_all(const OSettings& st, const OCamera& cam, const Inputs& in) {
    std::vector<Proj> pr((size_t)in.n);
    for (int64_t i = 0; i < in.n; ++i)
        pr[i] = project_gaussian(st, cam, in.means + 3 * i, in.log_scales + 3 * i, in.quats + 4 * i,
                                 in.opacity_logit[i]);
    return pr;
}

bool covers(const int rect[4], int tx, int ty) {
    return tx >= rect[0] && tx < rect[2] && ty >= rect[1] && ty < rect[3];
}

// Depth-sort key: the single-precision bit pattern of the camera depth (3DGS sorts its
// tile lists by float depth keys), rounded once from the exact double value; ties by index.
uint32_t depth_key(double z) {
    const float f = (float)z;
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}

bool depth_less(const std::vector<Proj>& pr, int64_t a, int64_t b) {
    const uint32_t ka = depth_key(pr[a].pc[2]), kb = depth_key(pr[b].pc[2]);
    if (ka != kb) return ka < kb;
    return a < b;
}

// Gaussians whose rect covers tile (tx,ty), in ascending (depth key, index) order.
std::vector<int64_t> tile_list(const std::vector<Proj>& pr, int tx, int ty) {
    std::vector<int64_t> L;
    for (int64_t i = 0; i < (int64_t)pr.size(); ++i)
        if (pr[i].visible && covers(pr[i].rect, tx, ty)) L.push_back(i);
    std::stable_sort(L.begin(), L.end(), [&](int64_t a, int64_t b) { return depth_less(pr, a, b); });
    return L;
}

// ------------------------------------------------------------------ per-pixel blending

struct Contrib {
    int64_t g;
    double alpha, T, G, dx, dy;
    bool clamped;
    size_t pos;  // position in the tile list
};

struct PixelResult {
    double C[3] = {0, 0, 0}, D = 0, A = 0, ins = 0, T = 1;
    int64_t n_contrib = 0;  // 1 + list position of the last blended Gaussian
    int64_t last_g = -1;    // index of the last blended Gaussian (-1: none)
    int32_t id = -1;
    double id_margin = 0;
    uint8_t amb = 0;        // bit0 threshold, bit2 tile membership, bit3 loss kink
    // every (Gaussian, kind) whose decision is near its threshold here; kind 1 alpha_min
    // skip, 2 clamp, 3 stop
    std::vector<std::pair<int64_t, int>> near;
    int64_t stop_pos = -1;  // list position where the walk stopped (-1: ran to the end)
    std::vector<int64_t> amb_rect;  // Gaussians whose uncertain tile membership matters here
    std::vector<Contrib> contribs;
};

const uint8_t AMB_THRESH = 1, AMB_RECT = 4, AMB_KINK = 8;
const int FLIP_SKIP = 1, FLIP_CLAMP = 2, FLIP_STOP = 3;

bool near_rel(double a, double b, double rel) { return std::fabs(a - b) <= rel * std::fabs(b); }

// A decision taken the other way: Gaussian g's alpha_min skip, clamp or stop decision.
struct Flip {
    int64_t g;
    int kind;
};

// Front-to-back blend of one pixel over the tile list L.  `flips` inverts the listed
// decisions (used to measure how much decisions near their thresholds matter).
PixelResult blend_pixel(const OSettings& st, const Inputs& in, const std::vector<Proj>& pr,
                        const std::vector<int64_t>& L, int px, int py, int32_t gt, bool keep,
                        const std::vector<Flip>& flips = {}) {
    PixelResult R;
    std::vector<double> Wk(st.num_objects > 0 ? st.num_objects : 0, 0.0);
    double T = 1.0;
    double eT = 0;  // relative error a single-precision evaluation may have accumulated in T
    for (size_t j = 0; j < L.size(); ++j) {
        const int64_t g = L[j];
        const Proj& P = pr[g];
        const double dx = px - P.xy[0], dy = py - P.xy[1];
        const double power = -0.5 * (P.conic[0] * dx * dx + P.conic[2] * dy * dy) - P.conic[1] * dx * dy;
        if (power > 0) continue;
        const double G = std::exp(power);
        const double oG = P.opac * G;
        // Single precision stores the pixel-space mean rounded to half an ulp; the
        // exponent then moves by |grad| * ulp / 2 and alpha by that much relatively.
        const double ulpx = std::ldexp(1.0, std::ilogb(std::fabs(P.xy[0]) + 1.0) - 23);
        const double ulpy = std::ldexp(1.0, std::ilogb(std::fabs(P.xy[1]) + 1.0) - 23);
        const double ea = 0.5 * (std::fabs(P.conic[0] * dx + P.conic[1] * dy) * ulpx +
                                 std::fabs(P.conic[1] * dx + P.conic[2] * dy) * ulpy) + 1e-6;
        const double marg = std::max(st.amb_rel, 4 * ea);
        auto flipped = [&](int kind) {
            for (const Flip& f : flips)
                if (f.g == g && f.kind == kind) return true;
            return false;
        };
        bool clamped = oG > st.alpha_clamp;
        if (flipped(FLIP_CLAMP)) clamped = !clamped;
        const double alpha = clamped ? st.alpha_clamp : oG;
        auto mark = [&](int kind) {
            R.amb |= AMB_THRESH;
            R.near.push_back({g, kind});
        };
        if (near_rel(oG, st.alpha_clamp, marg)) mark(FLIP_CLAMP);
        else if (near_rel(alpha, st.alpha_min, marg)) mark(FLIP_SKIP);
        if ((alpha < st.alpha_min) != flipped(FLIP_SKIP)) continue;
        const double Tn = T * (1 - alpha);
        eT += (clamped ? 0.0 : alpha * ea / (1 - alpha)) + 1e-7;
        if (near_rel(Tn, st.t_stop, std::max(st.amb_rel, 4 * eT))) mark(FLIP_STOP);
        if ((Tn < st.t_stop) != flipped(FLIP_STOP)) {
            R.stop_pos = (int64_t)j;
            break;
        }
        const double w = alpha * T;
        for (int c = 0; c < 3; ++c) R.C[c] += w * in.rgb[3 * g + c];
        R.D += w * P.pc[2];
        R.A += w;
        const int32_t id = in.obj_id[g];
        const bool has_obj = id >= 0 && id < st.num_objects;
        if (has_obj) {
            Wk[id] += w;
            const bool og = !st.og_filter || (in.flags[g] & 1);
            if (og && id == gt) R.ins += w;
        }
        if (keep) R.contribs.push_back({g, alpha, T, G, dx, dy, clamped, j});
        T = Tn;
        R.n_contrib = (int64_t)j + 1;
        R.last_g = g;
    }
    R.T = T;
    for (int c = 0; c < 3; ++c) R.C[c] += T * st.bg[c];
    // argmax over objects, ties to the smallest id, -1 if nothing was blended
    double best = 0, second = 0;
    for (int k = 0; k < st.num_objects; ++k) {
        if (Wk[k] > best) { second = best; best = Wk[k]; R.id = k; }
        else if (Wk[k] > second) second = Wk[k];
    }
    R.id_margin = best - second;
    return R;
}

struct PixelGrad { double dC[3], dD, dA, dins; };

// Loss terms of one pixel (Eq. 7-10 reading) and dL/d(outputs).
void pixel_loss(const OSettings& st, const PixelResult& R, const double* trgb, double tdepth, int32_t gt,
                double inv_hw, double loss[3], PixelGrad& g, uint8_t& amb) {
    g = PixelGrad{{0, 0, 0}, 0, 0, 0};
    if (gt < 0) return;
    auto sgn = [](double v) { return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0); };
    for (int c = 0; c < 3; ++c) {
        const double e = R.C[c] - trgb[c];
        loss[0] += std::fabs(e) * inv_hw;
        g.dC[c] = sgn(e) * inv_hw;
        if (e != 0 && std::fabs(e) < 1e-4) amb |= AMB_KINK;
    }
    if (tdepth > 0) {
        const double e = R.D - tdepth;
        loss[1] += std::fabs(e) * inv_hw;
        g.dD = sgn(e) * inv_hw;
        if (e != 0 && std::fabs(e) < 1e-4) amb |= AMB_KINK;
    }
    const double e = R.ins - 1.0;
    loss[2] += std::fabs(e) * inv_hw;
    g.dins = st.lambda_ins * sgn(e) * inv_hw;
}

// 2D gradient record per Gaussian: dxy(2), dconic(3: a,b,c), dopac, drgb(3), dz.
const int G2 = 10;

// Adjoint of one pixel's blend (plain definition: C = sum c_j a_j T_j + T_N bg, etc.).
// acc(g) returns the 10-entry record of Gaussian g to add into.
struct NoMag {
    double* operator()(int64_t) const { return nullptr; }
};

// acc(g): record to add the terms into; mag(g) (may return NULL): record to add their
// magnitudes into.
template <class Acc, class Mag = NoMag>
void pixel_backward(const OSettings& st, const Inputs& in, const std::vector<Proj>& pr,
                    const PixelResult& R, const PixelGrad& pg, int32_t gt, Acc acc, Mag mag = Mag()) {
    const size_t n = R.contribs.size();
    // suffix sums of w_k * (upstream . value_k) behind each contributor, plus the background
    double behind = R.T * (pg.dC[0] * st.bg[0] + pg.dC[1] * st.bg[1] + pg.dC[2] * st.bg[2]);
    for (size_t jj = n; jj-- > 0;) {
        const Contrib& c = R.contribs[jj];
        const int64_t g = c.g;
        const Proj& P = pr[g];
        const int32_t id = in.obj_id[g];
        const bool counts = id >= 0 && id < st.num_objects && id == gt && (!st.og_filter || (in.flags[g] & 1));
        const double U = pg.dC[0] * in.rgb[3 * g] + pg.dC[1] * in.rgb[3 * g + 1] + pg.dC[2] * in.rgb[3 * g + 2] +
                         pg.dD * P.pc[2] + pg.dA + (counts ? pg.dins : 0.0);
        const double w = c.alpha * c.T;
        // dL/dalpha_j = T_j U_j - (sum_{k>j} w_k U_k + T_N bg.dC) / (1 - alpha_j)
        const double dalpha = c.T * U - behind / (1 - c.alpha);
        behind += w * U;
        double t[G2] = {0, 0, 0, 0, 0, 0, w * pg.dC[0], w * pg.dC[1], w * pg.dC[2], w * pg.dD};
        if (!c.clamped) {
            // alpha = o G, G = exp(power), power = -(a dx^2 + c dy^2)/2 - b dx dy, dx = px - x
            t[5] = dalpha * c.G;
            const double dpow = dalpha * P.opac * c.G;
            t[0] = dpow * (P.conic[0] * c.dx + P.conic[1] * c.dy);
            t[1] = dpow * (P.conic[1] * c.dx + P.conic[2] * c.dy);
            t[2] = dpow * (-0.5 * c.dx * c.dx);
            t[3] = dpow * (-c.dx * c.dy);
            t[4] = dpow * (-0.5 * c.dy * c.dy);
        }
        double* o = acc(g);
        for (int k = 0; k < G2; ++k) o[k] += t[k];
        if (double* m = mag(g))
            for (int k = 0; k < G2; ++k) m[k] += std::fabs(t[k]);
    }
}

// Magnitude arithmetic: every value is replaced by its absolute value and every sum or
// difference by the sum of the absolute values, so that a chain of operations evaluated
// on Mag gives the sum of the magnitudes of all the terms it combines (the quantity a
// first-order bound on its floating-point rounding is proportional to).
struct Mag {
    double v = 0;
    Mag() = default;
    Mag(double x) : v(std::fabs(x)) {}
    Mag& operator+=(const Mag& o) { v += o.v; return *this; }
    Mag& operator-=(const Mag& o) { v += o.v; return *this; }
};
Mag operator+(const Mag& a, const Mag& b) { return Mag(a.v + b.v); }
Mag operator-(const Mag& a, const Mag& b) { return Mag(a.v + b.v); }
Mag operator-(const Mag& a) { return a; }
Mag operator*(const Mag& a, double b) { return Mag(a.v * std::fabs(b)); }
Mag operator*(double a, const Mag& b) { return Mag(std::fabs(a) * b.v); }
Mag operator/(const Mag& a, double b) { return Mag(a.v / std::fabs(b)); }

// Chain a Gaussian's 2D gradient record back to its parameters (T = double; T = Mag
// evaluates the same chain on magnitudes).
template <class T>
void preprocess_backward(const OSettings& st, const OCamera& cam, const Proj& P, double opacity_logit,
                         const T* g2, T* dmean, T* dlog_scale, T* dquat, T* dlogit, T* drgb) {
    (void)st;
    for (int c = 0; c < 3; ++c) drgb[c] += g2[6 + c];
    *dlogit += g2[5] * P.opac * (1 - P.opac);
    (void)opacity_logit;
    const double x = P.pc[0], y = P.pc[1], z = P.pc[2];
    const double* V = cam.viewmat;
    T dpc[3] = {0, 0, 0};
    // 2D mean
    dpc[0] += g2[0] * cam.fx / z;
    dpc[1] += g2[1] * cam.fy / z;
    dpc[2] += -g2[0] * cam.fx * x / (z * z) - g2[1] * cam.fy * y / (z * z);
    // depth output
    dpc[2] += g2[9];
    // conic = inverse(Sigma'): dL/dSigma' = -M^-1 Gm M^-1 with Gm the matrix gradient of the conic
    const double M[2][2] = {{P.conic[0], P.conic[1]}, {P.conic[1], P.conic[2]}};
    const T Gm[2][2] = {{g2[2], 0.5 * g2[3]}, {0.5 * g2[3], g2[4]}};
    T GS[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            T acc = 0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) acc += M[i][k] * Gm[k][l] * M[l][j];
            GS[i][j] = -acc;
        }
    // Sigma' = T2 S3 T2^T + lowpass I;  dL/dS3 = T2^T GS T2;  dL/dT2 = 2 GS T2 S3
    T dS3[3][3], dT2[2][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T acc = 0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) acc += P.T2[k][i] * GS[k][l] * P.T2[l][j];
            dS3[i][j] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            T acc = 0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 3; ++l) acc += GS[i][k] * P.T2[k][l] * P.S3[l][j];
            dT2[i][j] = 2 * acc;
        }
    // T2 = J W  ->  dL/dJ = dT2 W^T
    T dJ[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            T acc = 0;
            for (int k = 0; k < 3; ++k) acc += dT2[i][k] * V[4 * j + k];
            dJ[i][j] = acc;
        }
    // J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]]
    dpc[0] += dJ[0][2] * (-cam.fx / (z * z));
    dpc[1] += dJ[1][2] * (-cam.fy / (z * z));
    dpc[2] += dJ[0][0] * (-cam.fx / (z * z)) + dJ[0][2] * (2 * cam.fx * x / (z * z * z)) +
              dJ[1][1] * (-cam.fy / (z * z)) + dJ[1][2] * (2 * cam.fy * y / (z * z * z));
    // p_c = Rv mean + t
    for (int j = 0; j < 3; ++j) dmean[j] += V[j] * dpc[0] + V[4 + j] * dpc[1] + V[8 + j] * dpc[2];
    // S3 = M M^T with M = Rq diag(s):  dL/dM = (dS3 + dS3^T) M
    double Mm[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mm[i][j] = P.Rq[i][j] * P.s[j];
    T dM[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T acc = 0;
            for (int k = 0; k < 3; ++k) acc += (dS3[i][k] + dS3[k][i]) * Mm[k][j];
            dM[i][j] = acc;
        }
    T dR[3][3];
    for (int j = 0; j < 3; ++j) {
        T ds = 0;
        for (int i = 0; i < 3; ++i) {
            ds += dM[i][j] * P.Rq[i][j];
            dR[i][j] = dM[i][j] * P.s[j];
        }
        dlog_scale[j] += ds * P.s[j];
    }
    // R(q) for the normalised quaternion (w,x,y,z)
    const double w = P.qn[0], qx = P.qn[1], qy = P.qn[2], qz = P.qn[3];
    T dqn[4];
    dqn[0] = 2 * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] - qy * dR[2][0] + qx * dR[2][1]);
    dqn[1] = 2 * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2 * qx * dR[1][1] - w * dR[1][2] +
                  qz * dR[2][0] + w * dR[2][1] - 2 * qx * dR[2][2]);
    dqn[2] = 2 * (-2 * qy * dR[0][0] + qx * dR[0][1] + w * dR[0][2] + qx * dR[1][0] + qz * dR[1][2] -
                  w * dR[2][0] + qz * dR[2][1] - 2 * qy * dR[2][2]);
    dqn[3] = 2 * (-2 * qz * dR[0][0] - w * dR[0][1] + qx * dR[0][2] + w * dR[1][0] - 2 * qz * dR[1][1] +
                  qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
    // normalisation q / |q|
    T dot = 0;
    for (int k = 0; k < 4; ++k) dot += dqn[k] * P.qn[k];
    for (int k = 0; k < 4; ++k) dquat[k] += (dqn[k] - P.qn[k] * dot) / P.qnorm;
}

Inputs make_inputs(int64_t n, const double* means, const double* log_scales, const double* quats,
                   const double* opacity_logit, const double* rgb, const int32_t* obj_id, const uint8_t* flags) {
    return Inputs{n, means, log_scales, quats, opacity_logit, rgb, obj_id, flags};
}

// Per tile, the Gaussians whose tile membership is uncertain there: tiles in the union of
// a Gaussian's perturbed rects but not in their intersection.
std::vector<std::vector<int64_t>> rect_ambiguity(const std::vector<Proj>& pr, int ntx, int nty) {
    std::vector<std::vector<int64_t>> amb((size_t)ntx * nty);
    for (int64_t g = 0; g < (int64_t)pr.size(); ++g) {
        const Proj& P = pr[g];
        if (!P.ambiguous) continue;
        for (int ty = P.urect[1]; ty < P.urect[3] && ty < nty; ++ty)
            for (int tx = P.urect[0]; tx < P.urect[2] && tx < ntx; ++tx)
                if (!covers(P.irect, tx, ty)) amb[(size_t)ty * ntx + tx].push_back(g);
    }
    return amb;
}

// A pixel's result depends on an uncertain membership only if that Gaussian would reach
// alpha_min there; records those Gaussians and flags the pixel.
void rect_check(const OSettings& st, const std::vector<Proj>& pr, const std::vector<int64_t>& cand, int px,
                int py, PixelResult& R) {
    for (int64_t g : cand) {
        const Proj& P = pr[g];
        if (P.opac <= 0 || P.conic[0] == 0) {
            if (!P.visible) { R.amb |= AMB_RECT; R.amb_rect.push_back(g); }
            continue;
        }
        const double dx = px - P.xy[0], dy = py - P.xy[1];
        const double power = -0.5 * (P.conic[0] * dx * dx + P.conic[2] * dy * dy) - P.conic[1] * dx * dy;
        const double alpha = std::min(st.alpha_clamp, P.opac * std::exp(power));
        if (alpha >= st.alpha_min * (1 - st.amb_rel)) {
            R.amb |= AMB_RECT;
            R.amb_rect.push_back(g);
        }
    }
}

}  // namespace

// ====================================================================== C entry points

extern "C" {

// Per-Gaussian projection.  Outputs (each may be NULL): xy[n*2], conic[n*3] (Sigma'^-1),
// z[n], opac[n], radius[n], rect[n*4] (tx0,ty0,tx1,ty1 exclusive), visible[n], ambiguous[n].
int oracle_preprocess(const OSettings* st, const OCamera* cam, int64_t n, const double* means,
                      const double* log_scales, const double* quats, const double* opacity_logit,
                      double* xy, double* conic, double* z, double* opac, int32_t* radius, int32_t* rect,
                      uint8_t* visible, uint8_t* ambiguous) {
    for (int64_t i = 0; i < n; ++i) {
        Proj P = project_gaussian(*st, *cam, means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity_logit[i]);
        if (xy) { xy[2 * i] = P.xy[0]; xy[2 * i + 1] = P.xy[1]; }
        if (conic) for (int k = 0; k < 3; ++k) conic[3 * i + k] = P.conic[k];
        if (z) z[i] = P.pc[2];
        if (opac) opac[i] = P.opac;
        if (radius) radius[i] = P.radius;
        if (rect) for (int k = 0; k < 4; ++k) rect[4 * i + k] = P.visible ? P.rect[k] : 0;
        if (visible) visible[i] = P.visible;
        if (ambiguous) ambiguous[i] = P.ambiguous;
    }
    return 0;
}

// Full render.  mode 0: per-tile sorted lists; mode 1: per-pixel brute force over all
// Gaussians in (depth key, index) order.  Targets may be NULL (then no loss / pixel gradients).
// Outputs (each may be NULL): rgb[H*W*3], depth, alpha, ins, id_map, T_final, n_contrib,
// amb[H*W] (flag bits), id_margin[H*W], loss[4] (rgb, depth, ins, total),
// dl[H*W*6] (dC r,g,b, dD, dA, dins), update_mask, mask_amb, last[H*W] (index of the last
// blended Gaussian, -1 if none).  Only pixel rows y0 <= v < y1 are rendered (y1 <= 0:
// every row); other rows' outputs are left as they are and add nothing to the losses.
int oracle_render(const OSettings* st, const OCamera* cam, int64_t n, const double* means,
                  const double* log_scales, const double* quats, const double* opacity_logit,
                  const double* rgb, const int32_t* obj_id, const uint8_t* flags,
                  const double* t_rgb, const double* t_depth, const int32_t* t_gt, int mode,
                  double* o_rgb, double* o_depth, double* o_alpha, double* o_ins, int32_t* o_id,
                  double* o_T, int64_t* o_ncontrib, uint8_t* o_amb, double* o_margin, double* o_loss,
                  double* o_dl, uint8_t* o_mask, uint8_t* o_mask_amb, int64_t* o_last, int32_t y0, int32_t y1) {
    const Inputs in = make_inputs(n, means, log_scales, quats, opacity_logit, rgb, obj_id, flags);
    const int W = cam->width, H = cam->height;
    if (W <= 0 || H <= 0 || st->tile_w <= 0 || st->tile_h <= 0) return 1;
    if (y1 <= 0 || y1 > H) y1 = H;
    if (y0 < 0) y0 = 0;
    const int ntx = (W + st->tile_w - 1) / st->tile_w, nty = (H + st->tile_h - 1) / st->tile_h;
    std::vector<Proj> pr = project_all(*st, *cam, in);
    const std::vector<std::vector<int64_t>> tile_amb = rect_ambiguity(pr, ntx, nty);
    std::vector<int64_t> all;
    if (mode == 1) {
        for (int64_t i = 0; i < n; ++i) all.push_back(i);
        std::stable_sort(all.begin(), all.end(), [&](int64_t a, int64_t b) { return depth_less(pr, a, b); });
    }
    double loss[3] = {0, 0, 0};
    const double inv_hw = 1.0 / ((double)W * H);
    for (int ty = y0 / st->tile_h; ty < nty && ty * st->tile_h < y1; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            std::vector<int64_t> L;
            if (mode == 0) L = tile_list(pr, tx, ty);
            for (int py = std::max(y0, ty * st->tile_h); py < std::min(y1, (ty + 1) * st->tile_h); ++py)
                for (int px = tx * st->tile_w; px < std::min(W, (tx + 1) * st->tile_w); ++px) {
                    const size_t p = (size_t)py * W + px;
                    const int32_t gt = t_gt ? t_gt[p] : -1;
                    std::vector<int64_t> Lp;
                    if (mode == 1) {
                        for (int64_t i : all)
                            if (pr[i].visible && covers(pr[i].rect, px / st->tile_w, py / st->tile_h)) Lp.push_back(i);
                    }
                    PixelResult R = blend_pixel(*st, in, pr, mode == 0 ? L : Lp, px, py, gt, false);
                    rect_check(*st, pr, tile_amb[(size_t)ty * ntx + tx], px, py, R);
                    PixelGrad pg{{0, 0, 0}, 0, 0, 0};
                    if (t_gt) pixel_loss(*st, R, t_rgb + 3 * p, t_depth ? t_depth[p] : 0.0, gt, inv_hw, loss, pg, R.amb);
                    if (o_rgb) for (int c = 0; c < 3; ++c) o_rgb[3 * p + c] = R.C[c];
                    if (o_depth) o_depth[p] = R.D;
                    if (o_alpha) o_alpha[p] = R.A;
                    if (o_ins) o_ins[p] = R.ins;
                    if (o_id) o_id[p] = R.id;
                    if (o_T) o_T[p] = R.T;
                    if (o_ncontrib) o_ncontrib[p] = R.n_contrib;
                    if (o_last) o_last[p] = R.last_g;
                    if (o_amb) o_amb[p] = R.amb;
                    if (o_margin) o_margin[p] = R.id_margin;
                    if (o_dl) {
                        double* d = o_dl + 6 * p;
                        d[0] = pg.dC[0]; d[1] = pg.dC[1]; d[2] = pg.dC[2]; d[3] = pg.dD; d[4] = pg.dA; d[5] = pg.dins;
                    }
                    if (o_mask && t_gt) {
                        // Eq. 11 update masks; o_mask_amb flags values within 1e-4 of a threshold
                        uint8_t m = 0, am = 0;
                        if (gt >= 0) {
                            const double td = t_depth ? t_depth[p] : 0.0;
                            const double ed = std::fabs(R.D - td);
                            const bool geo = R.ins < st->theta_alpha || (td > 0 && ed > st->theta_d);
                            double ec = 0;
                            for (int c = 0; c < 3; ++c) ec = std::max(ec, std::fabs(R.C[c] - t_rgb[3 * p + c]));
                            m = (uint8_t)((geo ? 1 : 0) | (ec > st->theta_c ? 2 : 0));
                            if (std::fabs(R.ins - st->theta_alpha) < 1e-4 || (td > 0 && std::fabs(ed - st->theta_d) < 1e-4))
                                am |= 1;
                            if (std::fabs(ec - st->theta_c) < 1e-4) am |= 2;
                        }
                        o_mask[p] = m;
                        if (o_mask_amb) o_mask_amb[p] = am;
                    }
                }
        }
    if (o_loss) {
        o_loss[0] = loss[0]; o_loss[1] = loss[1]; o_loss[2] = loss[2];
        o_loss[3] = loss[0] + loss[1] + st->lambda_ins * loss[2];
    }
    return 0;
}

// Render at a list of pixels only (for parity at full size).  px[npix*2] = (u, v).
// Outputs per sampled pixel: rgb[npix*3], depth, alpha, ins, id, T, n_contrib, amb, margin.
int oracle_render_pixels(const OSettings* st, const OCamera* cam, int64_t n, const double* means,
                         const double* log_scales, const double* quats, const double* opacity_logit,
                         const double* rgb, const int32_t* obj_id, const uint8_t* flags,
                         const int32_t* t_gt, int64_t npix, const int32_t* pxy, double* o_rgb,
                         double* o_depth, double* o_alpha, double* o_ins, int32_t* o_id, double* o_T,
                         int64_t* o_ncontrib, uint8_t* o_amb, double* o_margin) {
    const Inputs in = make_inputs(n, means, log_scales, quats, opacity_logit, rgb, obj_id, flags);
    const int W = cam->width, H = cam->height;
    const int ntx = (W + st->tile_w - 1) / st->tile_w, nty = (H + st->tile_h - 1) / st->tile_h;
    std::vector<Proj> pr = project_all(*st, *cam, in);
    const std::vector<std::vector<int64_t>> tile_amb = rect_ambiguity(pr, ntx, nty);
    for (int64_t k = 0; k < npix; ++k) {
        const int px = pxy[2 * k], py = pxy[2 * k + 1];
        if (px < 0 || px >= W || py < 0 || py >= H) return 1;
        const int tx = px / st->tile_w, ty = py / st->tile_h;
        std::vector<int64_t> L = tile_list(pr, tx, ty);
        const int32_t gt = t_gt ? t_gt[(size_t)py * W + px] : -1;
        PixelResult R = blend_pixel(*st, in, pr, L, px, py, gt, false);
        rect_check(*st, pr, tile_amb[(size_t)ty * ntx + tx], px, py, R);
        if (o_rgb) for (int c = 0; c < 3; ++c) o_rgb[3 * k + c] = R.C[c];
        if (o_depth) o_depth[k] = R.D;
        if (o_alpha) o_alpha[k] = R.A;
        if (o_ins) o_ins[k] = R.ins;
        if (o_id) o_id[k] = R.id;
        if (o_T) o_T[k] = R.T;
        if (o_ncontrib) o_ncontrib[k] = R.n_contrib;
        if (o_amb) o_amb[k] = R.amb;
        if (o_margin) o_margin[k] = R.id_margin;
    }
    return 0;
}

// The outcomes a correct single-precision render may produce at selected pixels.  A pixel
// whose result hangs on decisions within rounding distance of their thresholds (alpha_min
// skip, clamp, transmittance stop; tile membership of a Gaussian whose rect edge is
// uncertain) is re-rendered with each subset of those decisions taken the other way: every
// subset when there are at most `full_items` of them, else the subsets of one or two.
// Alternative 0 is the render as it stands.  px[npix*2] = (u, v).  Outputs per (pixel k,
// alternative a), index k*max_alt + a: vals[*7] = (r, g, b, depth, alpha, ins, T_final),
// n_contrib, id, id_margin, last (index of the last blended Gaussian, -1 if none);
// count[k] = alternatives written (at most max_alt).
int oracle_render_alternatives(const OSettings* st, const OCamera* cam, int64_t n, const double* means,
                               const double* log_scales, const double* quats, const double* opacity_logit,
                               const double* rgb, const int32_t* obj_id, const uint8_t* flags,
                               const int32_t* t_gt, int64_t npix, const int32_t* pxy, int32_t max_alt,
                               int32_t full_items, int32_t* o_count, double* o_vals, int64_t* o_ncontrib,
                               int32_t* o_id, double* o_margin, int64_t* o_last) {
    const Inputs in = make_inputs(n, means, log_scales, quats, opacity_logit, rgb, obj_id, flags);
    const int W = cam->width, H = cam->height;
    if (W <= 0 || H <= 0 || max_alt < 1) return 1;
    const int ntx = (W + st->tile_w - 1) / st->tile_w, nty = (H + st->tile_h - 1) / st->tile_h;
    std::vector<Proj> pr = project_all(*st, *cam, in);
    const std::vector<std::vector<int64_t>> tile_amb = rect_ambiguity(pr, ntx, nty);
    std::map<int64_t, std::vector<int64_t>> lists;  // tile lists of the tiles asked for
    for (int64_t k = 0; k < npix; ++k) {
        const int px = pxy[2 * k], py = pxy[2 * k + 1];
        if (px < 0 || px >= W || py < 0 || py >= H) return 1;
        const int tx = px / st->tile_w, ty = py / st->tile_h;
        const int64_t tile = (int64_t)ty * ntx + tx;
        auto it = lists.find(tile);
        if (it == lists.end()) it = lists.emplace(tile, tile_list(pr, tx, ty)).first;
        const std::vector<int64_t>& L = it->second;
        const int32_t gt = t_gt ? t_gt[(size_t)py * W + px] : -1;
        PixelResult R = blend_pixel(*st, in, pr, L, px, py, gt, false);
        rect_check(*st, pr, tile_amb[(size_t)tile], px, py, R);
        // the uncertain items: decision flips, then membership toggles (each Gaussian once)
        std::vector<Flip> fl(R.near.size());
        for (size_t i = 0; i < R.near.size(); ++i) fl[i] = Flip{R.near[i].first, R.near[i].second};
        std::vector<int64_t> tog = R.amb_rect;
        std::sort(tog.begin(), tog.end());
        tog.erase(std::unique(tog.begin(), tog.end()), tog.end());
        const int items = (int)(fl.size() + tog.size());
        std::vector<std::vector<int>> subsets{{}};
        if (items <= full_items) {
            for (int mask = 1; mask < (1 << items); ++mask) {
                std::vector<int> sub;
                for (int i = 0; i < items; ++i)
                    if (mask >> i & 1) sub.push_back(i);
                subsets.push_back(sub);
            }
        } else {
            for (int i = 0; i < items; ++i) subsets.push_back({i});
            for (int i = 0; i < items; ++i)
                for (int j = i + 1; j < items; ++j) subsets.push_back({i, j});
        }
        int a = 0;
        for (const std::vector<int>& sub : subsets) {
            if (a >= max_alt) break;
            std::vector<Flip> f;
            std::vector<int64_t> L1 = L;
            bool changed_list = false;
            for (int i : sub) {
                if (i < (int)fl.size()) { f.push_back(fl[(size_t)i]); continue; }
                const int64_t ga = tog[(size_t)i - fl.size()];
                auto pos = std::find(L1.begin(), L1.end(), ga);
                if (pos != L1.end()) L1.erase(pos);
                else { L1.push_back(ga); changed_list = true; }
            }
            if (changed_list)
                std::stable_sort(L1.begin(), L1.end(), [&](int64_t x, int64_t y) { return depth_less(pr, x, y); });
            const PixelResult R1 = sub.empty() ? R : blend_pixel(*st, in, pr, L1, px, py, gt, false, f);
            const size_t o = (size_t)k * max_alt + a;
            double* v = o_vals + 7 * o;
            v[0] = R1.C[0]; v[1] = R1.C[1]; v[2] = R1.C[2]; v[3] = R1.D; v[4] = R1.A; v[5] = R1.ins; v[6] = R1.T;
            o_ncontrib[o] = R1.n_contrib;
            o_last[o] = R1.last_g;
            o_id[o] = R1.id;
            o_margin[o] = R1.id_margin;
            ++a;
        }
        o_count[k] = a;
    }
    return 0;
}

// Backward of the render.  Pixel gradients: if dl (H*W*6 = dC rgb, dD, dA, dins) is NULL the
// fused L1 losses against the targets are differentiated.  Outputs (accumulated +=, each may be
// NULL): g2[n*10] (dxy, dconic a b c, dopac, drgb, dz), and parameter gradients.
// g_amb[n]: bit0 the Gaussian's alpha decision is near a threshold somewhere, bit2 its tile
// membership is uncertain somewhere, bit3 it feeds a pixel at an L1 kink.  A pixel whose
// upstream gradient is zero (all six dl entries zero, or, for the fused losses, an
// unlabelled pixel) adds exactly zero to every gradient and every bound, so it is skipped
// and sets no flag.
// unc[n*14]: per parameter (means, log_scales, quats, logit, rgb) the summed absolute change
// of the gradient when each near-threshold decision or uncertain membership is taken the
// other way, pixel by pixel, plus a bound on single-precision rounding of the gradient's
// sum and of the projection adjoint's chain -- the amount by which a correct
// single-precision evaluation may differ from this one.
int oracle_render_backward(const OSettings* st, const OCamera* cam, int64_t n, const double* means,
                           const double* log_scales, const double* quats, const double* opacity_logit,
                           const double* rgb, const int32_t* obj_id, const uint8_t* flags,
                           const double* t_rgb, const double* t_depth, const int32_t* t_gt,
                           const double* dl, double* g2_out, double* d_means, double* d_log_scales,
                           double* d_quats, double* d_logit, double* d_rgb, uint8_t* g_amb, double* unc) {
    const Inputs in = make_inputs(n, means, log_scales, quats, opacity_logit, rgb, obj_id, flags);
    const int W = cam->width, H = cam->height;
    if (W <= 0 || H <= 0) return 1;
    const int ntx = (W + st->tile_w - 1) / st->tile_w, nty = (H + st->tile_h - 1) / st->tile_h;
    std::vector<Proj> pr = project_all(*st, *cam, in);
    const std::vector<std::vector<int64_t>> tile_amb = rect_ambiguity(pr, ntx, nty);
    std::vector<double> g2((size_t)n * G2, 0.0);
    // magnitudes of the per-pixel terms: plain, and weighted by the pixel's walk length
    std::vector<double> magA(unc ? (size_t)n * G2 : 0, 0.0), magS(unc ? (size_t)n * G2 : 0, 0.0);
    const double inv_hw = 1.0 / ((double)W * H);
    auto dense = [&](int64_t g) { return g2.data() + G2 * g; };
    using Sparse = std::map<int64_t, std::array<double, G2>>;
    auto sparse_acc = [](Sparse& m) {
        return [&m](int64_t g) {
            auto it = m.find(g);
            if (it == m.end()) it = m.emplace(g, std::array<double, G2>{}).first;
            return it->second.data();
        };
    };
    // unc[14 i ..] += |parameter-gradient change| of Gaussian i if FP32 took the other
    // side of a decision near its threshold at some pixel (means 3, log_scales 3, quats 4,
    // opacity logit 1, rgb 3).
    auto add_uncertainty = [&](const Sparse& m0, const Sparse& m1) {
        Sparse keys = m0;
        for (const auto& kv : m1) keys.emplace(kv.first, std::array<double, G2>{});
        for (const auto& kv : keys) {
            const int64_t g = kv.first;
            const Proj& P = pr[g];
            if (P.conic[0] == 0) continue;  // culled before projection: no gradient either way
            std::array<double, G2> d{};
            auto i0 = m0.find(g), i1 = m1.find(g);
            for (int k = 0; k < G2; ++k)
                d[k] = (i1 != m1.end() ? i1->second[k] : 0.0) - (i0 != m0.end() ? i0->second[k] : 0.0);
            double dm[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlg = 0, dc[3] = {0, 0, 0};
            preprocess_backward(*st, *cam, P, opacity_logit[g], d.data(), dm, ds, dq, &dlg, dc);
            double* u = unc + 14 * g;
            for (int k = 0; k < 3; ++k) u[k] += std::fabs(dm[k]);
            for (int k = 0; k < 3; ++k) u[3 + k] += std::fabs(ds[k]);
            for (int k = 0; k < 4; ++k) u[6 + k] += std::fabs(dq[k]);
            u[10] += std::fabs(dlg);
            for (int k = 0; k < 3; ++k) u[11 + k] += std::fabs(dc[k]);
        }
    };
    // upstream gradient of pixel p is zero (see above)
    auto inactive = [&](size_t p) {
        if (dl) {
            for (int k = 0; k < 6; ++k)
                if (dl[6 * p + k] != 0) return false;
            return true;
        }
        return !t_gt || t_gt[p] < 0;
    };
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            bool any = false;
            for (int py = ty * st->tile_h; py < std::min(H, (ty + 1) * st->tile_h) && !any; ++py)
                for (int px = tx * st->tile_w; px < std::min(W, (tx + 1) * st->tile_w) && !any; ++px)
                    any = !inactive((size_t)py * W + px);
            if (!any) continue;
            std::vector<int64_t> L = tile_list(pr, tx, ty);
            for (int py = ty * st->tile_h; py < std::min(H, (ty + 1) * st->tile_h); ++py)
                for (int px = tx * st->tile_w; px < std::min(W, (tx + 1) * st->tile_w); ++px) {
                    const size_t p = (size_t)py * W + px;
                    if (inactive(p)) continue;
                    const int32_t gt = t_gt ? t_gt[p] : -1;
                    PixelResult R = blend_pixel(*st, in, pr, L, px, py, gt, true);
                    rect_check(*st, pr, tile_amb[(size_t)ty * ntx + tx], px, py, R);
                    PixelGrad pg{{0, 0, 0}, 0, 0, 0};
                    if (dl) {
                        const double* d = dl + 6 * p;
                        pg = PixelGrad{{d[0], d[1], d[2]}, d[3], d[4], d[5]};
                    } else if (t_gt) {
                        double loss[3] = {0, 0, 0};
                        pixel_loss(*st, R, t_rgb + 3 * p, t_depth ? t_depth[p] : 0.0, gt, inv_hw, loss, pg, R.amb);
                    }
                    if (unc) {
                        // a single-precision walk of k contributors carries a relative error
                        // of about k unit roundoffs in T (forward product, backward quotients)
                        std::vector<double> tmp(G2 * R.contribs.size());
                        size_t slot = 0;
                        std::map<int64_t, double*> where;
                        pixel_backward(*st, in, pr, R, pg, gt, dense, [&](int64_t g) {
                            double* m = tmp.data() + G2 * slot++;
                            where[g] = m;
                            return m;
                        });
                        const double wk = (double)R.contribs.size() + 16.0;
                        for (const auto& kv : where)
                            for (int k = 0; k < G2; ++k) {
                                magA[G2 * kv.first + k] += kv.second[k];
                                magS[G2 * kv.first + k] += wk * kv.second[k];
                            }
                    } else {
                        pixel_backward(*st, in, pr, R, pg, gt, dense);
                    }
                    if (g_amb && (R.amb & AMB_KINK))
                        for (const Contrib& c : R.contribs) g_amb[c.g] |= AMB_KINK;
                    if (unc && (R.amb & (AMB_THRESH | AMB_RECT))) {
                        Sparse m0;
                        pixel_backward(*st, in, pr, R, pg, gt, sparse_acc(m0));
                        for (const auto& nk : R.near) {
                            // the same pixel with one near-threshold decision taken the other way
                            PixelResult R1 = blend_pixel(*st, in, pr, L, px, py, gt, true, {Flip{nk.first, nk.second}});
                            Sparse m1;
                            pixel_backward(*st, in, pr, R1, pg, gt, sparse_acc(m1));
                            add_uncertainty(m0, m1);
                            if (g_amb) g_amb[nk.first] |= AMB_THRESH;
                        }
                        std::vector<int64_t> cand = R.amb_rect;
                        std::sort(cand.begin(), cand.end());
                        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
                        for (int64_t ga : cand) {
                            // the same pixel with ga's tile membership toggled
                            std::vector<int64_t> L1;
                            bool had = false;
                            for (int64_t g : L) {
                                if (g == ga) { had = true; continue; }
                                L1.push_back(g);
                            }
                            if (!had) {
                                L1.push_back(ga);
                                std::stable_sort(L1.begin(), L1.end(),
                                                 [&](int64_t a, int64_t b) { return depth_less(pr, a, b); });
                            }
                            PixelResult R1 = blend_pixel(*st, in, pr, L1, px, py, gt, true);
                            Sparse m1;
                            pixel_backward(*st, in, pr, R1, pg, gt, sparse_acc(m1));
                            add_uncertainty(m0, m1);
                            if (g_amb) g_amb[ga] |= AMB_RECT;
                        }
                    }
                }
        }
    // Single-precision rounding bound of every Gaussian's gradient: its per-pixel terms
    // carry ~(walk length + 16) unit roundoffs each, and the GPU adds them through about
    // sqrt(8 x tiles covered) levels of partial sums; chained to the parameters through
    // the element-wise magnitude of the projection Jacobian, times a safety factor of 4.
    const double u = std::ldexp(1.0, -24);
    for (int64_t i = 0; unc && i < n; ++i) {
        if (!pr[i].visible) continue;
        const int nt = (pr[i].rect[2] - pr[i].rect[0]) * (pr[i].rect[3] - pr[i].rect[1]);
        double bound2d[G2];
        for (int k = 0; k < G2; ++k)
            bound2d[k] = 4 * u * (magS[G2 * i + k] + std::sqrt(8.0 * nt) * magA[G2 * i + k]);
        for (int k = 0; k < G2; ++k) {
            if (bound2d[k] == 0) continue;
            double e[G2] = {0};
            e[k] = 1;
            double dm[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlg = 0, dc[3] = {0, 0, 0};
            preprocess_backward(*st, *cam, pr[i], opacity_logit[i], e, dm, ds, dq, &dlg, dc);
            double* uu = unc + 14 * i;
            for (int j = 0; j < 3; ++j) uu[j] += std::fabs(dm[j]) * bound2d[k];
            for (int j = 0; j < 3; ++j) uu[3 + j] += std::fabs(ds[j]) * bound2d[k];
            for (int j = 0; j < 4; ++j) uu[6 + j] += std::fabs(dq[j]) * bound2d[k];
            uu[10] += std::fabs(dlg) * bound2d[k];
            for (int j = 0; j < 3; ++j) uu[11 + j] += std::fabs(dc[j]) * bound2d[k];
        }
    }
    // Single-precision evaluation of the projection adjoint itself: to first order its
    // rounding error is at most a few tens of unit roundoffs (the chain is ~40 operations
    // deep, its coefficients -- conic, Jacobian, rotation, scales -- are themselves rounded)
    // times the magnitude sum of every term it combines, the same chain evaluated on
    // magnitudes; 64u of that.  It matters only where the chain cancels, e.g. a Gaussian
    // just beyond the near plane whose footprint covers the image.
    for (int64_t i = 0; unc && i < n; ++i) {
        if (!pr[i].visible) continue;
        Mag m2[G2], mm[3], ms[3], mq[4], ml, mc[3];
        for (int k = 0; k < G2; ++k) m2[k] = Mag(g2[G2 * i + k]);
        preprocess_backward<Mag>(*st, *cam, pr[i], opacity_logit[i], m2, mm, ms, mq, &ml, mc);
        const double cu = 64 * u;
        double* uu = unc + 14 * i;
        for (int j = 0; j < 3; ++j) uu[j] += cu * mm[j].v;
        for (int j = 0; j < 3; ++j) uu[3 + j] += cu * ms[j].v;
        for (int j = 0; j < 4; ++j) uu[6 + j] += cu * mq[j].v;
        uu[10] += cu * ml.v;
        for (int j = 0; j < 3; ++j) uu[11 + j] += cu * mc[j].v;
    }
    for (int64_t i = 0; i < n; ++i) {
        const double* r = g2.data() + G2 * i;
        if (g2_out) for (int k = 0; k < G2; ++k) g2_out[G2 * i + k] += r[k];
        if (!pr[i].visible) continue;
        double dm[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlg = 0, dc[3] = {0, 0, 0};
        preprocess_backward(*st, *cam, pr[i], opacity_logit[i], r, dm, ds, dq, &dlg, dc);
        if (d_means) for (int k = 0; k < 3; ++k) d_means[3 * i + k] += dm[k];
        if (d_log_scales) for (int k = 0; k < 3; ++k) d_log_scales[3 * i + k] += ds[k];
        if (d_quats) for (int k = 0; k < 4; ++k) d_quats[4 * i + k] += dq[k];
        if (d_logit) d_logit[i] += dlg;
        if (d_rgb) for (int k = 0; k < 3; ++k) d_rgb[3 * i + k] += dc[k];
    }
    return 0;
}

// Tile lists from given single-precision projections: Gaussians i with visible[i] and
// rect covering the tile, ordered by (tile row-major, zbits[i] as unsigned, i).
// ranges[T*2] = [start, end); list[M] must hold sum of rect areas.  Returns M.
int64_t oracle_bin_tiles(int64_t n, const int32_t* rect, const uint32_t* zbits, const uint8_t* visible,
                         int ntx, int nty, int64_t* ranges, int64_t* list) {
    int64_t m = 0;
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            const int64_t start = m;
            std::vector<int64_t> L;
            for (int64_t i = 0; i < n; ++i)
                if (visible[i] && tx >= rect[4 * i] && tx < rect[4 * i + 2] && ty >= rect[4 * i + 1] &&
                    ty < rect[4 * i + 3])
                    L.push_back(i);
            std::stable_sort(L.begin(), L.end(), [&](int64_t a, int64_t b) {
                if (zbits[a] != zbits[b]) return zbits[a] < zbits[b];
                return a < b;
            });
            for (int64_t i : L) list[m++] = i;
            ranges[2 * ((int64_t)ty * ntx + tx)] = start;
            ranges[2 * ((int64_t)ty * ntx + tx) + 1] = m;
        }
    return m;
}

}  // extern "C"

// ====================================================================== dual quadrics

namespace {

const int ND = 9;  // derivative directions = quadric parameters

struct Dual {
    double v;
    double d[ND];
    Dual() : v(0) { std::memset(d, 0, sizeof d); }
    Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }
};
Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r; }
Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
Dual sqrt(const Dual& a) { const double s = std::sqrt(a.v); Dual r(s); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / (2 * s); return r; }
Dual sin(const Dual& a) { Dual r(std::sin(a.v)); const double c = std::cos(a.v); for (int i = 0; i < ND; ++i) r.d[i] = c * a.d[i]; return r; }
Dual cos(const Dual& a) { Dual r(std::cos(a.v)); const double s = -std::sin(a.v); for (int i = 0; i < ND; ++i) r.d[i] = s * a.d[i]; return r; }
Dual exp(const Dual& a) { const double e = std::exp(a.v); Dual r(e); for (int i = 0; i < ND; ++i) r.d[i] = e * a.d[i]; return r; }
double val(const Dual& a) { return a.v; }
double val(double a) { return a; }
using std::sqrt; using std::sin; using std::cos; using std::exp;

// Rodrigues: R = I + A [r]x + B [r]x^2, A = sin(t)/t, B = (1 - cos t)/t^2, t = |r|.
template <class T>
void rotvec_to_rot(const T r[3], T R[3][3]) {
    const T t2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    T A, B;
    if (val(t2) < 1e-8) {
        A = T(1.0) - t2 / T(6.0);
        B = T(0.5) - t2 / T(24.0);
    } else {
        const T t = sqrt(t2);
        A = sin(t) / t;
        B = (T(1.0) - cos(t)) / t2;
    }
    const T K[3][3] = {{T(0.0), -r[2], r[1]}, {r[2], T(0.0), -r[0]}, {-r[1], r[0], T(0.0)}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T kk = T(0.0);
            for (int k = 0; k < 3; ++k) kk = kk + K[i][k] * K[k][j];
            R[i][j] = T(i == j ? 1.0 : 0.0) + A * K[i][j] + B * kk;
        }
}

// Eq. 1-3 reading: Q* = Z diag(a^2, b^2, c^2, -1) Z^T with Z = [R t; 0 1].
template <class T>
void quadric_from_params(const T p[9], T Q[4][4]) {
    T R[3][3];
    const T r[3] = {p[6], p[7], p[8]};
    rotvec_to_rot(r, R);
    T Z[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Z[i][j] = T(0.0);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Z[i][j] = R[i][j];
        Z[i][3] = p[i];
    }
    Z[3][3] = T(1.0);
    const T D[4] = {exp(T(2.0) * p[3]), exp(T(2.0) * p[4]), exp(T(2.0) * p[5]), T(-1.0)};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            T acc = T(0.0);
            for (int k = 0; k < 4; ++k) acc = acc + Z[i][k] * D[k] * Z[j][k];
            Q[i][j] = acc;
        }
}

// Eq. 4 reading: C* = P Q* P^T.
template <class T>
void project_quadric(const T Q[4][4], const double P[12], T C[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T acc = T(0.0);
            for (int k = 0; k < 4; ++k)
                for (int l = 0; l < 4; ++l) acc = acc + T(P[4 * i + k]) * Q[k][l] * T(P[4 * j + l]);
            C[i][j] = acc;
        }
}

// BBox(C*): vertical line (1,0,-u) tangent iff c11 - 2u c13 + u^2 c33 = 0; likewise for v.
template <class T>
bool conic_bbox(const T C[3][3], double centre_depth, T box[4]) {
    const T du = C[0][2] * C[0][2] - C[0][0] * C[2][2];
    const T dv = C[1][2] * C[1][2] - C[1][1] * C[2][2];
    const bool valid = val(C[2][2]) < 0 && centre_depth > 0 && val(du) > 0 && val(dv) > 0;
    if (!valid) { for (int k = 0; k < 4; ++k) box[k] = T(0.0); return false; }
    const T su = sqrt(du), sv = sqrt(dv);
    const T u1 = (C[0][2] + su) / C[2][2], u2 = (C[0][2] - su) / C[2][2];
    const T v1 = (C[1][2] + sv) / C[2][2], v2 = (C[1][2] - sv) / C[2][2];
    box[0] = val(u1) < val(u2) ? u1 : u2;
    box[2] = val(u1) < val(u2) ? u2 : u1;
    box[1] = val(v1) < val(v2) ? v1 : v2;
    box[3] = val(v1) < val(v2) ? v2 : v1;
    return true;
}

// Axis-aligned IoU; the predicted box is not clipped to the image.
template <class T>
T box_iou(const T b[4], const double o[4]) {
    const T ix0 = val(b[0]) > o[0] ? b[0] : T(o[0]);
    const T iy0 = val(b[1]) > o[1] ? b[1] : T(o[1]);
    const T ix1 = val(b[2]) < o[2] ? b[2] : T(o[2]);
    const T iy1 = val(b[3]) < o[3] ? b[3] : T(o[3]);
    T iw = ix1 - ix0, ih = iy1 - iy0;
    if (val(iw) <= 0) iw = T(0.0);
    if (val(ih) <= 0) ih = T(0.0);
    const T inter = iw * ih;
    const T ap = (b[2] - b[0]) * (b[3] - b[1]);
    const T ao = T((o[2] - o[0]) * (o[3] - o[1]));
    return inter / (ap + ao - inter);
}

double centre_depth(const double p[9], const double P[12]) {
    return P[8] * p[0] + P[9] * p[1] + P[10] * p[2] + P[11];
}

}  // namespace

extern "C" {

// Per (quadric, view) pair in CSR order: pairs q_ptr[q] .. q_ptr[q+1]-1 belong to quadric q
// and use view pair_v[k].  Outputs: conic[npairs*6] (c11 c12 c13 c22 c23 c33), bbox[npairs*4],
// valid[npairs].  Each may be NULL.
int oracle_quadric_project(int nq, const double* params, int nv, const double* P, const int32_t* q_ptr,
                           const int32_t* pair_v, double* conic, double* bbox, uint8_t* valid) {
    for (int q = 0; q < nq; ++q) {
        double Q[4][4];
        quadric_from_params(params + 9 * q, Q);
        for (int k = q_ptr[q]; k < q_ptr[q + 1]; ++k) {
            const int v = pair_v[k];
            if (v < 0 || v >= nv) return 1;
            double C[3][3], box[4];
            project_quadric(Q, P + 12 * v, C);
            const bool ok = conic_bbox(C, centre_depth(params + 9 * q, P + 12 * v), box);
            if (conic) {
                double* c = conic + 6 * k;
                c[0] = C[0][0]; c[1] = C[0][1]; c[2] = C[0][2]; c[3] = C[1][1]; c[4] = C[1][2]; c[5] = C[2][2];
            }
            if (bbox) for (int j = 0; j < 4; ++j) bbox[4 * k + j] = box[j];
            if (valid) valid[k] = ok;
        }
    }
    return 0;
}

// Eq. 12 reading: loss[q] = sum over valid pairs of q of (1 - IoU); dparams[q*9] its gradient
// (overwritten).  Gradient by forward-mode dual numbers through the same forward.
int oracle_quadric_bbox_loss(int nq, const double* params, int nv, const double* P, const int32_t* q_ptr,
                             const int32_t* pair_v, const double* obs, double* loss, double* dparams) {
    for (int q = 0; q < nq; ++q) {
        Dual p[9];
        for (int i = 0; i < 9; ++i) { p[i] = Dual(params[9 * q + i]); p[i].d[i] = 1.0; }
        Dual Q[4][4];
        quadric_from_params(p, Q);
        Dual L(0.0);
        for (int k = q_ptr[q]; k < q_ptr[q + 1]; ++k) {
            const int v = pair_v[k];
            if (v < 0 || v >= nv) return 1;
            Dual C[3][3], box[4];
            project_quadric(Q, P + 12 * v, C);
            if (!conic_bbox(C, centre_depth(params + 9 * q, P + 12 * v), box)) continue;
            L = L + (Dual(1.0) - box_iou(box, obs + 4 * k));
        }
        if (loss) loss[q] = L.v;
        if (dparams) for (int i = 0; i < 9; ++i) dparams[9 * q + i] = L.d[i];
    }
    return 0;
}

// 4x4 dual quadric of each parameter vector (row-major), for the decomposition pins.
int oracle_quadric_matrix(int nq, const double* params, double* Q16) {
    for (int q = 0; q < nq; ++q) {
        double Q[4][4];
        quadric_from_params(params + 9 * q, Q);
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) Q16[16 * q + 4 * i + j] = Q[i][j];
    }
    return 0;
}

}  // extern "C"

// ====================================================================== plain multi-view fit

namespace {

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major, overwritten);
// eigenvalues on the diagonal of A, eigenvectors in the columns of V.
void jacobi_eigen(int n, double* A, double* V) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
                const double c = 1 / std::sqrt(t * t + 1), sn = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // V <- V J
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
}

// Rotation matrix -> rotation vector (axis times angle in [0, pi]).
void rot_to_rotvec(const double R[3][3], double r[3]) {
    const double w[3] = {R[2][1] - R[1][2], R[0][2] - R[2][0], R[1][0] - R[0][1]};
    const double ct = std::max(-1.0, std::min(1.0, 0.5 * (R[0][0] + R[1][1] + R[2][2] - 1)));
    const double th = std::acos(ct);
    const double sw = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (th < 1e-8) {
        for (int k = 0; k < 3; ++k) r[k] = 0.5 * w[k];
        return;
    }
    if (M_PI - th < 1e-4 || sw < 1e-12) {
        // near pi the skew part vanishes: (R + R^T)/2 = cos(th) I + (1 - cos(th)) a a^T
        double S[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] = (0.5 * (R[i][j] + R[j][i]) - (i == j ? ct : 0.0)) / (1 - ct);
        int k = 0;
        for (int i = 1; i < 3; ++i)
            if (S[i][i] > S[k][k]) k = i;
        const double d = std::sqrt(std::max(S[k][k], 1e-300));
        double ax[3] = {S[0][k] / d, S[1][k] / d, S[2][k] / d};
        if (ax[0] * w[0] + ax[1] * w[1] + ax[2] * w[2] < 0)
            for (int i = 0; i < 3; ++i) ax[i] = -ax[i];
        for (int i = 0; i < 3; ++i) r[i] = th * ax[i];
        return;
    }
    for (int k = 0; k < 3; ++k) r[k] = th / (2 * std::sin(th)) * w[k];
}

// Plain initialisation (Eq. 1): every bbox edge line l back-projects to a plane pi = P^T l
// tangent to the quadric, pi^T Q* pi = 0, linear in Q*'s 10 entries.  Reading: planes in a
// world frame centred on the views' camera centres and scaled to unit mean distance,
// each plane scaled to unit norm; the null vector is the eigenvector of A^T A with the
// smallest eigenvalue; Q* scaled to Q*44 = -1; t = -Q*[0:3,3]; R diag(a^2,b^2,c^2) R^T =
// Q*[0:3,0:3] + t t^T with eigenvalues sorted descending, clamped to >= 1e-6 m^2, det R = +1.
bool quadric_init(int nview, const double* const* Pv, const double* const* obs, double params[9],
                  double Qout[16]) {
    // camera centres C = -M^-1 p
    std::vector<std::array<double, 3>> C(nview);
    double c[3] = {0, 0, 0};
    for (int v = 0; v < nview; ++v) {
        const double* P = Pv[v];
        const double M[3][3] = {{P[0], P[1], P[2]}, {P[4], P[5], P[6]}, {P[8], P[9], P[10]}};
        const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        if (det == 0) return false;
        double inv[3][3];
        inv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
        inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
        inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
        inv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
        inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
        inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
        inv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
        inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
        inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
        for (int i = 0; i < 3; ++i) {
            C[v][i] = -(inv[i][0] * P[3] + inv[i][1] * P[7] + inv[i][2] * P[11]);
            c[i] += C[v][i] / nview;
        }
    }
    double md = 0;
    for (int v = 0; v < nview; ++v)
        md += std::sqrt((C[v][0] - c[0]) * (C[v][0] - c[0]) + (C[v][1] - c[1]) * (C[v][1] - c[1]) +
                        (C[v][2] - c[2]) * (C[v][2] - c[2])) / nview;
    const double sc = md > 0 ? 1.0 / md : 1.0;
    // A^T A over the normalised planes
    double AtA[100] = {0};
    for (int v = 0; v < nview; ++v) {
        const double* P = Pv[v];
        const double* b = obs[v];
        const double lines[4][3] = {{1, 0, -b[0]}, {1, 0, -b[2]}, {0, 1, -b[1]}, {0, 1, -b[3]}};
        for (int e = 0; e < 4; ++e) {
            double pi[4];
            for (int k = 0; k < 4; ++k)
                pi[k] = lines[e][0] * P[k] + lines[e][1] * P[4 + k] + lines[e][2] * P[8 + k];
            // plane in the normalised frame X' = sc (X - c): (n / sc, n.c + d)
            double pn[4] = {pi[0] / sc, pi[1] / sc, pi[2] / sc, pi[0] * c[0] + pi[1] * c[1] + pi[2] * c[2] + pi[3]};
            const double nrm = std::sqrt(pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2] + pn[3] * pn[3]);
            for (int k = 0; k < 4; ++k) pn[k] /= nrm;
            const double row[10] = {pn[0] * pn[0], 2 * pn[0] * pn[1], 2 * pn[0] * pn[2], 2 * pn[0] * pn[3],
                                    pn[1] * pn[1], 2 * pn[1] * pn[2], 2 * pn[1] * pn[3], pn[2] * pn[2],
                                    2 * pn[2] * pn[3], pn[3] * pn[3]};
            for (int i = 0; i < 10; ++i)
                for (int j = 0; j < 10; ++j) AtA[i * 10 + j] += row[i] * row[j];
        }
    }
    double V[100];
    jacobi_eigen(10, AtA, V);
    int kmin = 0;
    for (int k = 1; k < 10; ++k)
        if (AtA[k * 10 + k] < AtA[kmin * 10 + kmin]) kmin = k;
    double q[10];
    for (int k = 0; k < 10; ++k) q[k] = V[k * 10 + kmin];
    const int idx[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
    double Qn[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Qn[i][j] = q[idx[i][j]];
    // back to the world frame: Q* = T^-1 Q*' T^-T with T^-1 = [[I/sc, c], [0, 1]]
    double Ti[4][4] = {{1 / sc, 0, 0, c[0]}, {0, 1 / sc, 0, c[1]}, {0, 0, 1 / sc, c[2]}, {0, 0, 0, 1}};
    double Q[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0;
            for (int k = 0; k < 4; ++k)
                for (int l = 0; l < 4; ++l) acc += Ti[i][k] * Qn[k][l] * Ti[j][l];
            Q[i][j] = acc;
        }
    if (std::fabs(Q[3][3]) < 1e-300) return false;
    const double f = -1.0 / Q[3][3];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Q[i][j] *= f;
    if (Qout)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) Qout[4 * i + j] = Q[i][j];
    const double t[3] = {-Q[0][3], -Q[1][3], -Q[2][3]};
    double M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = Q[i][j] + t[i] * t[j];
    double E[9];
    jacobi_eigen(3, M, E);
    int order[3] = {0, 1, 2};
    std::sort(order, order + 3, [&](int a, int b) { return M[4 * a] > M[4 * b]; });
    double R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) R[i][k] = E[3 * i + order[k]];
    const double detR = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                        R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                        R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
    if (detR < 0)
        for (int i = 0; i < 3; ++i) R[i][2] = -R[i][2];
    for (int k = 0; k < 3; ++k) {
        params[k] = t[k];
        params[3 + k] = 0.5 * std::log(std::max(M[4 * order[k]], 1e-6));
    }
    rot_to_rotvec(R, params + 6);
    return true;
}

}  // namespace

extern "C" {

// Helpers exposed for pinning: symmetric eigen-decomposition and the rotation log map.
int oracle_jacobi_eigen(int n, double* A, double* V) {
    jacobi_eigen(n, A, V);
    return 0;
}
int oracle_rot_to_rotvec(const double* R9, double* r3) {
    const double R[3][3] = {{R9[0], R9[1], R9[2]}, {R9[3], R9[4], R9[5]}, {R9[6], R9[7], R9[8]}};
    rot_to_rotvec(R, r3);
    return 0;
}

// Plain multi-view fit of each quadric: the Eq. 1 initialisation from its views' boxes
// (or the given start[nq*9], if not NULL), then `iters` Adam steps (Kingma & Ba; lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the
// Eq. 12 bbox loss.  Outputs (each may be NULL): init[nq*9], params[nq*9], init_Q[nq*16]
// (Q* after the initialisation, Q*44 = -1), loss[nq] (loss at the final parameters),
// ok[nq] (initialisation succeeded).
int oracle_quadric_fit(int nq, int nv, const double* P, const int32_t* q_ptr, const int32_t* pair_v,
                       const double* obs, int iters, double lr, double* init, double* params, double* init_Q,
                       double* loss, uint8_t* ok, const double* start) {
    for (int q = 0; q < nq; ++q) {
        const int k0 = q_ptr[q], k1 = q_ptr[q + 1];
        std::vector<const double*> Pv, ob;
        for (int k = k0; k < k1; ++k) {
            if (pair_v[k] < 0 || pair_v[k] >= nv) return 1;
            Pv.push_back(P + 12 * pair_v[k]);
            ob.push_back(obs + 4 * k);
        }
        double p[9] = {0}, Q16[16] = {0};
        bool good;
        if (start) {  // refine from a given starting point instead of the initialisation
            for (int i = 0; i < 9; ++i) p[i] = start[9 * q + i];
            good = k1 - k0 >= 1;
        } else {
            good = k1 - k0 >= 3 && quadric_init(k1 - k0, Pv.data(), ob.data(), p, Q16);
        }
        if (ok) ok[q] = good;
        if (init) for (int i = 0; i < 9; ++i) init[9 * q + i] = p[i];
        if (init_Q) for (int i = 0; i < 16; ++i) init_Q[16 * q + i] = Q16[i];
        double m[9] = {0}, v2[9] = {0};
        double b1t = 1, b2t = 1;
        double L = 0, g[9];
        const int32_t zero_ptr[2] = {0, k1 - k0};
        std::vector<int32_t> views(pair_v + k0, pair_v + k1);
        for (int it = 1; good && it <= iters; ++it) {
            oracle_quadric_bbox_loss(1, p, nv, P, zero_ptr, views.data(), obs + 4 * k0, &L, g);
            b1t *= 0.9;
            b2t *= 0.999;
            for (int i = 0; i < 9; ++i) {
                m[i] = 0.9 * m[i] + 0.1 * g[i];
                v2[i] = 0.999 * v2[i] + 0.001 * g[i] * g[i];
                const double mh = m[i] / (1 - b1t), vh = v2[i] / (1 - b2t);
                p[i] -= lr * mh / (std::sqrt(vh) + 1e-8);
            }
        }
        if (good) oracle_quadric_bbox_loss(1, p, nv, P, zero_ptr, views.data(), obs + 4 * k0, &L, g);
        if (params) for (int i = 0; i < 9; ++i) params[9 * q + i] = p[i];
        if (loss) loss[q] = good ? L : 0;
    }
    return 0;
}

}  // extern "C"

// ============================================================================ learned proposal
//
// FP64 reference of the learned quadric proposal (an addition to the paper's method: a
// small network proposes the quadric's initial value, which the Eq. 12 refinement then
// fits).  Rounding to bfloat16 happens at the same points as in the kernels (weights,
// hidden activations, the output gradient and the hidden-layer gradients) unless `rb` is
// 0, which gives the plain FP64 network the finite-difference pins differentiate.

namespace {

// Nearest bfloat16 value (8 significant bits, ties to even; fp32 exponent range).
double round_bf16(double x) {
    if (x == 0 || !std::isfinite(x)) return x;
    int e;
    const double m = std::frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
    int bits = 8;
    if (e < -125) bits = std::max(0, 8 - (-125 - e));  // subnormal: spacing 2^-133
    return std::ldexp(std::nearbyint(std::ldexp(m, bits)), e - bits);
}

constexpr int MI = 128, MH = 128, MO = 9, MOP = 16;
constexpr int OW1 = 0, OB1 = 16384, OW2 = 16512, OB2 = 32896, OW3 = 33024, OB3 = 35072, OPARAMS = 35088;

// Upper-triangular K (positive diagonal, K22 = 1) and rotation R with M = lambda K R, from
// M M^T = lambda^2 K K^T: Cholesky of the row- and column-reversed matrix.
bool camera_from_P(const double P[12], double K[3][3], double R[3][3], double t[3]) {
    double M[3][3], p[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = P[4 * i + j];
        p[i] = P[4 * i + 3];
    }
    double A[3][3];  // A = J M M^T J, J the reversal
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += M[2 - i][k] * M[2 - j][k];
            A[i][j] = s;
        }
    double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0)) return false;
                L[i][i] = std::sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    // K = J L J is upper triangular with K K^T = M M^T
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K[i][j] = L[2 - i][2 - j];
    const double lam = K[2][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K[i][j] /= lam;
    // R = K^-1 M / lambda (back substitution), sign fixed by det R = +1
    double Ki[3][3];
    Ki[2][2] = 1; Ki[2][1] = 0; Ki[2][0] = 0; Ki[1][0] = 0; Ki[0][0] = 1 / K[0][0]; Ki[1][1] = 1 / K[1][1];
    Ki[1][2] = -K[1][2] / K[1][1];
    Ki[0][1] = -K[0][1] / (K[0][0] * K[1][1]);
    Ki[0][2] = (K[0][1] * K[1][2] - K[0][2] * K[1][1]) / (K[0][0] * K[1][1]);
    double sg = 1;
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int k = 0; k < 3; ++k) s += Ki[i][k] * M[k][j];
                R[i][j] = sg * s / lam;
            }
        const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                           R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                           R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
        if (det > 0) break;
        sg = -1;
    }
    for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += Ki[i][k] * p[k];
        t[i] = sg * s / lam;
    }
    return true;
}

void mlp_forward_one(const double* x, const double* prm, bool rb, double* h1, double* h2, double* y) {
    auto W = [&](int off, int o, int i, int ld) { const double w = prm[off + o * ld + i]; return rb ? round_bf16(w) : w; };
    for (int o = 0; o < MH; ++o) {
        double z = prm[OB1 + o];
        for (int i = 0; i < MI; ++i) z += W(OW1, o, i, MI) * x[i];
        const double h = std::max(z, 0.0);
        h1[o] = rb ? round_bf16(h) : h;
    }
    for (int o = 0; o < MH; ++o) {
        double z = prm[OB2 + o];
        for (int i = 0; i < MH; ++i) z += W(OW2, o, i, MH) * h1[i];
        const double h = std::max(z, 0.0);
        h2[o] = rb ? round_bf16(h) : h;
    }
    for (int o = 0; o < MO; ++o) {
        double z = prm[OB3 + o];
        for (int i = 0; i < MH; ++i) z += W(OW3, o, i, MH) * h2[i];
        y[o] = z;
    }
}

}  // namespace

extern "C" {

double oracle_round_bf16(double x) { return round_bf16(x); }

// Features of the learned proposal (FP64, not rounded): per quadric 8 view slots of
// [xn, yn, hw, hh, r1, r2, d, C * inv_scale]; see dqo_mlp_features for the definition.
int oracle_mlp_features(int nq, int nv, const double* P, const int32_t* q_ptr, const int32_t* pair_v,
                        const double* obs, const int32_t* counts, double inv_scale, double* F) {
    for (int q = 0; q < nq; ++q) {
        const int k0 = q_ptr[q], k1 = q_ptr[q + 1];
        int use = std::min(k1 - k0, 8);
        if (counts) use = std::min(use, (int)counts[q]);
        for (int j = 0; j < 8; ++j) {
            double* f = F + (int64_t)q * MI + 16 * j;
            for (int k = 0; k < 16; ++k) f[k] = 0;
            if (j >= use) continue;
            const int v = pair_v[k0 + j];
            if (v < 0 || v >= nv) return 1;
            double K[3][3], R[3][3], t[3];
            if (!camera_from_P(P + 12 * v, K, R, t)) continue;
            const double* b = obs + 4 * (int64_t)(k0 + j);
            const double uc = 0.5 * (b[0] + b[2]), vc = 0.5 * (b[1] + b[3]);
            // normalised coordinates = K^-1 (uc, vc, 1)
            const double yn = (vc - K[1][2]) / K[1][1];
            const double xn = (uc - K[0][2] - K[0][1] * yn) / K[0][0];
            f[0] = xn;
            f[1] = yn;
            f[2] = (b[2] - b[0]) / (2 * K[0][0]);
            f[3] = (b[3] - b[1]) / (2 * K[1][1]);
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = R[0][k] * xn + R[1][k] * yn + R[2][k];  // R^T (xn, yn, 1)
            const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int k = 0; k < 3; ++k) {
                f[4 + k] = R[0][k];
                f[7 + k] = R[1][k];
                f[10 + k] = d[k] / dn;
                f[13 + k] = -(R[0][k] * t[0] + R[1][k] * t[1] + R[2][k] * t[2]) * inv_scale;
            }
        }
    }
    return 0;
}

// Network outputs y [n][9] (and the hidden activations h1, h2 [n][128], each may be NULL)
// for inputs X [n][128] and the parameter vector prm (layout of dqo_mlp_features' network).
int oracle_mlp_forward(int64_t n, const double* X, const double* prm, int rb, double* y, double* h1, double* h2) {
    std::vector<double> a(MH), b(MH);
    for (int64_t s = 0; s < n; ++s) {
        double yy[MO];
        mlp_forward_one(X + s * MI, prm, rb != 0, a.data(), b.data(), yy);
        if (y) for (int k = 0; k < MO; ++k) y[s * MO + k] = yy[k];
        if (h1) for (int k = 0; k < MH; ++k) h1[s * MH + k] = a[k];
        if (h2) for (int k = 0; k < MH; ++k) h2[s * MH + k] = b[k];
    }
    return 0;
}

// Loss (1/n) sum_s sum_j w_j (y_sj - label_sj)^2 and its gradient w.r.t. the parameter
// vector (grads [35088] overwritten), by the chain rule through the three layers.
int oracle_mlp_backward(int64_t n, const double* X, const double* labels, const double* w, const double* prm,
                        int rb, double* grads, double* loss) {
    const bool r = rb != 0;
    auto W = [&](int off, int o, int i, int ld) { const double v = prm[off + o * ld + i]; return r ? round_bf16(v) : v; };
    for (int k = 0; k < OPARAMS; ++k) grads[k] = 0;
    double L = 0;
    std::vector<double> h1(MH), h2(MH), dz2(MH), dz1(MH);
    for (int64_t s = 0; s < n; ++s) {
        const double* x = X + s * MI;
        double y[MO], dy[MO];
        mlp_forward_one(x, prm, r, h1.data(), h2.data(), y);
        for (int j = 0; j < MO; ++j) {
            const double e = y[j] - labels[s * MO + j];
            L += w[j] * e * e / (double)n;
            dy[j] = 2 * w[j] * e / (double)n;
            if (r) dy[j] = round_bf16(dy[j]);
        }
        for (int j = 0; j < MO; ++j) {
            grads[OB3 + j] += dy[j];
            for (int i = 0; i < MH; ++i) grads[OW3 + j * MH + i] += dy[j] * h2[i];
        }
        for (int i = 0; i < MH; ++i) {
            double g = 0;
            for (int j = 0; j < MO; ++j) g += dy[j] * W(OW3, j, i, MH);
            const double v = h2[i] > 0 ? g : 0.0;
            dz2[i] = r ? round_bf16(v) : v;
        }
        for (int o = 0; o < MH; ++o) {
            grads[OB2 + o] += dz2[o];
            for (int i = 0; i < MH; ++i) grads[OW2 + o * MH + i] += dz2[o] * h1[i];
        }
        for (int i = 0; i < MH; ++i) {
            double g = 0;
            for (int o = 0; o < MH; ++o) g += dz2[o] * W(OW2, o, i, MH);
            const double v = h1[i] > 0 ? g : 0.0;
            dz1[i] = r ? round_bf16(v) : v;
        }
        for (int o = 0; o < MH; ++o) {
            grads[OB1 + o] += dz1[o];
            for (int i = 0; i < MI; ++i) grads[OW1 + o * MI + i] += dz1[o] * x[i];
        }
    }
    if (loss) *loss = L;
    return 0;
}

// Canonical parameters (see dqo_quadric_canonical): the same ellipsoid with axes
// descending (stable), the rotation's columns permuted with them, det +1, and of the four
// sign patterns diag(1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1) the first of largest trace.
int oracle_quadric_canonical(int nq, const double* in, double* out) {
    for (int q = 0; q < nq; ++q) {
        const double* p = in + 9 * q;
        double R[3][3];
        rotvec_to_rot(p + 6, R);
        int ord[3] = {0, 1, 2};
        std::stable_sort(ord, ord + 3, [&](int a, int b) { return p[3 + a] > p[3 + b]; });
        double S[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) S[i][k] = R[i][ord[k]];
        const double det = S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) -
                           S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0]) +
                           S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]);
        if (det < 0) for (int i = 0; i < 3; ++i) S[i][2] = -S[i][2];
        const double sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        int best = 0;
        double bt = -1e300;
        for (int c = 0; c < 4; ++c) {
            const double tr = sg[c][0] * S[0][0] + sg[c][1] * S[1][1] + sg[c][2] * S[2][2];
            if (tr > bt) { bt = tr; best = c; }
        }
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) S[i][k] *= sg[best][k];
        double* o = out + 9 * q;
        const double c0 = p[0], c1 = p[1], c2 = p[2], l0 = p[3 + ord[0]], l1 = p[3 + ord[1]], l2 = p[3 + ord[2]];
        o[0] = c0; o[1] = c1; o[2] = c2; o[3] = l0; o[4] = l1; o[5] = l2;
        rot_to_rotvec(S, o + 6);
    }
    return 0;
}

}  // extern "C"
