// K1 (projection) and K8 (projection adjoint) of the rasterizer.
//
// K1 maps each 3D Gaussian to its screen footprint (EWA splatting, the 3DGS rasterizer
// DQO-MAP optimises with; Sec. IV impl.): camera-space mean, 2D covariance
// Sigma' = J W M M^T W^T J^T + lowpass I with M = R(q) diag(exp(s)), its inverse (the
// conic, pre-scaled for exp2), a 3-sigma tile rect narrowed to where alpha can reach
// alpha_min, opacity = sigmoid(logit), and the depth-sort key.  One thread per Gaussian;
// each warp stages its 32 Gaussians' [n,3] rows through shared memory with float4 loads.
//
// K8 recomputes the same forward quantities and chains the per-Gaussian moment record
// of the blend backward through the conic inverse, the EWA Jacobian, the scale/rotation
// factorisation, quaternion normalisation and the sigmoid.
#include "dqo_internal.cuh"

namespace dqo {
namespace {

struct Footprint {
  bool visible;
  float pc[3];
  float xy[2];
  float cov[3];     // Sigma' (A, B, C)
  float conic[3];   // (a, b, c) = inverse of Sigma'
  float opac;
  ushort4 rect;
  uint32_t ntiles;
  // factors kept for the adjoint
  float R[3][3], s[3], qn[4], qinv;
  float T2[2][3], V[2][3];
};

__device__ __forceinline__ void quat_rot(const float q[4], float R[3][3]) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z);       R[0][2] = 2.f * (x * z + w * y);
  R[1][0] = 2.f * (x * y + w * z);       R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
  R[2][0] = 2.f * (x * z - w * y);       R[2][1] = 2.f * (y * z + w * x);       R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// s + err = a + b exactly (Knuth's two-sum; explicit roundings, nothing contracted).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a0 m0 + a1 m1 + a2 m2 + t, rounded once: each product is split exactly into its rounded
// value and its error (an FMA), the four leading terms are added with error-free two-sums
// and the small parts are added before the single final rounding.  The sum before that
// rounding is within about 2^-47 (relative) of the exact value, so the result is the exact
// value correctly rounded except within that distance of a rounding boundary -- what an
// evaluation in double precision rounded to float gives, without the double-precision
// pipe (a small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ float dot3_plus(float a0, float m0, float a1, float m1, float a2, float m2, float t) {
  const float p0 = __fmul_rn(a0, m0), e0 = __fmaf_rn(a0, m0, -p0);
  const float p1 = __fmul_rn(a1, m1), e1 = __fmaf_rn(a1, m1, -p1);
  const float p2 = __fmul_rn(a2, m2), e2 = __fmaf_rn(a2, m2, -p2);
  float s, r1, r2, r3;
  two_sum(p0, p1, s, r1);
  two_sum(s, p2, s, r2);
  two_sum(s, t, s, r3);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, r1)), __fadd_rn(r2, r3));
  return __fadd_rn(s, lo);
}

// Same footprint computation for K1 and K8 (identical code path, identical rounding).  K8
// passes kRect = false: it recomputes only what its chain rule reads and takes visibility
// from K1's tile count, so it stops before the tile rect (visible once the mean and conic
// are finite, as they were in K1).
template <bool kRect = true>
__device__ __forceinline__ void footprint(const RasterParams& rp, const float mean[3], const float ls[3],
                                          const float4 q4, float logit, Footprint& f) {
  f.visible = false;
  f.ntiles = 0;
  f.rect = make_ushort4(0, 0, 0, 0);
  const float* V = rp.vm;
  // Camera-space mean rounded once from its exact value, so z (the depth-sort key) is the
  // correctly rounded depth of the float inputs, reproducible by any exact evaluation.
#pragma unroll
  for (int i = 0; i < 3; ++i)
    f.pc[i] = dot3_plus(V[4 * i + 0], mean[0], V[4 * i + 1], mean[1], V[4 * i + 2], mean[2], V[4 * i + 3]);
  const float x = f.pc[0], y = f.pc[1], z = f.pc[2];
  f.opac = 1.f / (1.f + expf(-logit));
  if (!(z >= rp.znear)) return;
  const float qq = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
  if (!(qq > 0.f)) return;
  f.qinv = rsqrtf(qq);
  f.qn[0] = q4.x * f.qinv; f.qn[1] = q4.y * f.qinv; f.qn[2] = q4.z * f.qinv; f.qn[3] = q4.w * f.qinv;
  quat_rot(f.qn, f.R);
#pragma unroll
  for (int k = 0; k < 3; ++k) f.s[k] = expf(ls[k]);
  const float iz = 1.f / z;
  const float J00 = rp.fx * iz, J02 = -rp.fx * x * iz * iz;
  const float J11 = rp.fy * iz, J12 = -rp.fy * y * iz * iz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    f.T2[0][j] = J00 * V[j] + J02 * V[8 + j];
    f.T2[1][j] = J11 * V[4 + j] + J12 * V[8 + j];
  }
  // V = T2 R diag(s)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      f.V[i][k] = (f.T2[i][0] * f.R[0][k] + f.T2[i][1] * f.R[1][k] + f.T2[i][2] * f.R[2][k]) * f.s[k];
  const float a0 = f.V[0][0] * f.V[0][0] + f.V[0][1] * f.V[0][1] + f.V[0][2] * f.V[0][2];
  const float c0 = f.V[1][0] * f.V[1][0] + f.V[1][1] * f.V[1][1] + f.V[1][2] * f.V[1][2];
  f.cov[0] = a0 + rp.lowpass;
  f.cov[1] = f.V[0][0] * f.V[1][0] + f.V[0][1] * f.V[1][1] + f.V[0][2] * f.V[1][2];
  f.cov[2] = c0 + rp.lowpass;
  // det(V V^T + l I) = sum of squared 2x2 minors of V (Cauchy-Binet) + l (|V0|^2 + |V1|^2) + l^2:
  // all terms non-negative, so flat footprints seen edge-on keep full single precision
  // (A C - B^2 would cancel to a few digits).
  const float m01 = fmaf(f.V[0][0], f.V[1][1], -f.V[0][1] * f.V[1][0]);
  const float m02 = fmaf(f.V[0][0], f.V[1][2], -f.V[0][2] * f.V[1][0]);
  const float m12 = fmaf(f.V[0][1], f.V[1][2], -f.V[0][2] * f.V[1][1]);
  const float det = m01 * m01 + m02 * m02 + m12 * m12 + rp.lowpass * (a0 + c0) + rp.lowpass * rp.lowpass;
  if (!(det > 0.f)) return;
  const float idet = 1.f / det;
  f.conic[0] = f.cov[2] * idet;
  f.conic[1] = -f.cov[1] * idet;
  f.conic[2] = f.cov[0] * idet;
  const float mid = 0.5f * (f.cov[0] + f.cov[2]);
  const float lmax = mid + sqrtf(fmaxf(0.f, mid * mid - det));
  const float r = ceilf(rp.radius_sigma * sqrtf(lmax));
  f.xy[0] = fmaf(rp.fx, x * iz, rp.cx);
  f.xy[1] = fmaf(rp.fy, y * iz, rp.cy);
  if (!isfinite(f.xy[0]) || !isfinite(f.xy[1]) || !isfinite(r)) return;
  if (!kRect) {
    f.visible = true;
    return;
  }
  // The rect's half-widths: the 3-sigma radius r, narrowed (alpha_min > 0) to the bounding
  // box of the ellipse q <= T' outside of which no pixel blends the Gaussian.  The blend
  // skips alpha < alpha_min and alpha <= opacity * G, so a blended pixel has
  // q <= T = 2 ln(opacity / alpha_min).  T' = T (1 + 2^-10) + 2^-14 (a + c) R^2 + 2^-10 with
  // R = r + max(tile_w, tile_h) (no pixel of a tile of the square is farther from the
  // centre along either axis) exceeds T by more than the rounding of the conic, of dx and
  // dy and of the exponent's evaluation can move q at such a pixel (a few units of 2^-24
  // times (a + c) R^2), so every tile dropped here holds only pixels that skip the
  // Gaussian and no pixel value changes.  The box of {q <= T'} has half-widths
  // sqrt(T' Sigma'_xx) and sqrt(T' Sigma'_yy); T' <= 0 (opacity below alpha_min) culls.
  float hx = r, hy = r;
  if (rp.alpha_min > 0.f) {
    const float T = 2.f * (logf(f.opac) - logf(rp.alpha_min));
    const float R = r + (float)max(rp.tile_w, rp.tile_h);
    const float Tm = fmaf(T, 1.f + 0x1p-10f, fmaf(0x1p-14f * (f.conic[0] + f.conic[2]), R * R, 0x1p-10f));
    if (!(Tm > 0.f)) return;
    hx = fminf(r, sqrtf(Tm * f.cov[0]));
    hy = fminf(r, sqrtf(Tm * f.cov[2]));
  }
  // tiles holding a pixel centre inside [x - hx, x + hx] x [y - hy, y + hy]
  float ulo = ceilf(f.xy[0] - hx), uhi = floorf(f.xy[0] + hx);
  float vlo = ceilf(f.xy[1] - hy), vhi = floorf(f.xy[1] + hy);
  ulo = fmaxf(ulo, 0.f);
  vlo = fmaxf(vlo, 0.f);
  uhi = fminf(uhi, (float)(rp.W - 1));
  vhi = fminf(vhi, (float)(rp.H - 1));
  if (ulo > uhi || vlo > vhi) return;
  const int tx0 = (int)ulo / rp.tile_w, tx1 = (int)uhi / rp.tile_w + 1;
  const int ty0 = (int)vlo / rp.tile_h, ty1 = (int)vhi / rp.tile_h + 1;
  f.rect = make_ushort4((unsigned short)tx0, (unsigned short)ty0, (unsigned short)tx1, (unsigned short)ty1);
  f.ntiles = (uint32_t)((tx1 - tx0) * (ty1 - ty0));
  f.visible = true;
}

// A warp's 32 rows of an [n,3] array: whole warps with a 16-byte-aligned base load the 96
// floats as 24 float4 loads (lanes 0..23, issued by load_rows3_vec) and pass them through
// shared memory (take_rows3); others load scalars.
__device__ __forceinline__ float4 load_rows3_vec(const float* __restrict__ src, int64_t wbase, bool vec, int lane) {
  return vec && lane < 24 ? __ldg(reinterpret_cast<const float4*>(src + 3 * wbase) + lane)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void take_rows3(const float* __restrict__ src, const float4 v, bool vec, int lane,
                                           int64_t i, bool in, float* stage, float out[3]) {
  if (vec) {
    if (lane < 24) {
      stage[4 * lane + 0] = v.x; stage[4 * lane + 1] = v.y;
      stage[4 * lane + 2] = v.z; stage[4 * lane + 3] = v.w;
    }
    __syncwarp();
    out[0] = stage[3 * lane]; out[1] = stage[3 * lane + 1]; out[2] = stage[3 * lane + 2];
    __syncwarp();
  } else if (in) {
    out[0] = __ldg(src + 3 * i); out[1] = __ldg(src + 3 * i + 1); out[2] = __ldg(src + 3 * i + 2);
  }
}

// Gaussian i of g (inputs at i, outputs at base + i of o; the depth-sort value is the
// output index).  Called by every thread of a block; `stage` is the block's staging area.
__device__ __forceinline__ void preprocess_item(const RasterParams& rp, const dqo_gaussians& g, const ProjBuffers& o,
                                                int64_t i, int64_t base, float (*stage)[96]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wbase = i - lane;
  const bool full = wbase + 32 <= g.n;
  const bool in = i < g.n;
  float mean[3] = {0, 0, 0}, ls[3] = {0, 0, 0}, rgb[3] = {0, 0, 0};
  const bool vm = full && ((reinterpret_cast<uintptr_t>(g.means) & 15) == 0);
  const bool vl = full && ((reinterpret_cast<uintptr_t>(g.log_scales) & 15) == 0);
  const bool vc = full && ((reinterpret_cast<uintptr_t>(g.rgb) & 15) == 0);
  // every load of the Gaussian first (all in flight together), then the staging
  const float4 wm = load_rows3_vec(g.means, wbase, vm, lane);
  const float4 wl = load_rows3_vec(g.log_scales, wbase, vl, lane);
  const float4 wc = load_rows3_vec(g.rgb, wbase, vc, lane);
  float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
  float logit = 0.f;
  int32_t id = -1;
  uint32_t flags = 0u;
  if (in) {
    if ((reinterpret_cast<uintptr_t>(g.quats) & 15) == 0) {
      q = __ldg(reinterpret_cast<const float4*>(g.quats) + i);
    } else {
      q = make_float4(g.quats[4 * i], g.quats[4 * i + 1], g.quats[4 * i + 2], g.quats[4 * i + 3]);
    }
    logit = __ldg(g.opacity_logit + i);
    id = __ldg(g.obj_id + i);
    flags = __ldg(g.flags + i);
  }
  if (full || in) {
    take_rows3(g.means, wm, vm, lane, i, in, stage[warp], mean);
    take_rows3(g.log_scales, wl, vl, lane, i, in, stage[warp], ls);
    take_rows3(g.rgb, wc, vc, lane, i, in, stage[warp], rgb);
  }
  Footprint f;
  f.visible = false;
  if (in) {
    footprint(rp, mean, ls, q, logit, f);
    const bool has_obj = id >= 0 && id < rp.num_objects;
    const uint32_t og = (flags & 1u) ? 0x80000000u : 0u;
    const uint32_t idbits = (has_obj ? (uint32_t)id : kNoObject) | og;
    const float sc = -0.5f * kLog2e;
    const int64_t j = base + i;
    o.p0[j] = make_float4(f.xy[0], f.xy[1], sc * f.conic[0], 2.f * sc * f.conic[1]);
    o.p1[j] = make_float4(sc * f.conic[2], f.opac, f.pc[2], __uint_as_float(idbits));
    // Level of the alpha-support ellipse in the exponent's log2 units: alpha can reach
    // alpha_min only where -(a' dx^2 + b' dx dy + c' dy^2) <= log2(o / alpha_min).  Widened
    // by a small margin (the blend kernels cull with it, so it must be conservative);
    // negative if the Gaussian can reach no pixel.
    float lvl = -1.f;
    if (f.visible) {
      if (rp.alpha_min <= 0.f) {
        lvl = INFINITY;
      } else if (f.opac > rp.alpha_min) {
        const float q2 = log2f(f.opac / rp.alpha_min);
        lvl = q2 * (1.f + 1e-4f) + 1e-3f;
      }
    }
    o.p2[j] = make_float4(rgb[0], rgb[1], rgb[2], lvl);
    o.rect[j] = f.rect;
    o.ntiles[j] = f.ntiles;
    o.zkey[j] = f.visible ? __float_as_uint(f.pc[2]) : 0xFFFFFFFFu;
    o.zval[j] = (uint32_t)j;
    o.gid[j] = has_obj ? (uint32_t)id : 0xFFFFFFFFu;
    if (o.grad2d && f.ntiles > 0) {  // only binned Gaussians receive (and are read for) moments
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      o.grad2d[3 * j] = z;
      o.grad2d[3 * j + 1] = z;
      o.grad2d[3 * j + 2] = z;
    }
  }
  const uint32_t vis = __ballot_sync(0xFFFFFFFFu, in && f.visible);
  if (lane == 0 && vis) atomicAdd(o.n_visible, (uint32_t)__popc(vis));
}

__global__ void __launch_bounds__(kThreads) k_preprocess(RasterParams rp, dqo_gaussians g, ProjBuffers o) {
  __shared__ float stage[kThreads / 32][96];
  preprocess_item(rp, g, o, (int64_t)blockIdx.x * kThreads + threadIdx.x, 0, stage);
}

// Keyframe blockIdx.y of a batch.
__global__ void __launch_bounds__(kThreads) k_preprocess_batch(const __grid_constant__ PreTable t, ProjBuffers o) {
  pdl_wait();
  pdl_trigger();
  __shared__ float stage[kThreads / 32][96];
  const PreKf& kf = t.kf[blockIdx.y];
  if ((int64_t)blockIdx.x * kThreads >= kf.g.n) return;  // uniform over the block
  preprocess_item(kf.rp, kf.g, o, (int64_t)blockIdx.x * kThreads + threadIdx.x, kf.base, stage);
}

// Writes one gradient element in the call's mode: +=, atomic +=, or =.  The addition is
// rounded explicitly, so that v is formed first in every mode (0 += v gives exactly v).
__device__ __forceinline__ void put_grad(int mode, float* p, float v) {
  if (mode == kGradAtomic) atomicAdd(p, v);
  else if (mode == kGradStore) *p = v;
  else *p = __fadd_rn(*p, v);
}

// Zero gradient of a Gaussian that was never binned (written only when overwriting).
__device__ __forceinline__ void zero_grads(const PreBwdArgs& a, int64_t i) {
  if (a.mode != kGradStore) return;
  if (a.d_rgb) a.d_rgb[3 * i] = a.d_rgb[3 * i + 1] = a.d_rgb[3 * i + 2] = 0.f;
  if (a.d_logit) a.d_logit[i] = 0.f;
  if (a.d_means) a.d_means[3 * i] = a.d_means[3 * i + 1] = a.d_means[3 * i + 2] = 0.f;
  if (a.d_log_scales) a.d_log_scales[3 * i] = a.d_log_scales[3 * i + 1] = a.d_log_scales[3 * i + 2] = 0.f;
  if (a.d_quats) a.d_quats[4 * i] = a.d_quats[4 * i + 1] = a.d_quats[4 * i + 2] = a.d_quats[4 * i + 3] = 0.f;
}

// Adjoint of Gaussian i, written to a's parameter gradients in mode a.mode (atomically
// when several keyframes of a batch share them).
__device__ __forceinline__ void preprocess_backward_item(const PreBwdArgs& a, int64_t i) {
  if (i >= a.n) return;
  // every load of the Gaussian first, in flight together (the moment record is read for
  // every Gaussian and used only for the binned ones, the only ones it was written for)
  const uint32_t nt = a.ntiles[i];
  const float mean[3] = {a.means[3 * i], a.means[3 * i + 1], a.means[3 * i + 2]};
  const float ls[3] = {a.log_scales[3 * i], a.log_scales[3 * i + 1], a.log_scales[3 * i + 2]};
  const float4 q = make_float4(a.quats[4 * i], a.quats[4 * i + 1], a.quats[4 * i + 2], a.quats[4 * i + 3]);
  const float logit = a.opacity_logit[i];
  const float4 r0 = reinterpret_cast<const float4*>(a.grad2d)[3 * i + 0];  // m_x m_y m_xx m_xy
  const float4 r1 = reinterpret_cast<const float4*>(a.grad2d)[3 * i + 1];  // m_yy d_opac d_r d_g
  const float4 r2 = reinterpret_cast<const float4*>(a.grad2d)[3 * i + 2];  // d_b d_z - -
  if (nt == 0) {  // culled: never blended, zero gradient
    zero_grads(a, i);
    return;
  }
  const RasterParams& rp = a.rp;
  Footprint f;
  footprint<false>(rp, mean, ls, q, logit, f);
  if (!f.visible) {
    zero_grads(a, i);
    return;
  }
  const int mode = a.mode;
  const float ca = f.conic[0], cb = f.conic[1], cc = f.conic[2];
  // 2D mean and conic gradients from the moments (exponent -(a dx^2 + 2 b dx dy + c dy^2)/2)
  const float gx = ca * r0.x + cb * r0.y;
  const float gy = cb * r0.x + cc * r0.y;
  const float ga = -0.5f * r0.z, gb = -r0.w, gc = -0.5f * r1.x;
  if (a.d_rgb) {
    put_grad(mode, a.d_rgb + 3 * i + 0, r1.z);
    put_grad(mode, a.d_rgb + 3 * i + 1, r1.w);
    put_grad(mode, a.d_rgb + 3 * i + 2, r2.x);
  }
  if (a.d_logit) put_grad(mode, a.d_logit + i, r1.y * f.opac * (1.f - f.opac));
  // dL/dSigma' = -Cn Gm Cn, Cn = [[a, b], [b, c]], Gm = [[ga, gb/2], [gb/2, gc]]
  const float m00 = ca * ga + cb * 0.5f * gb, m01 = ca * 0.5f * gb + cb * gc;
  const float m10 = cb * ga + cc * 0.5f * gb, m11 = cb * 0.5f * gb + cc * gc;
  const float S00 = -(m00 * ca + m01 * cb);
  const float S01 = -(m00 * cb + m01 * cc);
  const float S11 = -(m10 * cb + m11 * cc);
  // Sigma' = V V^T (+ lowpass): dL/dV = 2 S V
  float dV[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dV[0][k] = 2.f * (S00 * f.V[0][k] + S01 * f.V[1][k]);
    dV[1][k] = 2.f * (S01 * f.V[0][k] + S11 * f.V[1][k]);
  }
  // V = T2 Mm, Mm = R diag(s): dT2 = dV Mm^T, dMm = T2^T dV
  float dT2[2][3], dR[3][3], ds[3];
#pragma unroll
  for (int i2 = 0; i2 < 2; ++i2)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      dT2[i2][j] = dV[i2][0] * f.R[j][0] * f.s[0] + dV[i2][1] * f.R[j][1] * f.s[1] + dV[i2][2] * f.R[j][2] * f.s[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float dM = f.T2[0][j] * dV[0][k] + f.T2[1][j] * dV[1][k];
      dR[j][k] = dM * f.s[k];
      acc += dM * f.R[j][k];
    }
    ds[k] = acc;
  }
  // T2 = J W: dJ = dT2 W^T
  const float* W = rp.vm;
  const float dJ00 = dT2[0][0] * W[0] + dT2[0][1] * W[1] + dT2[0][2] * W[2];
  const float dJ02 = dT2[0][0] * W[8] + dT2[0][1] * W[9] + dT2[0][2] * W[10];
  const float dJ11 = dT2[1][0] * W[4] + dT2[1][1] * W[5] + dT2[1][2] * W[6];
  const float dJ12 = dT2[1][0] * W[8] + dT2[1][1] * W[9] + dT2[1][2] * W[10];
  const float x = f.pc[0], y = f.pc[1], z = f.pc[2];
  const float iz = 1.f / z, iz2 = iz * iz, iz3 = iz2 * iz;
  float dpc0 = gx * rp.fx * iz + dJ02 * (-rp.fx * iz2);
  float dpc1 = gy * rp.fy * iz + dJ12 * (-rp.fy * iz2);
  float dpc2 = -gx * rp.fx * x * iz2 - gy * rp.fy * y * iz2 + r2.y + dJ00 * (-rp.fx * iz2) +
               dJ02 * (2.f * rp.fx * x * iz3) + dJ11 * (-rp.fy * iz2) + dJ12 * (2.f * rp.fy * y * iz3);
  if (a.d_means) {
#pragma unroll
    for (int j = 0; j < 3; ++j) put_grad(mode, a.d_means + 3 * i + j, W[j] * dpc0 + W[4 + j] * dpc1 + W[8 + j] * dpc2);
  }
  if (a.d_log_scales) {
#pragma unroll
    for (int k = 0; k < 3; ++k) put_grad(mode, a.d_log_scales + 3 * i + k, ds[k] * f.s[k]);
  }
  if (a.d_quats) {
    const float w = f.qn[0], qx = f.qn[1], qy = f.qn[2], qz = f.qn[3];
    float dq[4];
    dq[0] = 2.f * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] - qy * dR[2][0] + qx * dR[2][1]);
    dq[1] = 2.f * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2.f * qx * dR[1][1] - w * dR[1][2] +
                   qz * dR[2][0] + w * dR[2][1] - 2.f * qx * dR[2][2]);
    dq[2] = 2.f * (-2.f * qy * dR[0][0] + qx * dR[0][1] + w * dR[0][2] + qx * dR[1][0] + qz * dR[1][2] -
                   w * dR[2][0] + qz * dR[2][1] - 2.f * qy * dR[2][2]);
    dq[3] = 2.f * (-2.f * qz * dR[0][0] - w * dR[0][1] + qx * dR[0][2] + w * dR[1][0] - 2.f * qz * dR[1][1] +
                   qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
    const float dot = dq[0] * w + dq[1] * qx + dq[2] * qy + dq[3] * qz;
#pragma unroll
    for (int k = 0; k < 4; ++k) put_grad(mode, a.d_quats + 4 * i + k, (dq[k] - f.qn[k] * dot) * f.qinv);
  }
}

__global__ void __launch_bounds__(kThreads) k_preprocess_backward(PreBwdArgs a) {
  preprocess_backward_item(a, (int64_t)blockIdx.x * kThreads + threadIdx.x);
}

// Keyframe blockIdx.y of a batch (its ntiles and grad2d pointers already offset to its
// first Gaussian); each keyframe in its own mode (atomic where keyframes share buffers).
// CTA column 0 sums the keyframe's loss partials instead (launched first, so it runs beside
// the Gaussians' CTAs); columns 1.. take the Gaussians.
__global__ void __launch_bounds__(kThreads) k_preprocess_backward_batch(const __grid_constant__ PreBwdTable t) {
  pdl_wait();
  pdl_trigger();
  if (blockIdx.x == 0) {
    const LossKf& l = t.loss[blockIdx.y];
    if (l.loss) loss_reduce(l.part, l.tiles, l.lambda_ins, l.scale, l.loss);
    return;
  }
  preprocess_backward_item(t.kf[blockIdx.y], (int64_t)(blockIdx.x - 1) * kThreads + threadIdx.x);
}

}  // namespace

cudaError_t launch_preprocess(const RasterParams& rp, const dqo_gaussians& g, const ProjBuffers& out,
                              cudaStream_t s) {
  if (g.n == 0) return cudaSuccess;
  const int64_t blocks = (g.n + kThreads - 1) / kThreads;
  k_preprocess<<<(unsigned)blocks, kThreads, 0, s>>>(rp, g, out);
  return cudaGetLastError();
}

cudaError_t launch_preprocess_batch(const PreTable& t, int nkf, int64_t max_n, const ProjBuffers& out,
                                    cudaStream_t s) {
  if (nkf == 0 || max_n == 0) return cudaSuccess;
  const dim3 grid((unsigned)((max_n + kThreads - 1) / kThreads), (unsigned)nkf);
  launch_dep(k_preprocess_batch, dim3(grid), dim3(kThreads), s, t, out);
  return cudaGetLastError();
}

cudaError_t launch_preprocess_backward_batch(const PreBwdTable& t, int nkf, int64_t max_n, cudaStream_t s) {
  if (nkf == 0) return cudaSuccess;
  const dim3 grid((unsigned)(1 + (max_n + kThreads - 1) / kThreads), (unsigned)nkf);
  launch_dep(k_preprocess_backward_batch, dim3(grid), dim3(kThreads), s, t);
  return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(const PreBwdArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const int64_t blocks = (a.n + kThreads - 1) / kThreads;
  k_preprocess_backward<<<(unsigned)blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dqo
