// Q1-Q4: dual-quadric projection, conic -> bbox, bbox loss and its adjoint.
//
// Q* = Z diag(a^2, b^2, c^2, -1) Z^T with Z = [R t; 0 1] (Eq. 1-3 reading), projected by
// C* = P Q* P^T (Eq. 4 reading).  With P = [M | p] this is
//   C*_ij = sum_k d_k (MR)_ik (MR)_jk - h_i h_j,   d = (a^2, b^2, c^2),  h = M t + p,
// and the vertical tangents of the conic are u = (c13 -+ sqrt(du)) / c33 with
//   du = c13^2 - c11 c33 = S02^2 - S00 S22 + h2^2 S00 + h0^2 S22 - 2 h0 h2 S02,
// S_ij = sum_k d_k (MR)_ik (MR)_jk.  The expanded form drops the h0^2 h2^2 terms that
// cancel exactly, which keeps single precision accurate for small or distant objects.
// The loss of Eq. 12 (reading: sum of 1 - IoU over a quadric's valid views) is
// differentiated in reverse mode by hand; one warp per quadric walks its views (CSR)
// and reduces loss and gradient with shuffles.
#include "dqo_internal.cuh"

namespace dqo {
namespace {

struct RotCoef {
  float A, B, Cc, Dd;  // R = I + A K + B K^2; dA/dr_i = Cc r_i, dB/dr_i = Dd r_i
};

__device__ __forceinline__ RotCoef rot_coef(float s) {  // s = |r|^2
  RotCoef c;
  if (s < 0.5f) {
    c.A = 1.f + s * (-1.f / 6.f + s * (1.f / 120.f + s * (-1.f / 5040.f)));
    c.B = 0.5f + s * (-1.f / 24.f + s * (1.f / 720.f + s * (-1.f / 40320.f)));
    c.Cc = -1.f / 3.f + s * (1.f / 30.f + s * (-1.f / 840.f + s * (1.f / 45360.f)));
    c.Dd = -1.f / 12.f + s * (1.f / 180.f + s * (-1.f / 6720.f + s * (1.f / 453600.f)));
  } else {
    const float th = sqrtf(s);
    float sn, cs;
    sincosf(th, &sn, &cs);
    c.A = sn / th;
    c.B = (1.f - cs) / s;
    c.Cc = (th * cs - sn) / (s * th);
    c.Dd = (th * sn - 2.f * (1.f - cs)) / (s * s);
  }
  return c;
}

struct PairFwd {
  bool valid;
  float R[3][3], K[3][3], K2[3][3], MR[3][3], d[3], h[3];
  float S00, S01, S02, S11, S12, S22;
  float c13, c23, c33, su, sv;
  float box[4];
  RotCoef rc;
};

__device__ __forceinline__ void pair_forward(const float* __restrict__ p, const float* __restrict__ P, PairFwd& f) {
  const float r0 = p[6], r1 = p[7], r2 = p[8];
  f.rc = rot_coef(r0 * r0 + r1 * r1 + r2 * r2);
  f.K[0][0] = 0.f; f.K[0][1] = -r2; f.K[0][2] = r1;
  f.K[1][0] = r2;  f.K[1][1] = 0.f; f.K[1][2] = -r0;
  f.K[2][0] = -r1; f.K[2][1] = r0;  f.K[2][2] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      f.K2[i][j] = f.K[i][0] * f.K[0][j] + f.K[i][1] * f.K[1][j] + f.K[i][2] * f.K[2][j];
      f.R[i][j] = (i == j ? 1.f : 0.f) + f.rc.A * f.K[i][j] + f.rc.B * f.K2[i][j];
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) f.d[k] = expf(2.f * p[3 + k]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f.h[i] = P[4 * i] * p[0] + P[4 * i + 1] * p[1] + P[4 * i + 2] * p[2] + P[4 * i + 3];
#pragma unroll
    for (int k = 0; k < 3; ++k) f.MR[i][k] = P[4 * i] * f.R[0][k] + P[4 * i + 1] * f.R[1][k] + P[4 * i + 2] * f.R[2][k];
  }
  f.S00 = f.S01 = f.S02 = f.S11 = f.S12 = f.S22 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a0 = f.MR[0][k], a1 = f.MR[1][k], a2 = f.MR[2][k], dk = f.d[k];
    f.S00 += dk * a0 * a0; f.S01 += dk * a0 * a1; f.S02 += dk * a0 * a2;
    f.S11 += dk * a1 * a1; f.S12 += dk * a1 * a2; f.S22 += dk * a2 * a2;
  }
  const float h0 = f.h[0], h1 = f.h[1], h2 = f.h[2];
  f.c13 = f.S02 - h0 * h2;
  f.c23 = f.S12 - h1 * h2;
  f.c33 = f.S22 - h2 * h2;
  const float du = f.S02 * f.S02 - f.S00 * f.S22 + h2 * h2 * f.S00 + h0 * h0 * f.S22 - 2.f * h0 * h2 * f.S02;
  const float dv = f.S12 * f.S12 - f.S11 * f.S22 + h2 * h2 * f.S11 + h1 * h1 * f.S22 - 2.f * h1 * h2 * f.S12;
  f.valid = f.c33 < 0.f && h2 > 0.f && du > 0.f && dv > 0.f;
  f.su = f.valid ? sqrtf(du) : 0.f;
  f.sv = f.valid ? sqrtf(dv) : 0.f;
  if (f.valid) {
    const float ic = 1.f / f.c33;
    f.box[0] = (f.c13 + f.su) * ic;  // c33 < 0: the + root is the left edge
    f.box[2] = (f.c13 - f.su) * ic;
    f.box[1] = (f.c23 + f.sv) * ic;
    f.box[3] = (f.c23 - f.sv) * ic;
  } else {
    f.box[0] = f.box[1] = f.box[2] = f.box[3] = 0.f;
  }
}

// Loss 1 - IoU of one valid pair and its gradient w.r.t. the 9 parameters (added to g).
__device__ __forceinline__ float pair_loss_grad(const float* __restrict__ P, const float* __restrict__ p,
                                                const float* __restrict__ o, const PairFwd& f, float g[9]) {
  const float* b = f.box;
  const float ix0 = fmaxf(b[0], o[0]), iy0 = fmaxf(b[1], o[1]);
  const float ix1 = fminf(b[2], o[2]), iy1 = fminf(b[3], o[3]);
  const float iw = ix1 - ix0, ih = iy1 - iy0;
  const bool ov = iw > 0.f && ih > 0.f;
  const float inter = ov ? iw * ih : 0.f;
  const float bw = b[2] - b[0], bh = b[3] - b[1];
  const float U = bw * bh + (o[2] - o[0]) * (o[3] - o[1]) - inter;
  const float iou = inter / U;
  // d(1 - IoU)
  const float g_iou = -1.f;
  const float g_inter = g_iou * (U + inter) / (U * U);
  const float g_ap = -g_iou * inter / (U * U);
  float gb[4];
  gb[0] = -g_ap * bh; gb[2] = g_ap * bh;
  gb[1] = -g_ap * bw; gb[3] = g_ap * bw;
  if (ov) {
    const float g_iw = g_inter * ih, g_ih = g_inter * iw;
    if (b[0] > o[0]) gb[0] -= g_iw;
    if (b[2] < o[2]) gb[2] += g_iw;
    if (b[1] > o[1]) gb[1] -= g_ih;
    if (b[3] < o[3]) gb[3] += g_ih;
  }
  // box <- (c13, c23, c33, su, sv)
  const float ic = 1.f / f.c33;
  const float g_c13 = (gb[0] + gb[2]) * ic;
  const float g_su = (gb[0] - gb[2]) * ic;
  const float g_c23 = (gb[1] + gb[3]) * ic;
  const float g_sv = (gb[1] - gb[3]) * ic;
  const float g_c33 = -(gb[0] * b[0] + gb[2] * b[2] + gb[1] * b[1] + gb[3] * b[3]) * ic;
  const float g_du = g_su / (2.f * f.su);
  const float g_dv = g_sv / (2.f * f.sv);
  const float h0 = f.h[0], h1 = f.h[1], h2 = f.h[2];
  // (c13, c23, c33, du, dv) <- (S, h)
  const float gS02 = g_c13 + g_du * (2.f * f.S02 - 2.f * h0 * h2);
  const float gS00 = g_du * (h2 * h2 - f.S22);
  const float gS12 = g_c23 + g_dv * (2.f * f.S12 - 2.f * h1 * h2);
  const float gS11 = g_dv * (h2 * h2 - f.S22);
  const float gS22 = g_c33 + g_du * (h0 * h0 - f.S00) + g_dv * (h1 * h1 - f.S11);
  float gh[3];
  gh[0] = -h2 * g_c13 + g_du * (2.f * h0 * f.S22 - 2.f * h2 * f.S02);
  gh[1] = -h2 * g_c23 + g_dv * (2.f * h1 * f.S22 - 2.f * h2 * f.S12);
  gh[2] = -h0 * g_c13 - h1 * g_c23 - 2.f * h2 * g_c33 + g_du * (2.f * h2 * f.S00 - 2.f * h0 * f.S02) +
          g_dv * (2.f * h2 * f.S11 - 2.f * h1 * f.S12);
  // S <- (d, MR)
  float gMR[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a0 = f.MR[0][k], a1 = f.MR[1][k], a2 = f.MR[2][k], dk = f.d[k];
    const float gd = gS00 * a0 * a0 + gS02 * a0 * a2 + gS22 * a2 * a2 + gS11 * a1 * a1 + gS12 * a1 * a2;
    g[3 + k] += 2.f * dk * gd;  // d_k = exp(2 l_k)
    gMR[0][k] = dk * (2.f * gS00 * a0 + gS02 * a2);
    gMR[1][k] = dk * (2.f * gS11 * a1 + gS12 * a2);
    gMR[2][k] = dk * (gS02 * a0 + 2.f * gS22 * a2 + gS12 * a1);
  }
  // MR = M R, h = M t + p
  float gR[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    g[j] += P[j] * gh[0] + P[4 + j] * gh[1] + P[8 + j] * gh[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) gR[j][k] = P[j] * gMR[0][k] + P[4 + j] * gMR[1][k] + P[8 + j] * gMR[2][k];
  }
  // R = I + A K + B K^2 (Rodrigues), K = [r]x
  float gK = 0.f, gK2 = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gK += gR[i][j] * f.K[i][j];
      gK2 += gR[i][j] * f.K2[i][j];
    }
  // <gR, E_i> with E_i = [e_i]x, and <gR, E_i K + K E_i>
  const float r[3] = {p[6], p[7], p[8]};
  // [e_0]x = [[0,0,0],[0,0,-1],[0,1,0]], [e_1]x = [[0,0,1],[0,0,0],[-1,0,0]], [e_2]x = [[0,-1,0],[1,0,0],[0,0,0]]
  const float gE[3] = {gR[2][1] - gR[1][2], gR[0][2] - gR[2][0], gR[1][0] - gR[0][1]};
  // E_i K + K E_i = r e_i^T + e_i r^T - 2 (e_i . r) I  (identity for [a]x[b]x + [b]x[a]x)
  float tr = gR[0][0] + gR[1][1] + gR[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float gEK = -2.f * r[i] * tr;
#pragma unroll
    for (int j = 0; j < 3; ++j) gEK += (gR[j][i] + gR[i][j]) * r[j];
    g[6 + i] += f.rc.A * gE[i] + f.rc.B * gEK + f.rc.Cc * r[i] * gK + f.rc.Dd * r[i] * gK2;
  }
  return 1.f - iou;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void k_quadric_project(int nq, const float* __restrict__ params, int nv, const float* __restrict__ Pm,
                                  const int32_t* __restrict__ q_ptr, const int32_t* __restrict__ pair_v, int npairs,
                                  float* __restrict__ conic, float* __restrict__ bbox, uint8_t* __restrict__ valid) {
  const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  float p[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) p[k] = params[9 * q + k];
  const int k0 = max(q_ptr[q], 0), k1 = min(q_ptr[q + 1], npairs);
  for (int k = k0 + lane; k < k1; k += 32) {
    const int v = pair_v[k];
    PairFwd f;
    bool ok = v >= 0 && v < nv;
    if (ok) {
      pair_forward(p, Pm + 12 * v, f);
      ok = f.valid;
    }
    if (conic) {
      float* c = conic + 6 * (int64_t)k;
      if (v >= 0 && v < nv) {
        c[0] = f.S00 - f.h[0] * f.h[0];
        c[1] = f.S01 - f.h[0] * f.h[1];
        c[2] = f.c13;
        c[3] = f.S11 - f.h[1] * f.h[1];
        c[4] = f.c23;
        c[5] = f.c33;
      } else {
        c[0] = c[1] = c[2] = c[3] = c[4] = c[5] = 0.f;
      }
    }
    if (bbox) {
#pragma unroll
      for (int j = 0; j < 4; ++j) bbox[4 * (int64_t)k + j] = ok ? f.box[j] : 0.f;
    }
    if (valid) valid[k] = ok ? 1 : 0;
  }
}

__global__ void k_quadric_bbox_loss(int nq, const float* __restrict__ params, int nv, const float* __restrict__ Pm,
                                    const int32_t* __restrict__ q_ptr, const int32_t* __restrict__ pair_v, int npairs,
                                    const float* __restrict__ obs, float* __restrict__ loss,
                                    float* __restrict__ dparams) {
  const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  float p[9], g[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    p[k] = params[9 * q + k];
    g[k] = 0.f;
  }
  float l = 0.f;
  const int k0 = max(q_ptr[q], 0), k1 = min(q_ptr[q + 1], npairs);
  for (int k = k0 + lane; k < k1; k += 32) {
    const int v = pair_v[k];
    if (v < 0 || v >= nv) continue;
    PairFwd f;
    pair_forward(p, Pm + 12 * v, f);
    if (!f.valid) continue;
    l += pair_loss_grad(Pm + 12 * v, p, obs + 4 * (int64_t)k, f, g);
  }
  l = warp_sum(l);
#pragma unroll
  for (int k = 0; k < 9; ++k) g[k] = warp_sum(g[k]);
  if (lane == 0) {
    if (loss) loss[q] = l;
    if (dparams)
#pragma unroll
      for (int k = 0; k < 9; ++k) dparams[9 * q + k] = g[k];
  }
}

}  // namespace

cudaError_t launch_quadric_project(int nq, const float* params, int nv, const float* P, const int32_t* q_ptr,
                                   const int32_t* pair_v, int npairs, float* conic, float* bbox, uint8_t* valid,
                                   cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nq + 3) / 4);
  k_quadric_project<<<blocks, 128, 0, s>>>(nq, params, nv, P, q_ptr, pair_v, npairs, conic, bbox, valid);
  return cudaGetLastError();
}

cudaError_t launch_quadric_bbox_loss(int nq, const float* params, int nv, const float* P, const int32_t* q_ptr,
                                     const int32_t* pair_v, int npairs, const float* obs, float* loss, float* dparams,
                                     cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nq + 3) / 4);
  k_quadric_bbox_loss<<<blocks, 128, 0, s>>>(nq, params, nv, P, q_ptr, pair_v, npairs, obs, loss, dparams);
  return cudaGetLastError();
}

}  // namespace dqo
