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
    __sincosf(th, &sn, &cs);   // th < pi in the parameterisation's use; absolute error ~1e-6
    const float is = __fdividef(1.f, s);
    c.A = __fdividef(sn, th);
    c.B = (1.f - cs) * is;
    c.Cc = __fdividef((th * cs - sn) * is, th);
    c.Dd = (th * sn - 2.f * (1.f - cs)) * is * is;
  }
  return c;
}

// The parts of the projection that depend on the quadric only (shared by all its views).
struct QuadCommon {
  float R[3][3], K[3][3], K2[3][3], d[3];
  RotCoef rc;
};

__device__ __forceinline__ void quad_common(const float* __restrict__ p, QuadCommon& c) {
  const float r0 = p[6], r1 = p[7], r2 = p[8];
  c.rc = rot_coef(r0 * r0 + r1 * r1 + r2 * r2);
  c.K[0][0] = 0.f; c.K[0][1] = -r2; c.K[0][2] = r1;
  c.K[1][0] = r2;  c.K[1][1] = 0.f; c.K[1][2] = -r0;
  c.K[2][0] = -r1; c.K[2][1] = r0;  c.K[2][2] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      c.K2[i][j] = c.K[i][0] * c.K[0][j] + c.K[i][1] * c.K[1][j] + c.K[i][2] * c.K[2][j];
      c.R[i][j] = (i == j ? 1.f : 0.f) + c.rc.A * c.K[i][j] + c.rc.B * c.K2[i][j];
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) c.d[k] = __expf(2.f * p[3 + k]);
}

struct PairFwd {
  bool valid;
  float MR[3][3], h[3];
  float S00, S01, S02, S11, S12, S22;
  float c13, c23, c33, su, sv, ic;
  float box[4];
};

__device__ __forceinline__ void pair_forward(const float* __restrict__ p, const QuadCommon& qc,
                                             const float* __restrict__ P, PairFwd& f) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f.h[i] = P[4 * i] * p[0] + P[4 * i + 1] * p[1] + P[4 * i + 2] * p[2] + P[4 * i + 3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      f.MR[i][k] = P[4 * i] * qc.R[0][k] + P[4 * i + 1] * qc.R[1][k] + P[4 * i + 2] * qc.R[2][k];
  }
  f.S00 = f.S01 = f.S02 = f.S11 = f.S12 = f.S22 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a0 = f.MR[0][k], a1 = f.MR[1][k], a2 = f.MR[2][k], dk = qc.d[k];
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
    f.ic = __fdividef(1.f, f.c33);
    f.box[0] = (f.c13 + f.su) * f.ic;  // c33 < 0: the + root is the left edge
    f.box[2] = (f.c13 - f.su) * f.ic;
    f.box[1] = (f.c23 + f.sv) * f.ic;
    f.box[3] = (f.c23 - f.sv) * f.ic;
  } else {
    f.ic = 0.f;
    f.box[0] = f.box[1] = f.box[2] = f.box[3] = 0.f;
  }
}

// Loss 1 - IoU of one valid pair and its gradient w.r.t. the 9 parameters (added to g).
__device__ __forceinline__ float pair_loss_grad(const float* __restrict__ P, const float* __restrict__ p,
                                                const float* __restrict__ o, const QuadCommon& qc,
                                                const PairFwd& f, float g[9]) {
  const float* b = f.box;
  const float ix0 = fmaxf(b[0], o[0]), iy0 = fmaxf(b[1], o[1]);
  const float ix1 = fminf(b[2], o[2]), iy1 = fminf(b[3], o[3]);
  const float iw = ix1 - ix0, ih = iy1 - iy0;
  const bool ov = iw > 0.f && ih > 0.f;
  const float inter = ov ? iw * ih : 0.f;
  const float bw = b[2] - b[0], bh = b[3] - b[1];
  const float U = bw * bh + (o[2] - o[0]) * (o[3] - o[1]) - inter;
  const float iU = __fdividef(1.f, U);
  const float iou = inter * iU;
  // d(1 - IoU)
  const float g_iou = -1.f;
  const float g_inter = g_iou * (U + inter) * iU * iU;
  const float g_ap = -g_iou * inter * iU * iU;
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
  const float ic = f.ic;
  const float g_c13 = (gb[0] + gb[2]) * ic;
  const float g_su = (gb[0] - gb[2]) * ic;
  const float g_c23 = (gb[1] + gb[3]) * ic;
  const float g_sv = (gb[1] - gb[3]) * ic;
  const float g_c33 = -(gb[0] * b[0] + gb[2] * b[2] + gb[1] * b[1] + gb[3] * b[3]) * ic;
  const float g_du = __fdividef(g_su, 2.f * f.su);
  const float g_dv = __fdividef(g_sv, 2.f * f.sv);
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
    const float a0 = f.MR[0][k], a1 = f.MR[1][k], a2 = f.MR[2][k], dk = qc.d[k];
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
      gK += gR[i][j] * qc.K[i][j];
      gK2 += gR[i][j] * qc.K2[i][j];
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
    g[6 + i] += qc.rc.A * gE[i] + qc.rc.B * gEK + qc.rc.Cc * r[i] * gK + qc.rc.Dd * r[i] * gK2;
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
  QuadCommon qc;
  quad_common(p, qc);
  for (int k = k0 + lane; k < k1; k += 32) {
    const int v = pair_v[k];
    PairFwd f;
    bool ok = v >= 0 && v < nv;
    if (ok) {
      pair_forward(p, qc, Pm + 12 * v, f);
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
  QuadCommon qc;
  quad_common(p, qc);
  for (int k = k0 + lane; k < k1; k += 32) {
    const int v = pair_v[k];
    if (v < 0 || v >= nv) continue;
    PairFwd f;
    pair_forward(p, qc, Pm + 12 * v, f);
    if (!f.valid) continue;
    l += pair_loss_grad(Pm + 12 * v, p, obs + 4 * (int64_t)k, qc, f, g);
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


// ---------------------------------------------------------------- plain multi-view fit

constexpr int kFitWarps = 4;
constexpr int kAtA = 55;          // upper triangle of the 10 x 10 normal matrix

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix in shared memory (the
// element updates spread over the warp's lanes: lane k owns row / column k).  On return
// the diagonal of A holds the eigenvalues and the columns of V the eigenvectors.
template <typename T>
__device__ void warp_jacobi(int n, T* A, T* V, int lane, int max_sweeps, T tol) {
  for (int k = lane; k < n * n; k += 32) V[k] = (k / n == k % n) ? T(1) : T(0);
  __syncwarp();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0), tot = T(0);
    for (int k = lane; k < n * n; k += 32) {
      const T a = A[k] * A[k];
      tot += a;
      if (k / n != k % n) off += a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xFFFFFFFFu, off, o);
      tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    }
    if (off <= tol * tot || off == T(0)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const T apq = A[p * n + q];
        if (apq == T(0)) continue;  // uniform: every lane reads the same value
        const T th = (A[q * n + q] - A[p * n + p]) / (T(2) * apq);
        const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
        const T c = T(1) / sqrt(t * t + T(1)), sn = t * c;
        __syncwarp();
        if (lane < n) {
          const T akp = A[lane * n + p], akq = A[lane * n + q];
          A[lane * n + p] = c * akp - sn * akq;
          A[lane * n + q] = sn * akp + c * akq;
        }
        __syncwarp();
        if (lane < n) {
          const T apk = A[p * n + lane], aqk = A[q * n + lane];
          A[p * n + lane] = c * apk - sn * aqk;
          A[q * n + lane] = sn * apk + c * aqk;
          const T vkp = V[lane * n + p], vkq = V[lane * n + q];
          V[lane * n + p] = c * vkp - sn * vkq;
          V[lane * n + q] = sn * vkp + c * vkq;
        }
        __syncwarp();
      }
  }
}

// Rotation matrix -> rotation vector through the unit quaternion (Shepperd's branch).
template <typename T>
__device__ void rotmat_to_rotvec(const T R[3][3], T r[3]) {
  const T tr = R[0][0] + R[1][1] + R[2][2];
  T w, x, y, z;
  if (tr > T(0)) {
    const T s = T(2) * sqrt(tr + T(1));
    w = T(0.25) * s; x = (R[2][1] - R[1][2]) / s; y = (R[0][2] - R[2][0]) / s; z = (R[1][0] - R[0][1]) / s;
  } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
    const T s = T(2) * sqrt(T(1) + R[0][0] - R[1][1] - R[2][2]);
    w = (R[2][1] - R[1][2]) / s; x = T(0.25) * s; y = (R[0][1] + R[1][0]) / s; z = (R[0][2] + R[2][0]) / s;
  } else if (R[1][1] > R[2][2]) {
    const T s = T(2) * sqrt(T(1) + R[1][1] - R[0][0] - R[2][2]);
    w = (R[0][2] - R[2][0]) / s; x = (R[0][1] + R[1][0]) / s; y = T(0.25) * s; z = (R[1][2] + R[2][1]) / s;
  } else {
    const T s = T(2) * sqrt(T(1) + R[2][2] - R[0][0] - R[1][1]);
    w = (R[1][0] - R[0][1]) / s; x = (R[0][2] + R[2][0]) / s; y = (R[1][2] + R[2][1]) / s; z = T(0.25) * s;
  }
  if (w < T(0)) { w = -w; x = -x; y = -y; z = -z; }
  const T vn = sqrt(x * x + y * y + z * z);
  const T f = vn > T(1e-30) ? T(2) * atan2(vn, w) / vn : T(2);
  r[0] = f * x; r[1] = f * y; r[2] = f * z;
}

__device__ __forceinline__ float warp_sum(float v);

// Camera centre C = -M^-1 p of P = [M | p] (adjugate over the determinant); false if M is
// singular.
__device__ __forceinline__ bool camera_centre(const float* __restrict__ P, float C[3]) {
  const float a = P[0], b = P[1], c = P[2], d = P[4], e = P[5], f = P[6], g = P[8], h = P[9], i = P[10];
  const float det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
  if (det == 0.f) return false;
  const float p0 = P[3], p1 = P[7], p2 = P[11];
  const float id = 1.f / det;
  C[0] = -((e * i - f * h) * p0 + (c * h - b * i) * p1 + (b * f - c * e) * p2) * id;
  C[1] = -((f * g - d * i) * p0 + (a * i - c * g) * p1 + (c * d - a * f) * p2) * id;
  C[2] = -((d * h - e * g) * p0 + (b * g - a * h) * p1 + (a * e - b * d) * p2) * id;
  return true;
}

// Eq. 1 initialisation of one quadric by one warp, in single precision.  Same reading as
// the library's documentation: planes of the box edges in a frame centred on the views'
// camera centres and scaled to unit mean distance, unit-norm rows, null vector of A^T A,
// Q*44 = -1, eigen-decomposition of Q*[0:3,0:3] + t t^T (descending, >= 1e-6, det R = +1).
// The views are spread over the lanes: each lane accumulates the normal matrix of its own
// views' rows (55 entries), and the lanes' partial matrices are summed through shared
// memory.  sm: 32 x 56 floats of this warp.
__device__ bool warp_quadric_init(int k0, int k1, const float* __restrict__ Pm, const int32_t* __restrict__ pair_v,
                                  const float* __restrict__ obs, int nv, float* sm, int lane, float out[9]) {
  const int nview = k1 - k0;
  float cs[3] = {0.f, 0.f, 0.f};
  bool good = true;
  for (int k = k0 + lane; k < k1; k += 32) {
    const int v = pair_v[k];
    float C[3];
    if (v < 0 || v >= nv || !camera_centre(Pm + 12 * v, C)) { good = false; continue; }
    cs[0] += C[0]; cs[1] += C[1]; cs[2] += C[2];
  }
  good = __all_sync(0xFFFFFFFFu, good);
  if (!good || nview < 3) return false;
  const float inv_n = 1.f / (float)nview;
  const float cx = warp_sum(cs[0]) * inv_n, cy = warp_sum(cs[1]) * inv_n, cz = warp_sum(cs[2]) * inv_n;
  float md = 0.f;
  for (int k = k0 + lane; k < k1; k += 32) {
    float C[3];
    camera_centre(Pm + 12 * pair_v[k], C);
    md += sqrtf((C[0] - cx) * (C[0] - cx) + (C[1] - cy) * (C[1] - cy) + (C[2] - cz) * (C[2] - cz));
  }
  md = warp_sum(md) * inv_n;
  const float sc = md > 0.f ? 1.f / md : 1.f;
  // this lane's views: 4 tangent planes each, normalised, their monomial rows accumulated
  float acc[kAtA];
#pragma unroll
  for (int e = 0; e < kAtA; ++e) acc[e] = 0.f;
  for (int k = k0 + lane; k < k1; k += 32) {
    const float* P = Pm + 12 * pair_v[k];
    const float* bb = obs + 4 * (int64_t)k;
#pragma unroll
    for (int ed = 0; ed < 4; ++ed) {
      // edge lines u = u_min, u = u_max (l = (1, 0, -u)), v = v_min, v = v_max (l = (0, 1, -v))
      const float lb = -bb[ed == 0 ? 0 : ed == 1 ? 2 : ed == 2 ? 1 : 3];
      float pi[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) pi[j] = (ed < 2 ? P[j] : P[4 + j]) + lb * P[8 + j];
      float pn[4] = {pi[0] * md, pi[1] * md, pi[2] * md, pi[0] * cx + pi[1] * cy + pi[2] * cz + pi[3]};
      const float nr = rsqrtf(pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2] + pn[3] * pn[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j) pn[j] *= nr;
      const float row[10] = {pn[0] * pn[0], 2.f * pn[0] * pn[1], 2.f * pn[0] * pn[2], 2.f * pn[0] * pn[3],
                             pn[1] * pn[1], 2.f * pn[1] * pn[2], 2.f * pn[1] * pn[3], pn[2] * pn[2],
                             2.f * pn[2] * pn[3], pn[3] * pn[3]};
      int e = 0;
#pragma unroll
      for (int i = 0; i < 10; ++i)
#pragma unroll
        for (int j = i; j < 10; ++j) acc[e++] += row[i] * row[j];
    }
  }
  // sum the lanes' partial matrices: transpose through shared memory
  float* red = sm;          // [32][56]
#pragma unroll
  for (int e = 0; e < kAtA; ++e) red[lane * 56 + e] = acc[e];
  __syncwarp();
  float tot[2] = {0.f, 0.f};
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int e = lane + 32 * m;
    if (e < kAtA)
      for (int l = 0; l < 32; ++l) tot[m] += red[l * 56 + e];
  }
  __syncwarp();
  float* AtA = sm;          // 100, reusing the reduction area
  float* V = sm + 100;      // 100
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int e = lane + 32 * m;
    if (e < kAtA) {
      int i = 0, r = e;     // upper-triangle index -> (i, j)
      while (r >= 10 - i) { r -= 10 - i; ++i; }
      const int j = i + r;
      AtA[i * 10 + j] = tot[m];
      AtA[j * 10 + i] = tot[m];
    }
  }
  __syncwarp();
  warp_jacobi<float>(10, AtA, V, lane, 20, 1e-13f);
  // smallest eigenvalue's vector
  int kmin = 0;
  for (int k = 1; k < 10; ++k)
    if (AtA[k * 11] < AtA[kmin * 11]) kmin = k;
  float q[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = V[k * 10 + kmin];
  // back to the world frame: Q* = Ti Q' Ti^T, Ti = [[I/sc, c], [0, 1]]
  const float Qn[4][4] = {{q[0], q[1], q[2], q[3]}, {q[1], q[4], q[5], q[6]},
                          {q[2], q[5], q[7], q[8]}, {q[3], q[6], q[8], q[9]}};
  const float Ti[4][4] = {{md, 0.f, 0.f, cx}, {0.f, md, 0.f, cy}, {0.f, 0.f, md, cz}, {0.f, 0.f, 0.f, 1.f}};
  float Q[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float s2 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) s2 += Ti[i][k] * Qn[k][l] * Ti[j][l];
      Q[i][j] = s2;
    }
  (void)sc;
  if (fabsf(Q[3][3]) < 1e-30f) return false;
  const float fs = -1.f / Q[3][3];
  const float t[3] = {-Q[0][3] * fs, -Q[1][3] * fs, -Q[2][3] * fs};
  float* M = sm + 200;      // 9 entries + 9 eigenvectors
  float* E = sm + 216;
  __syncwarp();
  if (lane < 9) M[lane] = Q[lane / 3][lane % 3] * fs + t[lane / 3] * t[lane % 3];
  __syncwarp();
  warp_jacobi<float>(3, M, E, lane, 20, 1e-13f);
  int ord[3] = {0, 1, 2};
  if (M[4 * ord[1]] > M[4 * ord[0]]) { const int x = ord[0]; ord[0] = ord[1]; ord[1] = x; }
  if (M[4 * ord[2]] > M[4 * ord[1]]) { const int x = ord[1]; ord[1] = ord[2]; ord[2] = x; }
  if (M[4 * ord[1]] > M[4 * ord[0]]) { const int x = ord[0]; ord[0] = ord[1]; ord[1] = x; }
  float R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) R[i][k] = E[3 * i + ord[k]];
  const float dR = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) - R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                   R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
  if (dR < 0.f)
#pragma unroll
    for (int i = 0; i < 3; ++i) R[i][2] = -R[i][2];
  float rv[3];
  rotmat_to_rotvec<float>(R, rv);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out[k] = t[k];
    out[3 + k] = 0.5f * logf(fmaxf(M[4 * ord[k]], 1e-6f));
    out[6 + k] = rv[k];
  }
  __syncwarp();
  return true;
}

// Warp sum of 16 values per lane in 16 shuffles (a transposing reduction): each stage
// keeps half of the values and sends the other half to the partner lane.  Lane L returns
// the total of value (L >> 1) & 15 (lanes 2v and 2v + 1 hold value v).
__device__ __forceinline__ float warp_transpose_sum16(const float (&v)[16], int lane) {
  float a8[8];
  const bool b4 = lane & 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float keep = b4 ? v[i + 8] : v[i], send = b4 ? v[i] : v[i + 8];
    a8[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
  }
  float a4[4];
  const bool b3 = lane & 8;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b3 ? a8[i + 4] : a8[i], send = b3 ? a8[i] : a8[i + 4];
    a4[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
  }
  float a2[2];
  const bool b2 = lane & 4;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b2 ? a4[i + 2] : a4[i], send = b2 ? a4[i] : a4[i + 2];
    a2[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
  }
  const bool b1 = lane & 2;
  const float a1 = (b1 ? a2[1] : a2[0]) + __shfl_xor_sync(0xFFFFFFFFu, b1 ? a2[0] : a2[1], 2);
  return a1 + __shfl_xor_sync(0xFFFFFFFFu, a1, 1);
}

__global__ void __launch_bounds__(32 * kFitWarps) k_quadric_fit(int nq, int nv, const float* __restrict__ Pm,
                                                                  const int32_t* __restrict__ q_ptr,
                                                                  const int32_t* __restrict__ pair_v, int npairs,
                                                                  const float* __restrict__ obs, int iters, float lr,
                                                                  const float* __restrict__ start,
                                                                  float* __restrict__ init_out,
                                                                  float* __restrict__ params_out,
                                                                  float* __restrict__ loss_out,
                                                                  uint8_t* __restrict__ ok_out) {
  __shared__ float sm[kFitWarps][32 * 56];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * kFitWarps + w;
  if (q >= nq) return;
  const int k0 = max(q_ptr[q], 0), k1 = min(q_ptr[q + 1], npairs);
  float p[9];
  bool good;
  if (start) {  // refine from the given parameters instead of the Eq. 1 initialisation
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = start[9 * q + k];
    good = k1 > k0;
  } else {
    good = warp_quadric_init(k0, k1, Pm, pair_v, obs, nv, sm[w], lane, p);
  }
  if (lane == 0 && ok_out) ok_out[q] = good ? 1 : 0;
  if (!good) {
    if (lane < 9) {
      if (init_out) init_out[9 * q + lane] = 0.f;
      if (params_out) params_out[9 * q + lane] = 0.f;
    }
    if (lane == 0 && loss_out) loss_out[q] = 0.f;
    return;
  }
  if (init_out && lane < 9) init_out[9 * q + lane] = p[lane];
  // Refinement: Adam on the Eq. 12 loss.  Every lane evaluates its views with all nine
  // parameters; after the transposing reduction lanes 2k and 2k + 1 hold the gradient of
  // parameter k (k < 9; lanes 18, 19 the loss) and run that parameter's Adam update, and
  // the nine new values are broadcast back.
  const int mine = (lane >> 1) & 15;
  float pm = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (mine == k) pm = p[k];
  float m1 = 0.f, m2 = 0.f;
  float b1t = 1.f, b2t = 1.f, L = 0.f;
  for (int it = 0; it <= iters; ++it) {
    QuadCommon qc;
    quad_common(p, qc);
    float g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = 0.f;
    for (int k = k0 + lane; k < k1; k += 32) {
      const int vw = pair_v[k];
      PairFwd f;
      pair_forward(p, qc, Pm + 12 * vw, f);
      if (!f.valid) continue;
      g[9] += pair_loss_grad(Pm + 12 * vw, p, obs + 4 * (int64_t)k, qc, f, g);
    }
    const float tot = warp_transpose_sum16(g, lane);
    if (it == iters) {  // the last pass only evaluates the final loss
      L = __shfl_sync(0xFFFFFFFFu, tot, 18);
      break;
    }
    b1t *= 0.9f;
    b2t *= 0.999f;
    m1 = 0.9f * m1 + 0.1f * tot;
    m2 = 0.999f * m2 + 0.001f * tot * tot;
    const float mh = m1 / (1.f - b1t), vh = m2 / (1.f - b2t);
    pm -= lr * mh / (sqrtf(vh) + 1e-8f);
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = __shfl_sync(0xFFFFFFFFu, pm, 2 * k);
  }
  if (params_out && lane < 9) params_out[9 * q + lane] = p[lane];
  if (lane == 0 && loss_out) loss_out[q] = L;
}

// Canonical parameters of a quadric (the learned proposal's regression target): the same
// ellipsoid with its semi-axes in descending order (ties kept in index order), the
// rotation's columns permuted with them and the third negated if that makes det < 0, and,
// of the four rotations that differ by negating two columns (all describe the same
// ellipsoid), the one of largest trace (first in the order identity, flip axes 2-3,
// flip 1-3, flip 1-2 on ties).  Centre unchanged.
__global__ void k_quadric_canonical(int nq, const float* __restrict__ in, float* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double p[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) p[k] = in[9 * q + k];
  // rotation vector -> matrix, R = I + A K + B K^2
  const double th2 = p[6] * p[6] + p[7] * p[7] + p[8] * p[8];
  const double th = sqrt(th2);
  double A, B;
  if (th < 1e-4) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
  }
  const double Kx[3][3] = {{0.0, -p[8], p[7]}, {p[8], 0.0, -p[6]}, {-p[7], p[6], 0.0}};
  double R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double k2 = Kx[i][0] * Kx[0][j] + Kx[i][1] * Kx[1][j] + Kx[i][2] * Kx[2][j];
      R[i][j] = (i == j ? 1.0 : 0.0) + A * Kx[i][j] + B * k2;
    }
  int ord[3] = {0, 1, 2};
  const double* la = p + 3;
  if (la[ord[1]] > la[ord[0]]) { const int x = ord[0]; ord[0] = ord[1]; ord[1] = x; }
  if (la[ord[2]] > la[ord[1]]) { const int x = ord[1]; ord[1] = ord[2]; ord[2] = x; }
  if (la[ord[1]] > la[ord[0]]) { const int x = ord[0]; ord[0] = ord[1]; ord[1] = x; }
  double Rs[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) Rs[i][k] = R[i][ord[k]];
  const double det = Rs[0][0] * (Rs[1][1] * Rs[2][2] - Rs[1][2] * Rs[2][1]) -
                     Rs[0][1] * (Rs[1][0] * Rs[2][2] - Rs[1][2] * Rs[2][0]) +
                     Rs[0][2] * (Rs[1][0] * Rs[2][1] - Rs[1][1] * Rs[2][0]);
  if (det < 0.0)
#pragma unroll
    for (int i = 0; i < 3; ++i) Rs[i][2] = -Rs[i][2];
  const double sg[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  int best = 0;
  double bt = Rs[0][0] + Rs[1][1] + Rs[2][2];
  for (int c = 1; c < 4; ++c) {
    const double tr = sg[c][0] * Rs[0][0] + sg[c][1] * Rs[1][1] + sg[c][2] * Rs[2][2];
    if (tr > bt) { bt = tr; best = c; }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) Rs[i][k] *= sg[best][k];
  double rv[3];
  rotmat_to_rotvec<double>(Rs, rv);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out[9 * q + k] = (float)p[k];
    out[9 * q + 3 + k] = (float)la[ord[k]];
    out[9 * q + 6 + k] = (float)rv[k];
  }
}

}  // namespace

cudaError_t launch_quadric_fit(int nq, int nv, const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                               int npairs, const float* obs, int iters, float lr, const float* start, float* init,
                               float* params, float* loss, uint8_t* ok, cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nq + kFitWarps - 1) / kFitWarps);
  k_quadric_fit<<<blocks, 32 * kFitWarps, 0, s>>>(nq, nv, P, q_ptr, pair_v, npairs, obs, iters, lr, start, init,
                                                 params, loss, ok);
  return cudaGetLastError();
}

cudaError_t launch_quadric_canonical(int nq, const float* in, float* out, cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  k_quadric_canonical<<<(unsigned)((nq + 127) / 128), 128, 0, s>>>(nq, in, out);
  return cudaGetLastError();
}

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
