// K6 (blend forward + fused losses) and K7 (blend backward) of the rasterizer.
//
// Forward: one CTA of 256 threads per screen tile (16x16, 8x32 or 32x8 pixels); backward:
// one CTA of 128 threads per half tile.  One pixel per thread; each warp covers an 8x4
// pixel block and walks the tile's depth-ordered Gaussian list in chunks of 32, staging
// in shared memory the Gaussians that can reach its block.  Tiles (and backward half
// tiles) are taken heaviest first, in the order a one-CTA counting sort writes.
//
// Forward, per pixel, front to back (3DGS blending; Eq. 15 for ins; Eq. 7-10 losses):
//   alpha = min(clamp, o G), skipped if < alpha_min; stop before T (1 - alpha) < t_stop;
//   w = alpha T: C += w c, D += w z, ins += w if the Gaussian is opaque (or og_filter is
//   off) and its id equals the pixel's labelled id; W_k += w for the id map.
// Each warp walks the list on its own (no barrier inside the walk) and leaves it once
// all its pixels have stopped.  Per-object weights live in shared memory per tile: the tile's distinct ids are found first and mapped to dense
// slots, 16 slots per round (extra rounds re-walk the list only for tiles with more
// than 16 objects).  The loss terms and dL/d(pixel) are computed in the epilogue.
//
// Backward, per pixel, back to front from T_final and n_contrib: T_j = T_{j+1}/(1-a_j),
// dL/da_j = T_j U_j - R_j / (1 - a_j) with U_j = dC.c_j + dD z_j + dA + dins [j counts]
// and R_j = sum_{k>j} w_k U_k + T_final dC.bg.  The ten per-Gaussian partials are
// summed over the warp by a transposing reduction (12 shuffles) and added to the global
// per-Gaussian record with vector atomics once per (warp, Gaussian); when at most sixteen
// lanes contribute, each adds its own partials instead.
#include "dqo_internal.cuh"

namespace dqo {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kOgOut = 1u << 30;          // staged key bit: excluded from ins by the OG filter
constexpr uint32_t kSlotMask = kOgOut - 1u;    // staged key bits holding the dense slot
constexpr int kFwdIlp = 2;                     // Gaussians evaluated together in the forward walk
static_assert(32 % kFwdIlp == 0, "staging holds 32 slots");

// eval_gaussian without branches: the same operations, the skip decision returned
// instead of taken (outputs are defined either way).
__device__ __forceinline__ bool eval_terms(const float4& p0, const float4& p1, float px, float py, float alpha_clamp,
                                           float alpha_min, float& alpha, float& G, float& dx, float& dy) {
  dx = __fsub_rn(px, p0.x);
  dy = __fsub_rn(py, p0.y);
  const float t = __fmaf_rn(p0.w, dy, __fmul_rn(p0.z, dx));
  const float pw = __fmaf_rn(__fmul_rn(p1.x, dy), dy, __fmul_rn(t, dx));
  G = ex2_approx(pw);
  alpha = fminf(alpha_clamp, __fmul_rn(p1.y, G));
  return !(pw > 0.f) && alpha >= alpha_min;
}

// alpha of a Gaussian at pixel (px, py), without branches: the same operations as
// eval_gaussian, with the skip decision returned instead of taken.
__device__ __forceinline__ bool eval_alpha(const float4& p0, const float4& p1, float px, float py,
                                           float alpha_clamp, float alpha_min, float& alpha) {
  const float dx = __fsub_rn(px, p0.x);
  const float dy = __fsub_rn(py, p0.y);
  const float t = __fmaf_rn(p0.w, dy, __fmul_rn(p0.z, dx));
  const float pw = __fmaf_rn(__fmul_rn(p1.x, dy), dy, __fmul_rn(t, dx));
  alpha = fminf(alpha_clamp, __fmul_rn(p1.y, ex2_approx(pw)));
  return !(pw > 0.f) && alpha >= alpha_min;
}

template <int TW>
__device__ __forceinline__ void pixel_of(int tile_x0, int tile_y0, int& px, int& py, float& wx0, float& wy0,
                                         int warp = threadIdx.x >> 5) {
  constexpr int WX = TW / 8;
  const int lane = threadIdx.x & 31;
  const int bx = tile_x0 + (warp % WX) * 8, by = tile_y0 + (warp / WX) * 4;
  px = bx + (lane & 7);
  py = by + (lane >> 3);
  wx0 = (float)bx;
  wy0 = (float)by;
}

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// Can the Gaussian reach alpha_min at some pixel centre of the block [bx, bx + bw] x
// [by, by + bh]?  f(d) = -(a' dx^2 + b' dx dy + c' dy^2) is a convex quadratic of d = p - mean;
// its minimum over the rectangle is 0 if the mean lies inside, else the least of the
// four edge minima (each a clamped 1D minimum).  Hit iff that minimum <= the level in p2.w.
__device__ __forceinline__ bool ellipse_hits(const float4& p0, const float4& p1, const float4& p2, float bx,
                                             float by, float bw, float bh) {
  const float lvl = p2.w;
  if (!(lvl >= 0.f)) return false;
  const float A = -p0.z, B = -p0.w, C = -p1.x;
  const float X0 = bx - p0.x, X1 = X0 + bw, Y0 = by - p0.y, Y1 = Y0 + bh;
  if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return true;
  const float hA = 0.5f / A, hC = 0.5f / C;
  float m;
  {
    const float y = fminf(fmaxf(-B * X0 * hC, Y0), Y1);
    m = (A * X0 + B * y) * X0 + C * y * y;
  }
  {
    const float y = fminf(fmaxf(-B * X1 * hC, Y0), Y1);
    m = fminf(m, (A * X1 + B * y) * X1 + C * y * y);
  }
  {
    const float x = fminf(fmaxf(-B * Y0 * hA, X0), X1);
    m = fminf(m, (A * x + B * Y0) * x + C * Y0 * Y0);
  }
  {
    const float x = fminf(fmaxf(-B * Y1 * hA, X0), X1);
    m = fminf(m, (A * x + B * Y1) * x + C * Y1 * Y1);
  }
  return m <= lvl;
}

// Word of the hit record for the warp-block `wblock` of tile `tile` and the list chunk
// starting at position c of the tile's list [start, ..): the forward stores there the
// ballot of which chunk entries can reach the block, the backward reads it instead of
// testing again.  Words (floor(start / 32) + tile + chunk) * 8 + wblock never collide
// between tiles (a tile's chunks number at most floor(length / 32) + 1), so a record of
// 8 * (pairs / 32 + tiles + 1) words holds all.
__device__ __forceinline__ int64_t hit_word(int start, int c, int tile, int wblock) {
  return ((int64_t)(start >> 5) + tile + ((c - start) >> 5)) * 8 + wblock;
}

// Fills s_slot_id[s - first] with the object id of dense slot s for s in [first, first+kIdSlots).
__device__ __forceinline__ void slot_ids_for_round(const uint32_t* s_mask, const uint32_t* s_pref, int nw, int first,
                                                   int32_t* s_slot_id) {
  for (int t = threadIdx.x; t < nw; t += kThreads) {
    uint32_t m = s_mask[t];
    int s = (int)s_pref[t];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      if (s >= first && s < first + kIdSlots) s_slot_id[s - first] = t * 32 + b;
      ++s;
    }
  }
}

// Forward of one tile (tile index local to a's image).  Called by all threads of a
// block; uses the block's shared memory and barriers.
template <int TW, bool kId>
__device__ __forceinline__ void blend_fwd_tile(const BlendFwdArgs& a, const BlendCommon& cm, const int tile) {
  constexpr int NW = kThreads / 32;
  // per-warp staging of the Gaussians that can reach the warp's pixels
  __shared__ float4 s_q0[NW][32], s_q1[NW][32], s_q2[NW][32];
  __shared__ uint32_t s_mask[kId ? kMaskWords : 1], s_pref[kId ? kMaskWords : 1];
  __shared__ int32_t s_slot_id[kIdSlots];
  __shared__ float s_W[kId ? kIdSlots : 1][kThreads];
  __shared__ float s_red[3][kThreads / 32];
  __shared__ uint32_t s_wlast[kThreads / 32];
  __shared__ uint32_t s_nslots;

  const RasterParams& rp = a.rp;
  const int tx = tile % rp.ntx, ty = tile / rp.ntx;
  int px, py;
  float wx0, wy0;
  pixel_of<TW>(tx * rp.tile_w, ty * rp.tile_h, px, py, wx0, wy0);
  const bool inside = px < rp.W && py < rp.H;
  const int64_t pix = (int64_t)py * rp.W + px;
  const uint2 rg = a.ranges[tile];
  const int start = (int)rg.x, end = rg.y > rg.x ? (int)rg.y : (int)rg.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  int32_t gt = -1;
  if (inside && a.t_gt) gt = a.t_gt[pix];
  const uint32_t gt_match = (gt >= 0 && gt < rp.num_objects) ? (uint32_t)gt : 0xFFFFFFFEu;

  // ---- distinct object ids of this tile -> dense slots (ascending id order)
  int nslots = 0;
  const int nw = (rp.num_objects + 31) >> 5;
  if (kId) {
    for (int t = tid; t < nw; t += kThreads) s_mask[t] = 0u;
    __syncthreads();
    // four list entries per thread with their loads in flight; a warp whose ids all fall
    // in one mask word ORs them together and adds them with one atomic
    constexpr int kPre = 4;
    for (int b = start; b < end; b += kPre * kThreads) {  // uniform trip count: warp intrinsics below
      uint32_t id[kPre];
#pragma unroll
      for (int j = 0; j < kPre; ++j) {
        const int i = b + j * kThreads + tid;
        id[j] = i < end ? cm.list[i] : 0xFFFFFFFFu;
      }
#pragma unroll
      for (int j = 0; j < kPre; ++j) id[j] = id[j] != 0xFFFFFFFFu ? cm.gid[id[j]] : 0xFFFFFFFFu;
#pragma unroll
      for (int j = 0; j < kPre; ++j) {
        const bool has = id[j] != 0xFFFFFFFFu;
        const uint32_t word = has ? id[j] >> 5 : 0u, bit = has ? 1u << (id[j] & 31) : 0u;
        int same;
        __match_all_sync(kFull, word, &same);
        if (same) {
          const uint32_t m = __reduce_or_sync(kFull, bit);
          if (lane == 0 && m) atomicOr(&s_mask[word], m);
        } else if (has) {
          atomicOr(&s_mask[word], bit);
        }
      }
    }
    __syncthreads();
    if (tid < 32) {
      uint32_t carry = 0;
      for (int c = 0; c < nw; c += 32) {
        const int t = c + tid;
        const uint32_t pc = t < nw ? (uint32_t)__popc(s_mask[t]) : 0u;
        uint32_t inc = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (tid >= o) inc += u;
        }
        if (t < nw) s_pref[t] = carry + inc - pc;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
      }
      if (tid == 0) s_nslots = carry;
    }
    __syncthreads();
    nslots = (int)s_nslots;
    slot_ids_for_round(s_mask, s_pref, nw, 0, s_slot_id);
#pragma unroll
    for (int s = 0; s < kIdSlots; ++s) s_W[s][tid] = 0.f;
    __syncthreads();  // round 0's slot ids are published before the walk, not after it
  }

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, ins = 0.f;
  int last = 0;
  bool done = !inside;
  const float fpx = (float)px, fpy = (float)py;
  const uint32_t lt = lanemask_lt();

  // Dense slot of an object id in this tile's ascending-id slot map (-1: no object).
  auto slot_of = [&](uint32_t idbits) -> int {
    const uint32_t id = idbits & kNoObject;
    if (id == kNoObject) return -1;
    return (int)(s_pref[id >> 5] + __popc(s_mask[id >> 5] & ((1u << (id & 31)) - 1u)));
  };
  // Staged key of a Gaussian (replaces q1.w): with the id map, its dense slot, with bit 30
  // set when the OG filter excludes it from ins, all ones without an object; without the
  // id map, its object id, or all ones when the OG filter excludes it.  ins counts a
  // Gaussian iff its key equals the pixel's key gt_key.
  auto key_of = [&](uint32_t idog) -> uint32_t {
    const bool og_out = cm.og_filter && !(idog >> 31);
    if (kId) {
      const int sl = slot_of(idog);
      return sl < 0 ? 0xFFFFFFFFu : ((uint32_t)sl | (og_out ? kOgOut : 0u));
    }
    return og_out ? 0xFFFFFFFFu : (idog & kNoObject);
  };
  uint32_t gt_key = gt_match;
  if (kId && gt_match != 0xFFFFFFFEu)
    gt_key = (s_mask[gt_match >> 5] >> (gt_match & 31)) & 1u ? (uint32_t)slot_of(gt_match) : 0xFFFFFFFEu;
  uint32_t cur_key = 0xFFFFFFFFu;
  float cur_w = 0.f;
  // Stages, in list order, the Gaussians of list chunk [c, c+32) that can reach this warp's
  // pixels and sit before list position `lim`; returns how many.  q1.w holds the key and
  // q2.w the list position (both consumed at staging otherwise).
  // gi: list entry c + lane, already loaded by the caller (read only below lim).
  auto stage = [&](int c, int lim, uint32_t gi, bool record) -> int {
    const int i = c + lane;
    bool hit = false;
    float4 q0, q1, q2;
    if (i < lim) {
      const uint32_t g = gi;
      q0 = cm.p0[g];
      q1 = cm.p1[g];
      q2 = cm.p2[g];
      hit = ellipse_hits(q0, q1, q2, wx0, wy0, 7.f, 3.f);
    }
    const uint32_t m = __ballot_sync(kFull, hit);
    if (record && a.hitmask && lane == 0) a.hitmask[hit_word(start, c, tile, warp)] = m;
    if (hit) {
      const int k = __popc(m & lt);
      q1.w = __uint_as_float(key_of(__float_as_uint(q1.w)));
      q2.w = __int_as_float(i - start);
      s_q0[warp][k] = q0;
      s_q1[warp][k] = q1;
      s_q2[warp][k] = q2;
    }
    __syncwarp();
    return __popc(m);
  };
  // Blends one evaluated Gaussian into the pixel (front to back).
  auto blend = [&](float alpha, float z, uint32_t key, int h) {
    const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
    if (Tn < cm.t_stop) {
      done = true;
      return;
    }
    const float w = __fmul_rn(alpha, T);
    const float4 q2 = s_q2[warp][h];
    C0 = fmaf(w, q2.x, C0);
    C1 = fmaf(w, q2.y, C1);
    C2 = fmaf(w, q2.z, C2);
    D = fmaf(w, z, D);
    if (key == gt_key) ins += w;
    if (kId) {
      if (key == cur_key) {
        cur_w += w;
      } else {
        const uint32_t sl = cur_key & kSlotMask;
        if (sl < (uint32_t)kIdSlots) s_W[sl][tid] += cur_w;
        cur_key = key;
        cur_w = w;
      }
    }
    T = Tn;
    last = __float_as_int(q2.w) + 1;
  };

  // ---- front to back, each warp on its own: no block-wide barrier inside the walk.  kFwdIlp
  // staged Gaussians per iteration: their exponentials are independent, only the blending
  // is sequential.
  // the next chunk's list entries are loaded while the current chunk is blended
  uint32_t gnext = start + lane < end ? cm.list[start + lane] : 0u;
  for (int c = start; c < end; c += 32) {
    if (__all_sync(kFull, done)) break;
    const int nh = stage(c, end, gnext, true);
    if (c + 32 + lane < end) gnext = cm.list[c + 32 + lane];
    for (int h = 0; h < nh; h += kFwdIlp) {
      if (done) continue;
      // slots h .. h + kFwdIlp - 1 <= 31 are inside the staging arrays even past nh
      // (stale data, masked)
      float al[kFwdIlp], z[kFwdIlp];
      uint32_t key[kFwdIlp];
      bool v[kFwdIlp];
#pragma unroll
      for (int u = 0; u < kFwdIlp; ++u) {
        const float4 q0 = s_q0[warp][h + u], q1 = s_q1[warp][h + u];
        v[u] = eval_alpha(q0, q1, fpx, fpy, cm.alpha_clamp, cm.alpha_min, al[u]) && h + u < nh;
        z[u] = q1.z;
        key[u] = __float_as_uint(q1.w);
      }
#pragma unroll
      for (int u = 0; u < kFwdIlp; ++u)
        if (v[u] && !done) blend(al[u], z[u], key[u], h + u);
    }
    __syncwarp();
  }

  // ---- object-id argmax (ties to the smaller id: slots are in ascending id order)
  int32_t best_id = -1;
  if (kId) {
    if ((cur_key & kSlotMask) < (uint32_t)kIdSlots) s_W[cur_key & kSlotMask][tid] += cur_w;
    float best_w = 0.f;
    const int n0 = min(nslots, kIdSlots);
    for (int s = 0; s < n0; ++s) {
      const float v = s_W[s][tid];
      if (v > best_w) {
        best_w = v;
        best_id = s_slot_id[s];
      }
    }
    // tiles with more than kIdSlots objects: re-walk the blended prefix once per extra round
    if (nslots > kIdSlots) {
      const int wlast = (int)__reduce_max_sync(kFull, (uint32_t)last);
      for (int first = kIdSlots; first < nslots; first += kIdSlots) {
        __syncthreads();
        slot_ids_for_round(s_mask, s_pref, nw, first, s_slot_id);
#pragma unroll
        for (int s = 0; s < kIdSlots; ++s) s_W[s][tid] = 0.f;
        __syncthreads();
        float Tr = 1.f;
        for (int c = start; c < start + wlast; c += 32) {
          const int nh = stage(c, start + wlast, c + lane < start + wlast ? cm.list[c + lane] : 0u, false);
          for (int h = 0; h < nh; ++h) {
            if (__float_as_int(s_q2[warp][h].w) >= last) continue;
            float alpha, G, dx, dy;
            if (!eval_gaussian(s_q0[warp][h], s_q1[warp][h], fpx, fpy, cm.alpha_clamp, cm.alpha_min, alpha, G,
                               dx, dy))
              continue;
            const float w = __fmul_rn(alpha, Tr);
            Tr = __fmul_rn(Tr, __fsub_rn(1.f, alpha));
            const int s = (int)(__float_as_uint(s_q1[warp][h].w) & kSlotMask) - first;
            if (s >= 0 && s < kIdSlots) s_W[s][tid] += w;
          }
          __syncwarp();
        }
        const int nr = min(nslots - first, kIdSlots);
        for (int s = 0; s < nr; ++s) {
          const float v = s_W[s][tid];
          if (v > best_w) {
            best_w = v;
            best_id = s_slot_id[s];
          }
        }
      }
    }
  }

  // ---- outputs and fused losses
  float l_rgb = 0.f, l_d = 0.f, l_i = 0.f;
  if (inside) {
    const float c0 = fmaf(T, rp.bg[0], C0), c1 = fmaf(T, rp.bg[1], C1), c2 = fmaf(T, rp.bg[2], C2);
    if (a.o_rgb) {
      a.o_rgb[3 * pix + 0] = c0;
      a.o_rgb[3 * pix + 1] = c1;
      a.o_rgb[3 * pix + 2] = c2;
    }
    if (a.o_depth) a.o_depth[pix] = D;
    if (a.o_alpha) a.o_alpha[pix] = 1.f - T;
    if (a.o_ins) a.o_ins[pix] = ins;
    if (a.o_id) a.o_id[pix] = best_id;
    a.T_final[pix] = T;
    a.n_contrib[pix] = (uint32_t)last;
    if (a.t_gt) {
      const float inv_hw = 1.f / ((float)rp.W * (float)rp.H);
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, gd = 0.f, gi = 0.f;
      if (gt >= 0) {
        const float e0 = c0 - a.t_rgb[3 * pix + 0], e1 = c1 - a.t_rgb[3 * pix + 1], e2 = c2 - a.t_rgb[3 * pix + 2];
        l_rgb = fabsf(e0) + fabsf(e1) + fabsf(e2);
        g0 = sgnf(e0) * inv_hw;
        g1 = sgnf(e1) * inv_hw;
        g2 = sgnf(e2) * inv_hw;
        const float td = a.t_depth ? a.t_depth[pix] : 0.f;
        if (td > 0.f) {
          const float ed = D - td;
          l_d = fabsf(ed);
          gd = sgnf(ed) * inv_hw;
        }
        const float ei = ins - 1.f;
        l_i = fabsf(ei);
        gi = rp.lambda_ins * sgnf(ei) * inv_hw;
        if (a.o_mask) {
          // Eq. 11: Mask_geo (bit0) and Mask_rgb (bit1)
          const bool geo = ins < rp.theta_alpha || (td > 0.f && fabsf(D - td) > rp.theta_d);
          const bool col = fmaxf(fabsf(e0), fmaxf(fabsf(e1), fabsf(e2))) > rp.theta_c;
          a.o_mask[pix] = (uint8_t)((geo ? 1 : 0) | (col ? 2 : 0));
        }
      } else if (a.o_mask) {
        a.o_mask[pix] = 0;
      }
      a.dl_rgb[3 * pix + 0] = g0;
      a.dl_rgb[3 * pix + 1] = g1;
      a.dl_rgb[3 * pix + 2] = g2;
      a.dl_depth[pix] = gd;
      a.dl_ins[pix] = gi;
    }
  }
  if (a.t_gt) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l_rgb += __shfl_xor_sync(0xFFFFFFFFu, l_rgb, o);
      l_d += __shfl_xor_sync(0xFFFFFFFFu, l_d, o);
      l_i += __shfl_xor_sync(0xFFFFFFFFu, l_i, o);
    }
    if (lane == 0) {
      s_red[0][warp] = l_rgb;
      s_red[1][warp] = l_d;
      s_red[2][warp] = l_i;
    }
  }
  // the tile's backward cost: its longest blended prefix
  const uint32_t wlast = __reduce_max_sync(kFull, (uint32_t)last);
  if (lane == 0) s_wlast[warp] = wlast;
  if (a.t_gt || a.tile_cost) {
    __syncthreads();
    if (a.t_gt && tid < 3) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) s += s_red[tid][w];
      a.loss_part[3 * tile + tid] = s;
    }
    if (a.tile_cost && tid >= 32 && tid < 32 + kTileParts) {  // each part's longest prefix
      constexpr int kPartWarps = kThreads / 32 / kTileParts;
      const int p = tid - 32;
      uint32_t m = 0;
#pragma unroll
      for (int w = 0; w < kPartWarps; ++w) m = max(m, s_wlast[p * kPartWarps + w]);
      a.tile_cost[tile * kTileParts + p] = m;
    }
  }
}

template <int TW, bool kId>
__global__ void __launch_bounds__(kThreads) k_blend_forward(BlendFwdArgs a) {
  pdl_wait();
  pdl_trigger();
  const BlendCommon cm{a.p0, a.p1, a.p2, a.gid, a.list, nullptr, a.rp.alpha_clamp, a.rp.alpha_min, a.rp.t_stop,
                       a.rp.og_filter};
  blend_fwd_tile<TW, kId>(a, cm, a.tile_order ? (int)a.tile_order[blockIdx.x] : (int)blockIdx.x);
}

__global__ void k_loss_reduce(const float* __restrict__ part, int tiles, float lambda_ins, float scale,
                              float* __restrict__ loss) {
  pdl_wait();
  pdl_trigger();
  loss_reduce(part, tiles, lambda_ins, scale, loss);
}

// ---------------------------------------------------------------- tile schedule
// Tiles differ in cost by orders of magnitude (empty sky against cluttered objects), and a
// tile's CTA lives as long as its slowest warp: launched in raster order, the last wave is
// a few heavy tiles on otherwise idle SMs.  The blend kernels therefore take their tiles
// heaviest first (the hardware hands out CTAs roughly in block order): the forward by
// list length, the backward by the forward's longest blended prefix per tile.
constexpr int kSchedBuckets = 128;

// Bucket of a cost on a log scale, four buckets per octave (0 for cost 0).
__device__ __forceinline__ int sched_bucket(uint32_t x) {
  if (x == 0u) return 0;
  const int lz = 31 - __clz(x);
  const uint32_t frac = lz >= 2 ? (x >> (lz - 2)) & 3u : (x << (2 - lz)) & 3u;
  return min(kSchedBuckets - 1, lz * 4 + (int)frac + 1);
}

// One CTA of kSchedThreads: counting sort of the tiles by decreasing bucket.  Each round
// takes kSchedThreads * kSchedPer tiles with all their cost loads in flight; counts and
// placements are shared-memory atomics per tile (one SM runs the whole schedule, where a
// warp match per tile measured slower), so the order of tiles within a bucket is that of
// the atomics: the schedule is a heuristic and the results do not depend on it.
constexpr int kSchedThreads = 1024, kSchedPer = 8;

// Item i's cost: tile i's list length (ranges), else the largest of cost[i * group + j],
// j < group (a tile's parts, or one part).
__device__ __forceinline__ void schedule_tiles(const uint2* __restrict__ ranges, const uint32_t* __restrict__ cost,
                                               int group, int tiles, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_h[kSchedBuckets];
  const int tid = threadIdx.x, lane = tid & 31;
  auto buckets = [&](int base, int (&b)[kSchedPer]) {
    uint32_t c[kSchedPer];
#pragma unroll
    for (int j = 0; j < kSchedPer; ++j) {
      const int t = base + j * kSchedThreads + tid;
      c[j] = 0u;
      if (t < tiles) {
        if (cost) {
          for (int g = 0; g < group; ++g) c[j] = max(c[j], cost[(int64_t)t * group + g]);
        } else {
          const uint2 r = ranges[t];
          c[j] = r.y > r.x ? r.y - r.x : 0u;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kSchedPer; ++j) b[j] = base + j * kSchedThreads + tid < tiles ? sched_bucket(c[j]) : -1;
  };
  for (int b = tid; b < kSchedBuckets; b += kSchedThreads) s_h[b] = 0u;
  __syncthreads();
  // one round holds up to kSchedThreads * kSchedPer tiles: its buckets stay in registers for
  // the placement below instead of being loaded again
  const bool one_round = tiles <= kSchedThreads * kSchedPer;
  int held[kSchedPer];
  for (int base = 0; base < tiles; base += kSchedThreads * kSchedPer) {
    int b[kSchedPer];
    buckets(base, b);
#pragma unroll
    for (int j = 0; j < kSchedPer; ++j) {
      held[j] = b[j];
      if (b[j] >= 0) atomicAdd(&s_h[b[j]], 1u);
    }
  }
  __syncthreads();
  if (tid < 32) {
    // exclusive scan in decreasing bucket order: lane l owns buckets 127-4l .. 124-4l
    constexpr int kPer = kSchedBuckets / 32;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      v[j] = s_h[kSchedBuckets - 1 - (lane * kPer + j)];
      sum += v[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += u;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      s_h[kSchedBuckets - 1 - (lane * kPer + j)] = run;
      run += v[j];
    }
  }
  __syncthreads();
  for (int base = 0; base < tiles; base += kSchedThreads * kSchedPer) {
    int b[kSchedPer];
    if (one_round) {
#pragma unroll
      for (int j = 0; j < kSchedPer; ++j) b[j] = held[j];
    } else {
      buckets(base, b);
    }
#pragma unroll
    for (int j = 0; j < kSchedPer; ++j)
      if (b[j] >= 0) order[atomicAdd(&s_h[b[j]], 1u)] = (uint32_t)(base + j * kSchedThreads + tid);
  }
}

// Tile ranges of the joint tiles [first, first + tiles) from the pair counts of all joint
// tiles: ranges[t] = [base + e_t, base + e_t + counts[first + t]), e_t the exclusive prefix
// of the slice's counts and base the pairs of the tiles before it.  One CTA of
// kSchedThreads; ends with a barrier.
__device__ __forceinline__ void ranges_from_counts(const uint32_t* __restrict__ counts, uint32_t first, int tiles,
                                                   uint2* __restrict__ ranges) {
  __shared__ uint32_t s_w[kSchedThreads / 32];
  __shared__ uint32_t s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // base: sum of the counts before the slice
  uint32_t b = 0;
#pragma unroll 4
  for (uint32_t i = tid; i < first; i += kSchedThreads) b += counts[i];
  b = __reduce_add_sync(kFull, b);
  if (lane == 0) s_w[warp] = b;
  __syncthreads();
  if (tid == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSchedThreads / 32; ++w) t += s_w[w];
    s_base = t;
  }
  __syncthreads();
  // thread tid owns the contiguous chunk [tid * per, (tid + 1) * per) of the slice; chunks of
  // up to kHeld counts are loaded once, together, and kept in registers
  constexpr int kHeld = 8;
  const int per = (tiles + kSchedThreads - 1) / kSchedThreads;
  const int c0 = min(tid * per, tiles), c1 = min(c0 + per, tiles);
  uint32_t held[kHeld];
#pragma unroll
  for (int k = 0; k < kHeld; ++k) held[k] = c0 + k < c1 ? counts[first + c0 + k] : 0u;
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kHeld; ++k) sum += held[k];
  for (int i = c0 + kHeld; i < c1; ++i) sum += counts[first + i];
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = s_w[lane];
    uint32_t wi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += u;
    }
    s_w[lane] = wi - v;   // exclusive prefix of the warps' totals
  }
  __syncthreads();
  uint32_t run = s_base + s_w[warp] + inc - sum;
#pragma unroll
  for (int k = 0; k < kHeld; ++k) {
    if (c0 + k < c1) ranges[c0 + k] = make_uint2(run, run + held[k]);
    run += held[k];
  }
  for (int i = c0 + kHeld; i < c1; ++i) {
    const uint32_t c = counts[first + i];
    ranges[i] = make_uint2(run, run + c);
    run += c;
  }
  __syncthreads();
}

// counts (optional): the pair counts of the tiles, from which the tile ranges are written
// first (the batched step's pair sort counts them instead of a separate ranges kernel).
__global__ void __launch_bounds__(kSchedThreads) k_tile_schedule(const uint2* __restrict__ ranges,
                                                                 const uint32_t* __restrict__ cost, int group,
                                                                 int tiles, uint32_t* __restrict__ order,
                                                                 const uint32_t* __restrict__ counts) {
  pdl_wait();
  pdl_trigger();
  if (counts) {
    ranges_from_counts(counts, 0u, tiles, const_cast<uint2*>(ranges));
    schedule_tiles(nullptr, cost ? cost : counts, cost ? group : 1, tiles, order);   // list length = count
  } else {
    schedule_tiles(ranges, cost, group, tiles, order);
  }
}

// Sum over the warp of 10 per-lane values, transposing as it halves: stage 1 (lanes l and
// l^16) pairs value k with value k+5, stage 2 (l^8) pairs slots 0/2 and 1/3 and sums slot 4
// plainly, stage 3 (l^4) pairs slots 0/1 and sums slot 2 plainly, stage 4 (l^2) pairs the
// last two, stage 5 (l^1) sums plainly: 12 shuffles.  Lane l ends with the total of value
// (l & 16 ? 5 : 0) + (l & 2 ? 4 : (l & 8 ? 2 : 0) + (l & 4 ? 1 : 0)).
__device__ __forceinline__ float warp_transpose_sum10(const float v[10]) {
  const int lane = threadIdx.x & 31;
  float u[5], w[3], x[2];
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float send = hi ? v[k] : v[k + 5];
      const float keep = hi ? v[k + 5] : v[k];
      u[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
    }
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float send = hi ? u[k] : u[k + 2];
      const float keep = hi ? u[k + 2] : u[k];
      w[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
    }
    w[2] = u[4] + __shfl_xor_sync(0xFFFFFFFFu, u[4], 8);
  }
  {
    const bool hi = lane & 4;
    const float send = hi ? w[0] : w[1];
    const float keep = hi ? w[1] : w[0];
    x[0] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
    x[1] = w[2] + __shfl_xor_sync(0xFFFFFFFFu, w[2], 4);
  }
  const bool hi = lane & 2;
  const float send = hi ? x[0] : x[1];
  const float keep = hi ? x[1] : x[0];
  const float y = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 2);
  return y + __shfl_xor_sync(0xFFFFFFFFu, y, 1);
}

// Up to this many contributing lanes a (warp, Gaussian) adds its partials with per-lane
// atomics instead of a warp sum.
constexpr int kFewLanes = 16;

// Backward of one tile's warp-blocks (local tile index); warp-autonomous, no block barrier.
// The CTA holds NW warps; its warp w covers the tile's 8x4 block w0 + w.
template <int TW, int NW = kThreads / 32>
__device__ __forceinline__ void blend_bwd_tile(const BlendBwdArgs& a, const BlendCommon& cm, const int tile,
                                               const int w0 = 0) {
  __shared__ float4 s_q0[NW][32], s_q1[NW][32], s_q2[NW][32];
  __shared__ uint32_t s_g[NW][32];

  const RasterParams& rp = a.rp;
  const int tx = tile % rp.ntx, ty = tile / rp.ntx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int px, py;
  float wx0, wy0;
  pixel_of<TW>(tx * rp.tile_w, ty * rp.tile_h, px, py, wx0, wy0, w0 + warp);
  const bool inside = px < rp.W && py < rp.H;
  const int64_t pix = (int64_t)py * rp.W + px;
  const int start = (int)a.ranges[tile].x;

  uint32_t nc = 0;
  float T = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gA = 0.f, gI = 0.f;
  uint32_t gt_match = 0xFFFFFFFEu;
  if (inside) {
    nc = a.n_contrib[pix];
    T = a.T_final[pix];
    if (a.g_rgb) {
      gC0 = a.g_rgb[3 * pix];
      gC1 = a.g_rgb[3 * pix + 1];
      gC2 = a.g_rgb[3 * pix + 2];
    }
    if (a.g_depth) gD = a.g_depth[pix];
    if (a.g_alpha) gA = a.g_alpha[pix];
    if (a.g_ins) gI = a.g_ins[pix];
    if (a.t_gt) {
      const int32_t gt = a.t_gt[pix];
      if (gt >= 0 && gt < rp.num_objects) gt_match = (uint32_t)gt;
    }
  }
  // each warp walks its own pixels' lists back to front: no block-wide barrier
  const int wmax = (int)__reduce_max_sync(kFull, nc);
  float R = T * (gC0 * rp.bg[0] + gC1 * rp.bg[1] + gC2 * rp.bg[2]);
  const float fpx = (float)px, fpy = (float)py;
  const uint32_t lt = lanemask_lt();
  // lanes 0..2 gather the ten warp totals as float4s: lane 0 values 0-3 (held by lanes 0,
  // 4, 8, 12), lane 1 values 4-7 (lanes 2, 16, 20, 24), lane 2 values 8-9 (lanes 28, 18)
  const int src0 = lane == 1 ? 2 : (lane == 2 ? 28 : 0);
  const int src1 = lane == 1 ? 16 : (lane == 2 ? 18 : 4);
  const int src2 = lane == 1 ? 20 : 8;
  const int src3 = lane == 1 ? 24 : 12;

  // the next (earlier) chunk's list entries are loaded while the current one is processed
  const int c0 = (wmax - 1) & ~31;
  uint32_t gnext = wmax > 0 && c0 + lane < wmax ? cm.list[start + c0 + lane] : 0u;
  for (int c = c0; c >= 0 && wmax > 0; c -= 32) {
    const int jl = c + lane;
    bool hit = false;
    float4 q0, q1, q2;
    uint32_t g = 0;
    // the forward's ballot for this chunk and block, when recorded: the same test on the
    // same records, so only its hits are loaded and nothing is tested again
    const uint32_t rec = a.hitmask ? a.hitmask[hit_word(start, start + c, tile, w0 + warp)] : kFull;
    if (jl < wmax && ((rec >> lane) & 1u)) {
      g = gnext;
      q0 = cm.p0[g];
      q1 = cm.p1[g];
      q2 = cm.p2[g];
      hit = a.hitmask ? true : ellipse_hits(q0, q1, q2, wx0, wy0, 7.f, 3.f);
    }
    const uint32_t m = __ballot_sync(kFull, hit);
    if (hit) {
      const int k = __popc(m & lt);
      // q1.w becomes the ins key: the object id, or all ones when the OG filter excludes it
      const uint32_t idog = __float_as_uint(q1.w);
      q1.w = __uint_as_float(cm.og_filter && !(idog >> 31) ? 0xFFFFFFFFu : (idog & kNoObject));
      s_q0[warp][k] = q0;
      s_q1[warp][k] = q1;
      s_q2[warp][k] = q2;
      s_g[warp][k] = g;
    }
    __syncwarp();
    if (c >= 32) gnext = cm.list[start + c - 32 + lane];  // below c <= wmax - 1: in the list
    // staged slots [0, hlim) hold this lane's contributors (list positions below nc): the
    // slots are in list order and slot k came from chunk lane k's position c + k
    const int below = (int)nc - c;
    const int hlim = __popc(m & (below >= 32 ? kFull : (below <= 0 ? 0u : (1u << below) - 1u)));
    // Adds one evaluated Gaussian's partials (staged slot h) back to front and sums them
    // into its gradient record.
    auto accumulate = [&](bool act, float alpha, float G, float dx, float dy, int h) {
      float v[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] = 0.f;
      if (act) {
        const float4 p1 = s_q1[warp][h];
        const float inv = rcp_approx(1.f - alpha);   // 1 - alpha in [1 - clamp, 1]: no special cases
        T = T * inv;
        const float w = alpha * T;
        const float4 p2 = s_q2[warp][h];
        const bool counts = __float_as_uint(p1.w) == gt_match;
        const float U = gC0 * p2.x + gC1 * p2.y + gC2 * p2.z + gD * p1.z + gA + (counts ? gI : 0.f);
        const float dalpha = T * U - R * inv;
        R = fmaf(w, U, R);
        const bool clamped = __fmul_rn(p1.y, G) > cm.alpha_clamp;
        const float dpow = clamped ? 0.f : dalpha * alpha;
        v[0] = dpow * dx;
        v[1] = dpow * dy;
        v[2] = v[0] * dx;
        v[3] = v[0] * dy;
        v[4] = v[1] * dy;
        v[5] = clamped ? 0.f : dalpha * G;
        v[6] = w * gC0;
        v[7] = w * gC1;
        v[8] = w * gC2;
        v[9] = w * gD;
      }
      const uint32_t am = __ballot_sync(kFull, act);
      if (am != 0u && __popc(am) <= kFewLanes) {
        // few contributing lanes: each adds its own partials (three vector atomics, one
        // warp instruction each) instead of the 46-instruction warp sum
        if (act) {
          float4* dst = reinterpret_cast<float4*>(cm.grad2d) + 3 * (int64_t)s_g[warp][h];
          atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
          atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
          atomicAdd(dst + 2, make_float4(v[8], v[9], 0.f, 0.f));
        }
      } else if (am != 0u) {
        const float y = warp_transpose_sum10(v);
        const float a0 = __shfl_sync(kFull, y, src0);
        const float a1 = __shfl_sync(kFull, y, src1);
        float a2 = __shfl_sync(kFull, y, src2);
        float a3 = __shfl_sync(kFull, y, src3);
        if (lane == 2) a2 = a3 = 0.f;   // record slots 10 and 11 are unused
        if (lane < 3) {
          float4* dst = reinterpret_cast<float4*>(cm.grad2d) + 3 * (int64_t)s_g[warp][h] + lane;
          atomicAdd(dst, make_float4(a0, a1, a2, a3));
        }
      }
    };
    // two staged Gaussians per iteration (h, then h - 1): their exponentials are
    // independent; the transmittance and partial sums stay sequential
    for (int h = __popc(m) - 1; h >= 0; h -= 2) {
      const int hb = h > 0 ? h - 1 : 0;
      float aA, GA, dxA, dyA, aB, GB, dxB, dyB;
      const bool eA =
          eval_terms(s_q0[warp][h], s_q1[warp][h], fpx, fpy, cm.alpha_clamp, cm.alpha_min, aA, GA, dxA, dyA);
      const bool eB =
          eval_terms(s_q0[warp][hb], s_q1[warp][hb], fpx, fpy, cm.alpha_clamp, cm.alpha_min, aB, GB, dxB, dyB);
      const bool vA = eA && h < hlim;
      const bool vB = eB && h > 0 && hb < hlim;
      accumulate(vA, aA, GA, dxA, dyA, h);
      if (h > 0) accumulate(vB, aB, GB, dxB, dyB, hb);
    }
    __syncwarp();
  }
}

// The backward kernel's CTAs hold kBwdWarps warps (a part of a tile): a CTA's resources
// are freed only when its last warp ends, and the warps of one tile walk lists of very
// different lengths.  CTA b covers part b % kBwdParts of the b / kBwdParts-th scheduled tile.
constexpr int kBwdWarps = 4;
constexpr int kBwdParts = kThreads / 32 / kBwdWarps;
static_assert(kBwdParts == kTileParts, "tile parts of the backward and of the cost records");

// Eight 4-warp CTAs per SM (64 registers, no spills): 32 resident warps instead of the 28
// that 71 registers allowed; measured 1.4 us faster per step on the indoor keyframe.
template <int TW>
__global__ void __launch_bounds__(32 * kBwdWarps, 32 / kBwdWarps) k_blend_backward(BlendBwdArgs a) {
  pdl_wait();
  pdl_trigger();
  const BlendCommon cm{a.p0, a.p1, a.p2, nullptr, a.list, a.grad2d, a.rp.alpha_clamp, a.rp.alpha_min, 0.f,
                       a.rp.og_filter};
  const int u = (int)(blockIdx.x / kBwdParts);
  blend_bwd_tile<TW, kBwdWarps>(a, cm, a.tile_order ? (int)a.tile_order[u] : u,
                                (int)(blockIdx.x % kBwdParts) * kBwdWarps);
}

// Persistent step over the tiles of a batch of keyframes: each CTA takes tiles from an
// atomic work queue (joint tile numbering, keyframe k owning [tile_off[k],
// tile_off[k+1])) and runs the tile's forward with the fused losses and then its
// backward.  A tile's backward needs only its own pixels' forward state (transmittance,
// blended count, dL/dpixel), written by the same threads just before, so no grid-wide
// barrier separates the two.  Per-keyframe arguments are read from the kernel's
// parameter table.
template <int TW, bool kId>
__global__ void __launch_bounds__(kThreads, 4) k_blend_step(const __grid_constant__ StepTable t, BlendCommon cm,
                                                            uint32_t* __restrict__ queue,
                                                            const uint32_t* __restrict__ order) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_item;
  const uint32_t total = t.tile_off[t.nkf];
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t q = atomicAdd(queue, 1u);
      s_item = q < total && order ? order[q] : q;
    }
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= total) break;
    int k = 0;
    while (k + 1 < t.nkf && t.tile_off[k + 1] <= it) ++k;
    const int tile = (int)(it - t.tile_off[k]);
    blend_fwd_tile<TW, kId>(t.f[k], cm, tile);
    blend_bwd_tile<TW>(t.b[k], cm, tile);
    __syncthreads();
  }
}

// The same queue walk with the forward and the backward as two persistent kernels (each
// with its own queue): fewer registers per kernel than the fused walk.
template <int TW, bool kId>
__global__ void __launch_bounds__(kThreads) k_blend_fwd_queue(const __grid_constant__ StepTable t, BlendCommon cm,
                                                              uint32_t* __restrict__ queue,
                                                              const uint32_t* __restrict__ order) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_item;
  const uint32_t total = t.tile_off[t.nkf];
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t q = atomicAdd(queue, 1u);
      s_item = q < total && order ? order[q] : q;
    }
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= total) break;
    int k = 0;
    while (k + 1 < t.nkf && t.tile_off[k + 1] <= it) ++k;
    blend_fwd_tile<TW, kId>(t.f[k], cm, (int)(it - t.tile_off[k]));
    __syncthreads();
  }
}

// The backward on a work queue of tile parts (CTAs of kBwdWarps warps, like the
// one-keyframe backward): queue entry q is part q % kBwdParts of the (q / kBwdParts)-th
// tile of the order (a tile's parts run next to each other, which measured faster than
// ordering the parts on their own).
template <int TW>
__global__ void __launch_bounds__(32 * kBwdWarps, 28 / kBwdWarps)
    k_blend_bwd_queue(const __grid_constant__ StepTable t, BlendCommon cm, uint32_t* __restrict__ queue,
                      const uint32_t* __restrict__ order) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_item;
  const uint32_t total = t.tile_off[t.nkf] * kBwdParts;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t q = atomicAdd(queue, 1u);
      s_item = q < total && order ? order[q / kBwdParts] * kBwdParts + q % kBwdParts : q;
    }
    __syncthreads();
    const uint32_t u = s_item;
    if (u >= total) break;
    const uint32_t jt = u / kBwdParts;
    int k = 0;
    while (k + 1 < t.nkf && t.tile_off[k + 1] <= jt) ++k;
    blend_bwd_tile<TW, kBwdWarps>(t.b[k], cm, (int)(jt - t.tile_off[k]), (int)(u % kBwdParts) * kBwdWarps);
    __syncthreads();
  }
}

template <int TW>
cudaError_t launch_fwd_tw(const BlendFwdArgs& a, bool with_id, cudaStream_t s) {
  const unsigned tiles = (unsigned)(a.rp.ntx * a.rp.nty);
  if (with_id)
    launch_dep(k_blend_forward<TW, true>, dim3(tiles), dim3(kThreads), s, a);
  else
    launch_dep(k_blend_forward<TW, false>, dim3(tiles), dim3(kThreads), s, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_forward(const BlendFwdArgs& a, bool with_id, cudaStream_t s) {
  if (a.rp.ntx * a.rp.nty == 0) return cudaSuccess;
  switch (a.rp.tile_w) {
    case 8: return launch_fwd_tw<8>(a, with_id, s);
    case 16: return launch_fwd_tw<16>(a, with_id, s);
    case 32: return launch_fwd_tw<32>(a, with_id, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_schedule(const uint2* ranges, const uint32_t* cost, int tiles, uint32_t* order,
                                 cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  launch_dep(k_tile_schedule, dim3(1), dim3(kSchedThreads), s, ranges, cost, kTileParts, tiles, order,
             static_cast<const uint32_t*>(nullptr));
  return cudaGetLastError();
}

cudaError_t launch_loss_reduce(const float* part, int tiles, float lambda_ins, float scale, float* loss,
                               cudaStream_t s) {
  launch_dep(k_loss_reduce, dim3(1), dim3(kThreads), s, part, tiles, lambda_ins, scale, loss);
  return cudaGetLastError();
}

cudaError_t launch_blend_backward(const BlendBwdArgs& a, cudaStream_t s) {
  const unsigned tiles = (unsigned)(a.rp.ntx * a.rp.nty);
  if (tiles == 0) return cudaSuccess;
  switch (a.rp.tile_w) {
    case 8: launch_dep(k_blend_backward<8>, dim3(tiles * kBwdParts), dim3(32 * kBwdWarps), s, a); break;
    case 16: launch_dep(k_blend_backward<16>, dim3(tiles * kBwdParts), dim3(32 * kBwdWarps), s, a); break;
    case 32: launch_dep(k_blend_backward<32>, dim3(tiles * kBwdParts), dim3(32 * kBwdWarps), s, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dqo

namespace dqo {
namespace {

template <typename Kernel>
unsigned persistent_grid(Kernel k, int ctas_per_sm, int sms, uint32_t total, cudaError_t* e,
                         int threads = kThreads) {
  int occ = 0;
  *e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, 0);
  if (*e != cudaSuccess) return 0;
  if (occ < 1) occ = 1;
  const int per = ctas_per_sm > 0 ? (ctas_per_sm < occ ? ctas_per_sm : occ) : occ;
  unsigned grid = (unsigned)(per * sms);
  return grid > total ? total : grid;
}

// One CTA per keyframe of a step table: which = 0 orders t.f[k]'s tiles by list length
// into t.f[k].tile_order, which = 1 by t.f[k].tile_cost into t.b[k].tile_order.
__global__ void __launch_bounds__(kSchedThreads) k_tile_schedule_batch(const __grid_constant__ StepTable t,
                                                                       int which) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.x;
  const int tiles = (int)(t.tile_off[k + 1] - t.tile_off[k]);
  if (which == 0) {
    if (t.tile_count) {
      // the ranges from the pair counts; a tile's cost (its list length) is its count
      ranges_from_counts(t.tile_count, t.tile_off[k], tiles, const_cast<uint2*>(t.f[k].ranges));
      schedule_tiles(nullptr, t.tile_count + t.tile_off[k], 1, tiles, const_cast<uint32_t*>(t.f[k].tile_order));
    } else {
      schedule_tiles(t.f[k].ranges, nullptr, 1, tiles, const_cast<uint32_t*>(t.f[k].tile_order));
    }
  }
  else
    schedule_tiles(nullptr, t.f[k].tile_cost, kTileParts, tiles, const_cast<uint32_t*>(t.b[k].tile_order));
}

// Blend schedules of a batch: 0 = fused queue kernel, 1 = forward and backward queue
// kernels, 2 = the one-keyframe kernels launched per keyframe (arguments by value).
template <int TW, bool kId>
cudaError_t step_tw(const StepTable& t, const BlendCommon& cm, uint32_t* queue, int ctas_per_sm, int sms,
                    int schedule, cudaStream_t s) {
  const uint32_t total = t.tile_off[t.nkf];
  if (total == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  // heaviest tiles first (see schedule_tiles): the queue kernels take the batch's joint
  // tiles in one joint order (the per-keyframe arrays are slices of joint arrays, so
  // keyframe 0's pointers are the joint bases), the per-keyframe kernels per keyframe
  const bool sched = t.f[0].tile_order && t.f[0].tile_cost && t.b[0].tile_order && t.tile_off[0] == 0;
  if (t.tile_count && !sched) return cudaErrorInvalidValue;   // the ranges come from the forward's schedule
  uint32_t* f_order = sched ? const_cast<uint32_t*>(t.f[0].tile_order) : nullptr;
  uint32_t* b_order = sched ? const_cast<uint32_t*>(t.b[0].tile_order) : nullptr;
  if (schedule == 0) {
    const unsigned grid = persistent_grid(k_blend_step<TW, kId>, ctas_per_sm, sms, total, &e);
    if (e != cudaSuccess) return e;
    if (sched)
      launch_dep(k_tile_schedule, dim3(1), dim3(kSchedThreads), s, t.f[0].ranges, nullptr, 1, (int)total, f_order,
                 t.tile_count);
    k_blend_step<TW, kId><<<grid, kThreads, 0, s>>>(t, cm, queue, f_order);
  } else if (schedule == 1) {
    unsigned grid = persistent_grid(k_blend_fwd_queue<TW, kId>, ctas_per_sm, sms, total, &e);
    if (e != cudaSuccess) return e;
    if (sched)
      launch_dep(k_tile_schedule, dim3(1), dim3(kSchedThreads), s, t.f[0].ranges, nullptr, 1, (int)total, f_order,
                 t.tile_count);
    k_blend_fwd_queue<TW, kId><<<grid, kThreads, 0, s>>>(t, cm, queue, f_order);
    // the backward's CTAs are tile parts: as many warps per SM as ctas_per_sm whole tiles
    grid = persistent_grid(k_blend_bwd_queue<TW>, ctas_per_sm > 0 ? ctas_per_sm * kBwdParts : 0, sms,
                           total * kBwdParts, &e, 32 * kBwdWarps);
    if (e != cudaSuccess) return e;
    if (sched)
      launch_dep(k_tile_schedule, dim3(1), dim3(kSchedThreads), s, nullptr, t.f[0].tile_cost, kTileParts,
                 (int)total, b_order, nullptr);
    k_blend_bwd_queue<TW><<<grid, 32 * kBwdWarps, 0, s>>>(t, cm, queue + 1, b_order);
  } else {
    if (sched) launch_dep(k_tile_schedule_batch, dim3((unsigned)t.nkf), dim3(kSchedThreads), s, t, 0);
    for (int k = 0; k < t.nkf; ++k) {
      const unsigned tiles = t.tile_off[k + 1] - t.tile_off[k];
      if (tiles == 0) continue;
      BlendFwdArgs f = t.f[k];
      f.p0 = cm.p0;
      f.p1 = cm.p1;
      f.p2 = cm.p2;
      f.gid = cm.gid;
      f.list = cm.list;
      launch_dep(k_blend_forward<TW, kId>, dim3(tiles), dim3(kThreads), s, f);
    }
    if (sched) launch_dep(k_tile_schedule_batch, dim3((unsigned)t.nkf), dim3(kSchedThreads), s, t, 1);
    for (int k = 0; k < t.nkf; ++k) {
      const unsigned tiles = t.tile_off[k + 1] - t.tile_off[k];
      if (tiles == 0) continue;
      BlendBwdArgs b = t.b[k];
      b.p0 = cm.p0;
      b.p1 = cm.p1;
      b.p2 = cm.p2;
      b.list = cm.list;
      b.grad2d = cm.grad2d;
      launch_dep(k_blend_backward<TW>, dim3(tiles * kBwdParts), dim3(32 * kBwdWarps), s, b);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_step(const StepTable& t, const BlendCommon& cm, uint32_t* queue, int tile_w, bool with_id,
                              int ctas_per_sm, int sms, int schedule, cudaStream_t s) {
  switch (tile_w * 2 + (with_id ? 1 : 0)) {
    case 16: return step_tw<8, false>(t, cm, queue, ctas_per_sm, sms, schedule, s);
    case 17: return step_tw<8, true>(t, cm, queue, ctas_per_sm, sms, schedule, s);
    case 32: return step_tw<16, false>(t, cm, queue, ctas_per_sm, sms, schedule, s);
    case 33: return step_tw<16, true>(t, cm, queue, ctas_per_sm, sms, schedule, s);
    case 64: return step_tw<32, false>(t, cm, queue, ctas_per_sm, sms, schedule, s);
    case 65: return step_tw<32, true>(t, cm, queue, ctas_per_sm, sms, schedule, s);
    default: return cudaErrorInvalidValue;
  }
}


}  // namespace dqo
