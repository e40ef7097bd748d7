// Internal declarations of the dqo CUDA library (sm_103a).  Host launchers are
// declared here and defined next to their kernels; dqo_api.cu drives them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dqo.h"

namespace dqo {

constexpr int kThreads = 256;          // CTA size of every rasterizer kernel (one pixel / thread)
constexpr int kMaxRadixPasses = 8;    // 8-bit digits of up to 64-bit keys
constexpr int kMaxObjects = 4096;      // object ids per scene handled by the id-map prepass
constexpr int kMaskWords = kMaxObjects / 32;
constexpr int kIdSlots = 16;           // per-tile object slots held in shared memory per round
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
// Scratch words of a radix sort over `tiles` CTA tiles and `passes` passes: per pass the
// digit histogram, its exclusive scan and every tile's look-back status row; per pass a
// tile counter; a block counter of the histogram kernel; an error word.
constexpr size_t onesweep_scratch_words(int64_t tiles, int passes) {
  return (size_t)passes * kRadixBins * (size_t)(tiles + 2) + (size_t)passes + 2;
}
constexpr int kScanItems = 8;         // values per thread in the scan kernel
constexpr int kScanTile = kThreads * kScanItems;   // values per CTA of the scan
constexpr uint32_t kNoObject = 0x7FFFFFFFu;
constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------- device helpers

// One MUFU.EX2: 2^x (x <= 0 here), flushing denormal results to zero.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// PTX rcp.approx (relative error within 1 ulp on normal inputs).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-pixel evaluation of one projected Gaussian, shared bit-for-bit by the forward and
// backward blend kernels so both take the same skip / clamp decisions.  p0 = (x, y, a',
// b'), p1 = (c', opacity, z, id bits) with the conic pre-scaled so that
// G = 2^(a' dx^2 + b' dx dy + c' dy^2) = exp(-q/2).  Returns false if the Gaussian is
// skipped (exponent > 0 or alpha < alpha_min).
__device__ __forceinline__ bool eval_gaussian(const float4& p0, const float4& p1, float px, float py,
                                              float alpha_clamp, float alpha_min, float& alpha,
                                              float& G, float& dx, float& dy) {
  dx = __fsub_rn(px, p0.x);
  dy = __fsub_rn(py, p0.y);
  const float t = __fmaf_rn(p0.w, dy, __fmul_rn(p0.z, dx));
  const float pw = __fmaf_rn(__fmul_rn(p1.x, dy), dy, __fmul_rn(t, dx));
  if (pw > 0.f) return false;
  G = ex2_approx(pw);
  alpha = fminf(alpha_clamp, __fmul_rn(p1.y, G));
  return alpha >= alpha_min;
}

// Programmatic dependent launch.  A kernel started with launch_dep may become resident
// while the previous kernel of its stream drains; it calls pdl_wait() before it touches
// memory (returns once the previous kernel has completed and its writes are visible), and
// pdl_trigger() so that its own dependent may be scheduled early.  Both are no-ops for a
// kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Deterministic sum of the per-tile loss partials, scaled by 1/(HW).  The first kThreads
// threads of the block each add their tiles t, t + kThreads, ... in that order in FP32
// (loads issued eight tiles at a time before the additions), the per-thread sums are added
// by a fixed FP32 shuffle tree within each warp, and thread 0 adds the warps' sums in
// order in FP64.  The order depends on nothing but the tile count, so the result is the
// same for any block of at least kThreads threads and on every run.  The partials are
// non-negative, so the FP32 sums carry a relative error of a few 1e-7.  (An FP64 sum of
// every partial took 10 us: this GPU's FP64 pipe is slow.)  Every thread takes part in
// the barrier.
__device__ __forceinline__ void loss_reduce(const float* __restrict__ part, int tiles, float lambda_ins, float scale,
                                            float* __restrict__ loss) {
  constexpr int kBatch = 8;
  __shared__ float s[3][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < kThreads) {
    float acc[3] = {0.f, 0.f, 0.f};
    for (int t0 = threadIdx.x; t0 < tiles; t0 += kBatch * kThreads) {
      float v[kBatch][3];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int t = t0 + j * kThreads;
#pragma unroll
        for (int k = 0; k < 3; ++k) v[j][k] = t < tiles ? part[3 * t + k] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] += v[j][k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float x = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      if (lane == 0) s[k][warp] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0, d = 0, i = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      r += (double)s[0][w];
      d += (double)s[1][w];
      i += (double)s[2][w];
    }
    r *= scale;
    d *= scale;
    i *= scale;
    loss[0] = (float)r;
    loss[1] = (float)d;
    loss[2] = (float)i;
    loss[3] = (float)(r + d + (double)lambda_ins * i);
  }
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  return launch_dep_smem(kernel, grid, block, 0, s, args...);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------- launch descriptors

struct RasterParams {
  int W, H, tile_w, tile_h, ntx, nty;
  float fx, fy, cx, cy;
  float vm[12];
  float alpha_clamp, alpha_min, t_stop, znear, lowpass, radius_sigma, lambda_ins;
  float bg[3];
  int og_filter;
  int batch;
  int num_objects;
  float theta_alpha, theta_d, theta_c;
};

struct ProjBuffers {
  float4* p0;
  float4* p1;
  float4* p2;
  ushort4* rect;
  uint32_t* ntiles;
  uint32_t* zkey;    // depth sort keys: float bits of z, 0xFFFFFFFF if culled
  uint32_t* zval;    // depth sort values: Gaussian index
  uint32_t* gid;     // object id (kNoObject if none) for the id-map prepass
  uint32_t* n_visible;
  float4* grad2d = nullptr;  // if set: each binned Gaussian's backward moment record is zeroed
};

struct BlendFwdArgs {
  RasterParams rp;
  const float4* p0;
  const float4* p1;
  const float4* p2;
  const uint32_t* gid;
  const uint2* ranges;
  const uint32_t* list;
  const float* t_rgb;
  const float* t_depth;
  const int32_t* t_gt;
  float* o_rgb;
  float* o_depth;
  float* o_alpha;
  float* o_ins;
  int32_t* o_id;
  float* T_final;
  uint32_t* n_contrib;
  float* dl_rgb;     // saved dL/dC  [H*W*3] (with targets)
  float* dl_depth;   // saved dL/dD  [H*W]
  float* dl_ins;     // saved dL/dins[H*W]
  float* loss_part;  // [T*3] per-tile loss sums
  uint8_t* o_mask;   // [H*W] Eq. 11 update masks (with targets)
  const uint32_t* tile_order = nullptr;  // [T] block b blends tile tile_order[b] (null: tile b)
  uint32_t* tile_cost = nullptr;         // [T * kTileParts] out: longest blended prefix per tile part
  uint32_t* hitmask = nullptr;           // [8 * (M/32 + T + 1)] out: per warp-block and list chunk, the
                                         // ballot of the entries that can reach the block (null: none)
};

struct BlendBwdArgs {
  RasterParams rp;
  const float4* p0;
  const float4* p1;
  const float4* p2;
  const uint2* ranges;
  const uint32_t* list;
  const int32_t* t_gt;
  const float* T_final;
  const uint32_t* n_contrib;
  const float* g_rgb;
  const float* g_depth;
  const float* g_alpha;
  const float* g_ins;
  float* grad2d;     // [n*12] moment records (accumulated with atomics)
  const uint32_t* tile_order = nullptr;  // [T] block b walks tile tile_order[b] (null: tile b)
  const uint32_t* hitmask = nullptr;     // the forward's hit record (null: test again)
};

struct PreBwdArgs {
  RasterParams rp;
  int64_t n;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logit;
  const uint32_t* ntiles;
  const float* grad2d;
  float* d_means;
  float* d_log_scales;
  float* d_quats;
  float* d_logit;
  float* d_rgb;
  int32_t mode;        // kGradAdd, kGradAtomic or kGradStore
};
constexpr int32_t kGradAdd = 0;     // gradients += (one keyframe)
constexpr int32_t kGradAtomic = 1;  // gradients added atomically (buffers shared by keyframes)
constexpr int32_t kGradStore = 2;   // gradients overwritten, zero for Gaussians never binned

// ---------------------------------------------------------------- launchers (return cudaGetLastError)

cudaError_t launch_preprocess(const RasterParams& rp, const dqo_gaussians& g, const ProjBuffers& out,
                              cudaStream_t s);
cudaError_t launch_preprocess_backward(const PreBwdArgs& a, cudaStream_t s);

// ----------------------------------------------------------------------------- batches
// Per-keyframe tables of a batch travel as __grid_constant__ kernel parameters (captured
// with the launch in a CUDA graph; no staging buffer).

constexpr int kMaxBatch = 16;

// One keyframe of a batch for projection: its parameters, Gaussians and global offset.
struct PreKf {
  RasterParams rp;
  dqo_gaussians g;
  int64_t base;
};
struct PreTable {
  PreKf kf[kMaxBatch];
};
// Keyframe k's loss: its per-tile partials, summed (loss_reduce) into loss[0..3].
struct LossKf {
  const float* part;
  int tiles;
  float lambda_ins, scale;
  float* loss;
};
// The batch's projection adjoint also sums each keyframe's loss partials (CTA column 0):
// the blend backward needs no loss value, so the sums run beside the adjoint's Gaussians.
struct PreBwdTable {
  PreBwdArgs kf[kMaxBatch];
  LossKf loss[kMaxBatch];
};
cudaError_t launch_preprocess_batch(const PreTable& t, int nkf, int64_t max_n, const ProjBuffers& out,
                                    cudaStream_t s);
cudaError_t launch_preprocess_backward_batch(const PreBwdTable& t, int nkf, int64_t max_n, cudaStream_t s);

// Exclusive scan of n uint32 values in[i] (in[gather[i]] when gather is given; one kernel,
// decoupled look-back); total (uint64) written to *total.  scratch must hold
// scan_scratch_words(n) uint64 words, cleared by the call unless `zeroed` says the caller
// cleared them.  err (optional): set to 1 if a look-back wait gave up.
size_t scan_scratch_words(int64_t n);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* scratch,
                                  uint64_t* total, cudaStream_t s, uint32_t* err = nullptr,
                                  const uint32_t* gather = nullptr, bool zeroed = false);

// Stable LSD radix sort of n keys on bits [begin_bit, end_bit), optional uint32 values: one kernel
// counts all digits, then one kernel per 8-bit digit with decoupled look-back.  Results
// land in whichever of the double buffers *sel says (0: *_a, 1: *_b).  scratch holds
// radix_scratch_words(n) uint32 words (histograms, look-back status, counters).  rank
// (optional, with values): rank[value] = the value's position in the sorted order, written
// by the last pass.  n_dev (optional): live count on the device, n being the capacity.
// err (optional): set to 1 if a look-back wait gave up (about a second); NULL keeps the
// flag inside scratch.  The call clears the radix_scratch_used_words(n, begin_bit, end_bit)
// words it uses first, unless `zeroed` says the caller already did (so that the sort's first
// kernel follows the previous kernel directly).
size_t radix_scratch_words(int64_t n);
size_t radix_scratch_used_words(int64_t n, int begin_bit, int end_bit);
int64_t radix_sort_launches(int64_t n, int end_bit, int begin_bit = 0);
cudaError_t radix_sort_u32(uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a, uint32_t* vals_b, int64_t n,
                           int end_bit, uint32_t* scratch, int* sel, cudaStream_t s, uint32_t* rank = nullptr,
                           uint32_t* err = nullptr, int begin_bit = 0, bool zeroed = false);
cudaError_t radix_sort_u64(uint64_t* keys_a, uint64_t* keys_b, int64_t n, int end_bit, uint32_t* scratch, int* sel,
                           cudaStream_t s, const uint64_t* n_dev = nullptr, uint32_t* err = nullptr,
                           int begin_bit = 0);
cudaError_t radix_sort_u32_dev(uint32_t* keys_a, uint32_t* keys_b, int64_t n, int end_bit, uint32_t* scratch,
                               int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* err = nullptr,
                               int begin_bit = 0);

// Pairs (tile << rank_bits | depth rank) of the Gaussians in depth order: rank r's Gaussian
// order[r] writes its tiles' keys from offsets[r] (tile counts scanned in rank order).
cudaError_t launch_emit_pairs_u32(const ushort4* rect, const uint32_t* offsets, const uint32_t* order,
                                  int64_t n, int ntx, int rank_bits, uint32_t* keys, cudaStream_t s);
cudaError_t launch_emit_pairs_u64(const ushort4* rect, const uint32_t* offsets, const uint32_t* order,
                                  int64_t n, int ntx, int rank_bits, uint64_t* keys, cudaStream_t s);
cudaError_t launch_tile_ranges_u32(const uint32_t* keys, int64_t m, int rank_bits, const uint32_t* order,
                                   uint2* ranges, uint32_t* list, cudaStream_t s, const uint64_t* m_dev = nullptr);

cudaError_t launch_tile_ranges_u64(const uint64_t* keys, int64_t m, int rank_bits, const uint32_t* order,
                                   uint2* ranges, uint32_t* list, cudaStream_t s, const uint64_t* m_dev = nullptr);

// One keyframe of a batch for pair emission: its Gaussians occupy global indices
// [base, base + n), its tiles [tile_off, tile_off + ntx * nty) of the joint numbering.
struct EmitKf {
  int64_t base;
  int64_t n;
  uint32_t tile_off;
  int ntx;
};
struct EmitTable {
  EmitKf kf[16];
};
// The same over a batch's n joint Gaussians in joint depth order.  keys: uint32_t[capacity]
// if k32 (tile and rank bits fit 32), else uint64_t[capacity].  A Gaussian whose pairs do
// not fit the capacity sets *overflow; *live (all ones before) becomes min(*total, first
// pair not written), the count the pair sort then reads.
cudaError_t launch_emit_pairs_batch(const EmitTable& t, int nkf, int64_t n, const ushort4* rect,
                                    const uint32_t* offsets, const uint32_t* order, int rank_bits, uint64_t capacity,
                                    void* keys, bool k32, uint32_t* overflow, const uint64_t* total, uint64_t* live,
                                    cudaStream_t s);
// The same emission with the scan of the pair counts in the kernel (no offsets array):
// scratch holds scan_emit_scratch_words(n) uint64 words, all zero before the call; the
// pair total goes to *total and bounds *live.  err: look-back timeout flag (scratch's own
// word if NULL).
size_t scan_emit_scratch_words(int64_t n);
cudaError_t launch_scan_emit_pairs_batch(const EmitTable& t, int nkf, int64_t n, const ushort4* rect,
                                         const uint32_t* order, int rank_bits, uint64_t capacity, void* keys, bool k32,
                                         uint32_t* overflow, uint64_t* scratch, uint32_t* err, uint64_t* total,
                                         uint64_t* live, cudaStream_t s);

// What the last pass of a pair sort writes instead of the sorted keys: the tile list
// (list[p] = order[rank of key p]) and each tile's pair count (added to counts[tile], zero
// before).  Keys whose tile or rank is out of range are skipped, and positions at or past
// the live count are not written.
struct PairOut {
  const uint32_t* order;
  uint32_t* list;
  uint32_t* counts;
  int rank_bits;
  uint32_t tiles;
  uint32_t n_order;
};
// Pair sorts whose last pass writes the tile list and the per-tile counts (po).
cudaError_t radix_sort_pairs_u32(uint32_t* keys_a, uint32_t* keys_b, int64_t n, int end_bit, uint32_t* scratch,
                                 int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* err, int begin_bit,
                                 const PairOut& po, bool zeroed = false);
cudaError_t radix_sort_pairs_u64(uint64_t* keys_a, uint64_t* keys_b, int64_t n, int end_bit, uint32_t* scratch,
                                 int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* err, int begin_bit,
                                 const PairOut& po, bool zeroed = false);

cudaError_t launch_blend_forward(const BlendFwdArgs& a, bool with_id, cudaStream_t s);
// Tile schedule: order[0..tiles) lists the tiles by decreasing cost (cost[t], or the
// tile's list length ranges[t].y - ranges[t].x when cost is null), on a log scale of four
// buckets per octave; tiles of one bucket come in no fixed order.  One CTA.
// The backward walks a tile in kTileParts parts of kTileWarps / kTileParts warps (8x4
// blocks); the forward reports each part's cost.
constexpr int kTileParts = 2;
cudaError_t launch_tile_schedule(const uint2* ranges, const uint32_t* cost, int tiles, uint32_t* order,
                                 cudaStream_t s);
cudaError_t launch_loss_reduce(const float* part, int tiles, float lambda_ins, float scale, float* loss,
                               cudaStream_t s);
cudaError_t launch_blend_backward(const BlendBwdArgs& a, cudaStream_t s);

// Persistent forward + backward over the tiles of a batch (tables in device memory).
// ctas_per_sm <= 0: as many as fit.
struct StepTable {
  BlendFwdArgs f[16];
  BlendBwdArgs b[16];
  const uint32_t* tile_count;  // pairs per joint tile; the forward schedule turns them into ranges
  uint32_t tile_off[17];  // keyframe k owns joint tiles [tile_off[k], tile_off[k+1])
  int nkf;
};
// What every tile of a batch reads in its inner loops: the joint projected-Gaussian arrays,
// the tile lists, the gradient record and the blending thresholds.  Passed by value, so the
// loops read it as constant-bank operands; the per-keyframe table is read only at a tile's
// start and end.
struct BlendCommon {
  const float4* p0;
  const float4* p1;
  const float4* p2;
  const uint32_t* gid;
  const uint32_t* list;
  float* grad2d;
  float alpha_clamp, alpha_min, t_stop;
  int og_filter;
};
// schedule: 0 = one fused persistent kernel (forward then backward per tile), 1 = forward
// and backward persistent kernels (queue and queue + 1), 2 = the one-keyframe kernels per
// keyframe.
cudaError_t launch_blend_step(const StepTable& t, const BlendCommon& cm, uint32_t* queue, int tile_w, bool with_id,
                              int ctas_per_sm, int sms, int schedule, cudaStream_t s);

cudaError_t launch_quadric_project(int nq, const float* params, int nv, const float* P, const int32_t* q_ptr,
                                   const int32_t* pair_v, int npairs, float* conic, float* bbox, uint8_t* valid,
                                   cudaStream_t s);
cudaError_t launch_quadric_bbox_loss(int nq, const float* params, int nv, const float* P, const int32_t* q_ptr,
                                     const int32_t* pair_v, int npairs, const float* obs, float* loss,
                                     float* dparams, cudaStream_t s);

cudaError_t launch_quadric_fit(int nq, int nv, const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                               int npairs, const float* obs, int iters, float lr, const float* start, float* init,
                               float* params, float* loss, uint8_t* ok, cudaStream_t s);
cudaError_t launch_quadric_canonical(int nq, const float* in, float* out, cudaStream_t s);

// ----------------------------------------------------------------------------- learned proposal

constexpr int kMlpViews = 8, kMlpIn = 128, kMlpHidden = 128, kMlpOut = 9, kMlpOutPad = 16;
// FP32 parameter vector: W1 [128][128] (out x in), b1, W2 [128][128], b2, W3 [16][128]
// (rows 9..15 zero), b3 [16]
constexpr int kMlpW1 = 0, kMlpB1 = 16384, kMlpW2 = 16512, kMlpB2 = 32896, kMlpW3 = 33024, kMlpB3 = 35072,
              kMlpParams = 35088;

// Element offset of (r, c) in a BF16 weight copy [R][128] kept in the tensor-core tile layout:
// column blocks of 8, each R rows of 8 contiguous values (the kernels copy it unchanged into
// shared memory).
__host__ __device__ __forceinline__ int grid_index(int r, int c, int R) { return (c >> 3) * R * 8 + r * 8 + (c & 7); }

// Views into the caller-owned state buffer.
struct MlpState {
  float *param, *grad, *m1, *m2;       // [kMlpParams] each
  __nv_bfloat16 *w1b, *w2b;            // W1, W2 [128][128], tile layout (grid_index)
  __nv_bfloat16* w3b;                  // W3 [16][128], tile layout
  int* step;                           // optimiser steps taken
};

// Context workspace: the forward's activations and the training kernel's per-tile gradients.
struct MlpWork {
  __nv_bfloat16 *h1, *h2;  // [n][128]
  int* err;
  unsigned* bar;           // the training kernel's grid barrier counter
  float* gpart;            // [n / 128][kMlpParams]
};

__device__ __forceinline__ void write_bf16_copies(const MlpState& st, int i, float p) {
  const __nv_bfloat16 b = __float2bfloat16_rn(p);
  if (i < kMlpB1) {
    st.w1b[grid_index(i / kMlpIn, i % kMlpIn, kMlpHidden)] = b;
  } else if (i >= kMlpW2 && i < kMlpB2) {
    const int k = i - kMlpW2;
    st.w2b[grid_index(k / kMlpHidden, k % kMlpHidden, kMlpHidden)] = b;
  } else if (i >= kMlpW3 && i < kMlpB3) {
    const int k = i - kMlpW3;
    st.w3b[grid_index(k / kMlpHidden, k % kMlpHidden, kMlpOutPad)] = b;
  }
}

cudaError_t mlp_gemm_setup();
cudaError_t launch_bounded_wait_probe(int* flag, cudaStream_t s);
// FP32 FMA (kind 0) or ex2 (kind 1) throughput probe over every SM; *ops = operations launched.
cudaError_t launch_alu_probe(int kind, int iters, float* sink, double* ops, cudaStream_t s);
cudaError_t launch_mlp_features(int nq, int nv, const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                                int npairs, const float* obs, const int32_t* counts, float inv_scale, uint16_t* X,
                                uint16_t* XT, int64_t ldt, cudaStream_t s);
cudaError_t launch_mlp_set(const MlpState& st, const float* params, cudaStream_t s);
cudaError_t launch_mlp_forward(const MlpState& st, const MlpWork& wk, int64_t n, const uint16_t* X, float* y,
                               cudaStream_t s);
// Training: `steps` Adam steps on consecutive batches of `batch` rows of X / labels (the
// per-step losses into losses[steps], may be NULL), or with grad_mode the loss gradient of
// one batch into grads.  One cooperative launch (mlp_gemm_setup first).
cudaError_t launch_mlp_train(const MlpState& st, const dqo_mlp_hparams& hp, bool grad_mode, int steps,
                             int64_t batch, const uint16_t* X, const float* labels, float* losses, float* grads,
                             const MlpWork& wk, cudaStream_t s);
}  // namespace dqo
