// Host side of the C ABI declared in include/dqo.h: argument checks, the context's
// grow-only workspace, and the launch sequence of each entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dqo_internal.cuh"

using namespace dqo;

namespace {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

struct dqo_ctx {
  int device = 0;
  int last_err = 0;
  // per-Gaussian
  Buf p0, p1, p2, rect, ntiles, zkey_a, zkey_b, zval_a, zval_b, gid, offsets, grad2d;
  // sorting scratch
  Buf scan_scratch, depth_scan_scratch, hist, depth_hist, pair_a, pair_b, list;
  // per-tile / per-pixel
  Buf ranges, loss_part, T_final, n_contrib, dl_rgb, dl_depth, dl_ins;
  Buf tile_sched;           // uint32 [tiles] forward order, [tiles * kTileParts] part costs, backward order
  Buf hitrec;               // uint32 [8 (pairs / 32 + tiles + 1)]: the forward's hit ballots for the backward
  Buf counters;             // device: [0] uint64 total pairs, [1] uint32 n_visible
  Buf sort_err;             // device uint32: a radix sort's look-back wait gave up (sticky until read)
  uint64_t* host_counters = nullptr;  // pinned mirror
  cudaEvent_t count_ready = nullptr;  // recorded after the pair count is copied to the host
  // state of the last forward
  bool have_fwd = false;
  bool fwd_dl = false;
  int64_t n = 0, m = 0, n_vis = 0;
  int W = 0, H = 0, tile_w = 0, tile_h = 0, ntx = 0, nty = 0;
  int order_sel = 0;
  // phase timing and launch accounting
  bool timing = false;
  cudaEvent_t ev[2 * DQO_PHASE_COUNT] = {};
  bool pending[DQO_PHASE_COUNT] = {};
  bool captured[DQO_PHASE_COUNT] = {};  // recorded inside a graph capture: re-read each query
  float last_ms[DQO_PHASE_COUNT] = {};
  int64_t launches = 0;
  // batched step: joint buffers of all keyframes of a batch, pair capacity, side stream
  struct Batch {
    Buf p0, p1, p2, rect, ntiles, zkey_a, zkey_b, zval_a, zval_b, gid, offsets, grad2d;
    Buf scan_scratch, depth_scan_scratch, depth_hist, hist, pair_a, pair_b, list, ranges, tile_count, loss_part;
    Buf T_final, n_contrib, dl_rgb, dl_depth, dl_ins, counters, tile_sched, hitrec;
    uint64_t* host = nullptr;  // pinned: pair count of a sizing call
    std::vector<int64_t> sig;  // layout of the last sizing call
    uint64_t capacity = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int sms = 0;
  } b;
  // learned proposal: activations of the last batch size, error flag
  Buf mlp_work;
  int64_t mlp_n = 0;
  bool mlp_ready = false;
};

namespace {

dqo_status cuda_fail(dqo_ctx* c, cudaError_t e) {
  if (c) c->last_err = (int)e;
  return e == cudaErrorMemoryAllocation ? DQO_ENOMEM : DQO_ECUDA;
}

#define DQO_CUDA(ctx, expr)                         \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_); \
  } while (0)

cudaError_t ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return cudaSuccess;
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    if (e != cudaSuccess) return e;
    b.p = nullptr;
    b.cap = 0;
  }
  const size_t want = std::max(bytes, b.cap + b.cap / 4);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return e;
    }
    b.cap = bytes;
    return cudaSuccess;
  }
  b.cap = want;
  return cudaSuccess;
}

template <typename T>
T* as(const Buf& b) {
  return reinterpret_cast<T*>(b.p);
}

// Words of the blend's hit record: 8 warp-blocks x (pairs / 32 + tiles + 1) list chunks.
size_t hit_record_words(uint64_t pairs, uint64_t tiles) { return 8 * (size_t)(pairs / 32 + tiles + 1); }

int bits_for(uint64_t v) {  // smallest b with v <= 2^b (at least 1)
  int b = 1;
  while (b < 64 && (uint64_t(1) << b) < v) ++b;
  return b;
}

dqo_status check_settings(const dqo_settings* s) {
  if (!s) return DQO_EINVAL;
  if (!(s->tile_w == 8 || s->tile_w == 16 || s->tile_w == 32) || s->tile_w * s->tile_h != kThreads)
    return DQO_EINVAL;
  if (s->batch < 32 || s->batch > 256 || (s->batch & 31)) return DQO_EINVAL;
  if (s->grads_zero != 0 && s->grads_zero != 1) return DQO_EINVAL;
  if (!(s->alpha_clamp > 0.f) || !(s->alpha_min >= 0.f) || !(s->t_stop >= 0.f) || !(s->znear > 0.f) ||
      !(s->lowpass >= 0.f) || !(s->radius_sigma > 0.f) || !(s->lambda_ins >= 0.f))
    return DQO_EINVAL;
  return DQO_OK;
}

dqo_status check_gaussians(const dqo_gaussians* g) {
  if (!g) return DQO_EINVAL;
  if (g->n < 0 || g->n > (int64_t(1) << 26)) return DQO_EINVAL;
  if (g->num_objects < 1 || g->num_objects > kMaxObjects) return DQO_EINVAL;
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->rgb || !g->obj_id ||
                   !g->flags))
    return DQO_EINVAL;
  return DQO_OK;
}

dqo_status check_camera(const dqo_camera* c) {
  if (!c) return DQO_EINVAL;
  if (c->width < 1 || c->height < 1 || c->width > 32768 || c->height > 32768) return DQO_EINVAL;
  if (!(c->fx > 0.f) || !(c->fy > 0.f)) return DQO_EINVAL;
  return DQO_OK;
}

struct PhaseTimer {
  dqo_ctx* c;
  int ph;
  cudaStream_t s;
  unsigned flags = cudaEventRecordDefault;
  PhaseTimer(dqo_ctx* c_, int ph_, cudaStream_t s_) : c(c_), ph(ph_), s(s_) {
    if (!c->timing) return;
    // inside a graph capture the events must become event-record nodes of the graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      flags = cudaEventRecordExternal;
    cudaEventRecordWithFlags(c->ev[2 * ph], s, flags);
  }
  ~PhaseTimer() {
    if (c->timing) {
      cudaEventRecordWithFlags(c->ev[2 * ph + 1], s, flags);
      c->pending[ph] = true;
      c->captured[ph] = flags == cudaEventRecordExternal;
    }
  }
};

// kernels launched by one radix sort of n keys over end_bit bits, and by one scan
int64_t scan_launches(int64_t n) { return n > 0 ? 1 : 0; }

RasterParams make_params(const dqo_settings* s, const dqo_gaussians* g, const dqo_camera* c) {
  RasterParams rp;
  rp.W = c->width;
  rp.H = c->height;
  rp.tile_w = s->tile_w;
  rp.tile_h = s->tile_h;
  rp.ntx = (c->width + s->tile_w - 1) / s->tile_w;
  rp.nty = (c->height + s->tile_h - 1) / s->tile_h;
  rp.fx = c->fx;
  rp.fy = c->fy;
  rp.cx = c->cx;
  rp.cy = c->cy;
  std::memcpy(rp.vm, c->viewmat, sizeof(rp.vm));
  rp.alpha_clamp = s->alpha_clamp;
  rp.alpha_min = s->alpha_min;
  rp.t_stop = s->t_stop;
  rp.znear = s->znear;
  rp.lowpass = s->lowpass;
  rp.radius_sigma = s->radius_sigma;
  rp.lambda_ins = s->lambda_ins;
  rp.bg[0] = s->bg[0];
  rp.bg[1] = s->bg[1];
  rp.bg[2] = s->bg[2];
  rp.og_filter = s->og_filter ? 1 : 0;
  rp.batch = s->batch;
  rp.num_objects = g->num_objects;
  rp.theta_alpha = s->theta_alpha;
  rp.theta_d = s->theta_d;
  rp.theta_c = s->theta_c;
  return rp;
}

}  // namespace

extern "C" {

void dqo_settings_default(dqo_settings* s) {
  if (!s) return;
  s->tile_w = 16;
  s->tile_h = 16;
  s->alpha_clamp = 0.99f;
  s->alpha_min = 1.0f / 255.0f;
  s->t_stop = 1e-4f;
  s->znear = 0.2f;
  s->lowpass = 0.3f;
  s->radius_sigma = 3.0f;
  s->lambda_ins = 1.0f;
  s->bg[0] = s->bg[1] = s->bg[2] = 0.0f;
  s->og_filter = 1;
  s->batch = 256;
  s->theta_alpha = 0.5f;
  s->theta_d = 0.1f;
  s->theta_c = 0.1f;
  s->grads_zero = 0;
}

int dqo_version(void) { return 100; }

const char* dqo_status_str(dqo_status s) {
  switch (s) {
    case DQO_OK: return "ok";
    case DQO_EINVAL: return "invalid argument";
    case DQO_ENOMEM: return "out of device memory";
    case DQO_ECUDA: return "CUDA error";
    case DQO_ETIMEOUT: return "device wait timed out";
    case DQO_ENOTIMPL: return "not implemented";
    case DQO_ESTATE: return "no matching forward state";
  }
  return "unknown status";
}

dqo_status dqo_create(dqo_ctx** out, int device) {
  if (!out) return DQO_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return DQO_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return DQO_ECUDA;
  dqo_ctx* c = new (std::nothrow) dqo_ctx();
  if (!c) return DQO_ENOMEM;
  c->device = device;
  if (ensure(c->counters, 64) != cudaSuccess || ensure(c->sort_err, 16) != cudaSuccess ||
      cudaMemset(c->sort_err.p, 0, 16) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&c->host_counters), 64) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->count_ready, cudaEventDisableTiming) != cudaSuccess) {
    dqo_destroy(c);
    return DQO_ENOMEM;
  }
  *out = c;
  return DQO_OK;
}

void dqo_destroy(dqo_ctx* c) {
  if (!c) return;
  Buf* all[] = {&c->p0, &c->p1, &c->p2, &c->rect, &c->ntiles, &c->zkey_a, &c->zkey_b, &c->zval_a,
                &c->zval_b, &c->gid, &c->offsets, &c->grad2d, &c->scan_scratch,
                &c->depth_scan_scratch, &c->hist, &c->depth_hist,
                &c->pair_a, &c->pair_b, &c->list, &c->ranges, &c->loss_part, &c->T_final, &c->n_contrib,
                &c->dl_rgb, &c->dl_depth, &c->dl_ins, &c->counters, &c->sort_err, &c->tile_sched, &c->hitrec};
  for (Buf* b : all)
    if (b->p) cudaFree(b->p);
  dqo_ctx::Batch& B = c->b;
  Buf* ball[] = {&B.p0, &B.p1, &B.p2, &B.rect, &B.ntiles, &B.tile_count, &B.zkey_a, &B.zkey_b, &B.zval_a,
                 &B.zval_b, &B.gid, &B.offsets, &B.grad2d, &B.scan_scratch, &B.depth_scan_scratch, &B.depth_hist, &B.hist,
                 &B.pair_a, &B.pair_b, &B.list, &B.ranges, &B.loss_part, &B.T_final, &B.n_contrib, &B.dl_rgb,
                 &B.dl_depth, &B.dl_ins, &B.counters, &B.tile_sched, &B.hitrec, &c->mlp_work};
  for (Buf* b : ball)
    if (b->p) cudaFree(b->p);
  if (B.host) cudaFreeHost(B.host);
  if (B.fork) cudaEventDestroy(B.fork);
  if (B.join) cudaEventDestroy(B.join);
  if (B.side) cudaStreamDestroy(B.side);
  if (c->host_counters) cudaFreeHost(c->host_counters);
  if (c->count_ready) cudaEventDestroy(c->count_ready);
  for (int i = 0; i < 2 * DQO_PHASE_COUNT; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  delete c;
}

int dqo_last_cuda_error(const dqo_ctx* c) { return c ? c->last_err : 0; }

dqo_status dqo_render_forward(dqo_ctx* c, const dqo_settings* s, const dqo_gaussians* g, const dqo_camera* cam,
                              const dqo_targets* t, dqo_render_out* out, dqo_stream stream_) {
  if (!c || !out) return DQO_EINVAL;
  dqo_status st;
  if ((st = check_settings(s)) != DQO_OK) return st;
  if ((st = check_gaussians(g)) != DQO_OK) return st;
  if ((st = check_camera(cam)) != DQO_OK) return st;
  if (t && (!t->gt_id || !t->rgb)) return DQO_EINVAL;
  if ((out->loss || out->update_mask) && !t) return DQO_EINVAL;
  cudaStream_t s_ = reinterpret_cast<cudaStream_t>(stream_);
  DQO_CUDA(c, cudaSetDevice(c->device));
  c->have_fwd = false;

  const RasterParams rp = make_params(s, g, cam);
  const int64_t n = g->n;
  const int64_t HW = (int64_t)rp.W * rp.H;
  const int tiles = rp.ntx * rp.nty;

  // ---- workspace
  DQO_CUDA(c, ensure(c->p0, 16 * n));
  DQO_CUDA(c, ensure(c->p1, 16 * n));
  DQO_CUDA(c, ensure(c->p2, 16 * n));
  DQO_CUDA(c, ensure(c->rect, 8 * n));
  DQO_CUDA(c, ensure(c->ntiles, 4 * n));
  DQO_CUDA(c, ensure(c->zkey_a, 4 * n));
  DQO_CUDA(c, ensure(c->zkey_b, 4 * n));
  DQO_CUDA(c, ensure(c->zval_a, 4 * n));
  DQO_CUDA(c, ensure(c->zval_b, 4 * n));
  DQO_CUDA(c, ensure(c->gid, 4 * n));
  DQO_CUDA(c, ensure(c->offsets, 4 * n));
  DQO_CUDA(c, ensure(c->ranges, 8 * (size_t)tiles));
  DQO_CUDA(c, ensure(c->tile_sched, 4 * (1 + 2 * kTileParts) * (size_t)tiles));
  DQO_CUDA(c, ensure(c->loss_part, 12 * (size_t)tiles));
  DQO_CUDA(c, ensure(c->T_final, 4 * HW));
  DQO_CUDA(c, ensure(c->n_contrib, 4 * HW));
  if (t) {
    DQO_CUDA(c, ensure(c->dl_rgb, 12 * HW));
    DQO_CUDA(c, ensure(c->dl_depth, 4 * HW));
    DQO_CUDA(c, ensure(c->dl_ins, 4 * HW));
  }
  DQO_CUDA(c, ensure(c->scan_scratch, 8 * scan_scratch_words(n)));
  DQO_CUDA(c, ensure(c->depth_scan_scratch, 8 * scan_scratch_words(radix_scratch_words(n))));
  DQO_CUDA(c, ensure(c->depth_hist, 4 * radix_scratch_words(n)));
  DQO_CUDA(c, cudaMemsetAsync(c->counters.p, 0, 64, s_));

  uint64_t* d_total = as<uint64_t>(c->counters);
  uint32_t* d_nvis = reinterpret_cast<uint32_t*>(as<uint64_t>(c->counters) + 1);

  // ---- K1 projection
  ProjBuffers pb;
  const int64_t nb_launch = n > 0 ? 1 : 0;
  pb.p0 = as<float4>(c->p0);
  pb.p1 = as<float4>(c->p1);
  pb.p2 = as<float4>(c->p2);
  pb.rect = as<ushort4>(c->rect);
  pb.ntiles = as<uint32_t>(c->ntiles);
  pb.zkey = as<uint32_t>(c->zkey_a);
  pb.zval = as<uint32_t>(c->zval_a);
  pb.gid = as<uint32_t>(c->gid);
  pb.n_visible = d_nvis;
  {
    PhaseTimer pt(c, DQO_PHASE_PROJECT, s_);
    DQO_CUDA(c, launch_preprocess(rp, *g, pb, s_));
  }
  c->launches += nb_launch;

  // ---- K4a depth order, then K2: the scan of tiles per Gaussian in depth order (pair
  // offsets by rank); the pair count goes to the host
  int sel = 0;
  const uint32_t* order = nullptr;
  {
    PhaseTimer pt(c, DQO_PHASE_DEPTH_SORT, s_);
    DQO_CUDA(c, radix_sort_u32(as<uint32_t>(c->zkey_a), as<uint32_t>(c->zkey_b), as<uint32_t>(c->zval_a),
                               as<uint32_t>(c->zval_b), n, 32, as<uint32_t>(c->depth_hist), &sel, s_, nullptr,
                               as<uint32_t>(c->sort_err)));
    order = sel ? as<uint32_t>(c->zval_b) : as<uint32_t>(c->zval_a);
    DQO_CUDA(c, launch_exclusive_scan(as<uint32_t>(c->ntiles), as<uint32_t>(c->offsets), n,
                                      as<uint64_t>(c->scan_scratch), d_total, s_, as<uint32_t>(c->sort_err), order));
    DQO_CUDA(c, cudaMemcpyAsync(c->host_counters, c->counters.p, 16, cudaMemcpyDeviceToHost, s_));
    DQO_CUDA(c, cudaMemcpyAsync(c->host_counters + 2, c->sort_err.p, 4, cudaMemcpyDeviceToHost, s_));
    DQO_CUDA(c, cudaEventRecord(c->count_ready, s_));
  }
  c->order_sel = sel;
  c->launches += scan_launches(n) + radix_sort_launches(n, 32);

  // ---- pair count on the host (the one wait of the forward)
  DQO_CUDA(c, cudaEventSynchronize(c->count_ready));
  const uint64_t m = c->host_counters[0];
  const uint64_t n_vis = (uint32_t)(c->host_counters[1] & 0xFFFFFFFFu);
  if (m >= (uint64_t(1) << 31)) return DQO_ENOMEM;  // tile ranges are int32 in the blend kernels
  if (c->host_counters[2] & 0xFFFFFFFFu) {          // an earlier call's sort wait gave up
    DQO_CUDA(c, cudaMemsetAsync(c->sort_err.p, 0, 4, s_));
    return DQO_ETIMEOUT;
  }

  // ---- K3-K5 pairs, pair sort, tile ranges
  {
  PhaseTimer pt(c, DQO_PHASE_BINNING, s_);
  DQO_CUDA(c, cudaMemsetAsync(c->ranges.p, 0, 8 * (size_t)tiles, s_));
  if (m > 0) {
    const int rank_bits = bits_for(n_vis);
    const int tile_bits = bits_for((uint64_t)tiles);
    const int end_bit = rank_bits + tile_bits;
    const bool k32 = end_bit <= 32;
    const size_t ks = k32 ? 4 : 8;
    DQO_CUDA(c, ensure(c->pair_a, ks * m));
    DQO_CUDA(c, ensure(c->pair_b, ks * m));
    DQO_CUDA(c, ensure(c->list, 4 * m));
    DQO_CUDA(c, ensure(c->hist, 4 * radix_scratch_words((int64_t)m)));
    DQO_CUDA(c, ensure(c->scan_scratch, 8 * scan_scratch_words(radix_scratch_words((int64_t)m))));
    int psel = 0;
    // pairs come out in depth-rank order: a stable sort on the tile bits finishes the job
    c->launches += 2 + radix_sort_launches((int64_t)m, end_bit, rank_bits);
    if (k32) {
      DQO_CUDA(c, launch_emit_pairs_u32(as<ushort4>(c->rect), as<uint32_t>(c->offsets), order, n, rp.ntx, rank_bits,
                                        as<uint32_t>(c->pair_a), s_));
      DQO_CUDA(c, radix_sort_u32(as<uint32_t>(c->pair_a), as<uint32_t>(c->pair_b), nullptr, nullptr, (int64_t)m,
                                 end_bit, as<uint32_t>(c->hist), &psel, s_, nullptr, as<uint32_t>(c->sort_err),
                                 rank_bits));
      DQO_CUDA(c, launch_tile_ranges_u32(psel ? as<uint32_t>(c->pair_b) : as<uint32_t>(c->pair_a), (int64_t)m,
                                         rank_bits, order, as<uint2>(c->ranges), as<uint32_t>(c->list), s_));
    } else {
      DQO_CUDA(c, launch_emit_pairs_u64(as<ushort4>(c->rect), as<uint32_t>(c->offsets), order, n, rp.ntx, rank_bits,
                                        as<uint64_t>(c->pair_a), s_));
      DQO_CUDA(c, radix_sort_u64(as<uint64_t>(c->pair_a), as<uint64_t>(c->pair_b), (int64_t)m, end_bit,
                                 as<uint32_t>(c->hist), &psel, s_, nullptr, as<uint32_t>(c->sort_err), rank_bits));
      DQO_CUDA(c, launch_tile_ranges_u64(psel ? as<uint64_t>(c->pair_b) : as<uint64_t>(c->pair_a), (int64_t)m,
                                         rank_bits, order, as<uint2>(c->ranges), as<uint32_t>(c->list), s_));
    }
  } else {
    DQO_CUDA(c, ensure(c->list, 4));
  }
  }

  // ---- K6 blend + fused losses
  BlendFwdArgs a;
  a.rp = rp;
  a.p0 = pb.p0;
  a.p1 = pb.p1;
  a.p2 = pb.p2;
  a.gid = pb.gid;
  a.ranges = as<uint2>(c->ranges);
  a.list = as<uint32_t>(c->list);
  a.t_rgb = t ? t->rgb : nullptr;
  a.t_depth = t ? t->depth : nullptr;
  a.t_gt = t ? t->gt_id : nullptr;
  a.o_rgb = out->rgb;
  a.o_depth = out->depth;
  a.o_alpha = out->alpha;
  a.o_ins = out->ins;
  a.o_id = out->id_map;
  a.T_final = as<float>(c->T_final);
  a.n_contrib = as<uint32_t>(c->n_contrib);
  a.dl_rgb = t ? as<float>(c->dl_rgb) : nullptr;
  a.dl_depth = t ? as<float>(c->dl_depth) : nullptr;
  a.dl_ins = t ? as<float>(c->dl_ins) : nullptr;
  a.loss_part = as<float>(c->loss_part);
  a.o_mask = out->update_mask;
  a.tile_order = as<uint32_t>(c->tile_sched);
  a.tile_cost = as<uint32_t>(c->tile_sched) + tiles;
  DQO_CUDA(c, ensure(c->hitrec, 4 * hit_record_words(m, tiles)));
  a.hitmask = as<uint32_t>(c->hitrec);
  {
    PhaseTimer pt(c, DQO_PHASE_BLEND_FWD, s_);
    DQO_CUDA(c, launch_tile_schedule(a.ranges, nullptr, tiles, const_cast<uint32_t*>(a.tile_order), s_));
    DQO_CUDA(c, launch_blend_forward(a, out->id_map != nullptr, s_));
    if (out->loss)
      DQO_CUDA(c, launch_loss_reduce(as<float>(c->loss_part), tiles, rp.lambda_ins,
                                     (float)(1.0 / ((double)rp.W * (double)rp.H)), out->loss, s_));
  }
  c->launches += (tiles > 0 ? 2 : 0) + (out->loss ? 1 : 0);

  c->have_fwd = true;
  c->fwd_dl = t != nullptr;
  c->n = n;
  c->m = (int64_t)m;
  c->n_vis = (int64_t)n_vis;
  c->W = rp.W;
  c->H = rp.H;
  c->tile_w = rp.tile_w;
  c->tile_h = rp.tile_h;
  c->ntx = rp.ntx;
  c->nty = rp.nty;
  return DQO_OK;
}

dqo_status dqo_render_backward(dqo_ctx* c, const dqo_settings* s, const dqo_gaussians* g, const dqo_camera* cam,
                               const dqo_targets* t, const dqo_pixel_grads* pg, dqo_gaussian_grads* grads,
                               dqo_stream stream_) {
  if (!c || !grads) return DQO_EINVAL;
  dqo_status st;
  if ((st = check_settings(s)) != DQO_OK) return st;
  if ((st = check_gaussians(g)) != DQO_OK) return st;
  if ((st = check_camera(cam)) != DQO_OK) return st;
  if (t && (!t->gt_id || !t->rgb)) return DQO_EINVAL;
  if (!c->have_fwd || c->n != g->n || c->W != cam->width || c->H != cam->height || c->tile_w != s->tile_w ||
      c->tile_h != s->tile_h)
    return DQO_ESTATE;
  if (!pg && !c->fwd_dl) return DQO_ESTATE;
  cudaStream_t s_ = reinterpret_cast<cudaStream_t>(stream_);
  DQO_CUDA(c, cudaSetDevice(c->device));
  const RasterParams rp = make_params(s, g, cam);
  const int64_t n = g->n;
  DQO_CUDA(c, ensure(c->grad2d, 48 * n));
  if (n > 0) DQO_CUDA(c, cudaMemsetAsync(c->grad2d.p, 0, 48 * n, s_));

  BlendBwdArgs a;
  a.rp = rp;
  a.p0 = as<float4>(c->p0);
  a.p1 = as<float4>(c->p1);
  a.p2 = as<float4>(c->p2);
  a.ranges = as<uint2>(c->ranges);
  a.list = as<uint32_t>(c->list);
  a.t_gt = t ? t->gt_id : nullptr;
  a.T_final = as<float>(c->T_final);
  a.n_contrib = as<uint32_t>(c->n_contrib);
  if (pg) {
    a.g_rgb = pg->rgb;
    a.g_depth = pg->depth;
    a.g_alpha = pg->alpha;
    a.g_ins = pg->ins;
  } else {
    a.g_rgb = as<float>(c->dl_rgb);
    a.g_depth = as<float>(c->dl_depth);
    a.g_alpha = nullptr;
    a.g_ins = as<float>(c->dl_ins);
  }
  a.grad2d = as<float>(c->grad2d);
  const int tiles = c->ntx * c->nty;
  a.tile_order = as<uint32_t>(c->tile_sched) + (1 + kTileParts) * (size_t)tiles;
  a.hitmask = as<uint32_t>(c->hitrec);
  {
    PhaseTimer pt(c, DQO_PHASE_BLEND_BWD, s_);
    DQO_CUDA(c, launch_tile_schedule(nullptr, as<uint32_t>(c->tile_sched) + tiles, tiles,
                                     const_cast<uint32_t*>(a.tile_order), s_));
    DQO_CUDA(c, launch_blend_backward(a, s_));
  }
  c->launches += tiles > 0 ? 2 : 0;

  PreBwdArgs b;
  b.rp = rp;
  b.n = n;
  b.means = g->means;
  b.log_scales = g->log_scales;
  b.quats = g->quats;
  b.opacity_logit = g->opacity_logit;
  b.ntiles = as<uint32_t>(c->ntiles);
  b.grad2d = as<float>(c->grad2d);
  b.d_means = grads->means;
  b.d_log_scales = grads->log_scales;
  b.d_quats = grads->quats;
  b.d_logit = grads->opacity_logit;
  b.d_rgb = grads->rgb;
  b.mode = s->grads_zero ? kGradStore : kGradAdd;
  {
    PhaseTimer pt(c, DQO_PHASE_PROJECT_BWD, s_);
    DQO_CUDA(c, launch_preprocess_backward(b, s_));
  }
  c->launches += n > 0 ? 1 : 0;
  return DQO_OK;
}

dqo_status dqo_get_buffer(dqo_ctx* c, dqo_buffer which, void* dst, size_t capacity, size_t* bytes,
                          dqo_stream stream_) {
  if (!c) return DQO_EINVAL;
  if (!c->have_fwd) return DQO_ESTATE;
  const void* src = nullptr;
  size_t sz = 0;
  const int64_t HW = (int64_t)c->W * c->H;
  switch (which) {
    case DQO_BUF_PROJ: {
      // three float4 planes, copied back to back
      sz = 48 * (size_t)c->n;
      if (bytes) *bytes = sz;
      if (!dst) return DQO_OK;
      if (capacity < sz) return DQO_EINVAL;
      cudaStream_t s_ = reinterpret_cast<cudaStream_t>(stream_);
      const size_t pl = 16 * (size_t)c->n;
      if (pl) {
        DQO_CUDA(c, cudaMemcpyAsync(dst, c->p0.p, pl, cudaMemcpyDefault, s_));
        DQO_CUDA(c, cudaMemcpyAsync((char*)dst + pl, c->p1.p, pl, cudaMemcpyDefault, s_));
        DQO_CUDA(c, cudaMemcpyAsync((char*)dst + 2 * pl, c->p2.p, pl, cudaMemcpyDefault, s_));
      }
      return DQO_OK;
    }
    case DQO_BUF_RECT: src = c->rect.p; sz = 8 * (size_t)c->n; break;
    case DQO_BUF_DEPTH_ORDER: src = c->order_sel ? c->zval_b.p : c->zval_a.p; sz = 4 * (size_t)c->n; break;
    case DQO_BUF_TILE_RANGES: src = c->ranges.p; sz = 8 * (size_t)c->ntx * c->nty; break;
    case DQO_BUF_TILE_LIST: src = c->list.p; sz = 4 * (size_t)c->m; break;
    case DQO_BUF_T_FINAL: src = c->T_final.p; sz = 4 * (size_t)HW; break;
    case DQO_BUF_N_CONTRIB: src = c->n_contrib.p; sz = 4 * (size_t)HW; break;
    case DQO_BUF_GRAD2D: src = c->grad2d.p; sz = c->grad2d.p ? 48 * (size_t)c->n : 0; break;
    default: return DQO_EINVAL;
  }
  if (bytes) *bytes = sz;
  if (!dst) return DQO_OK;
  if (capacity < sz) return DQO_EINVAL;
  if (sz) DQO_CUDA(c, cudaMemcpyAsync(dst, src, sz, cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream_)));
  return DQO_OK;
}

dqo_status dqo_set_timing(dqo_ctx* c, int enable) {
  if (!c) return DQO_EINVAL;
  if (enable && !c->ev[0]) {
    DQO_CUDA(c, cudaSetDevice(c->device));
    for (int i = 0; i < 2 * DQO_PHASE_COUNT; ++i) DQO_CUDA(c, cudaEventCreate(&c->ev[i]));
  }
  c->timing = enable != 0;
  for (int i = 0; i < DQO_PHASE_COUNT; ++i) {
    c->pending[i] = false;
    c->captured[i] = false;
    c->last_ms[i] = -1.f;
  }
  return DQO_OK;
}

dqo_status dqo_get_timings(dqo_ctx* c, float* ms, int32_t n) {
  if (!c || !ms || n < 1) return DQO_EINVAL;
  for (int i = 0; i < DQO_PHASE_COUNT; ++i) {
    if (c->pending[i] || c->captured[i]) {
      DQO_CUDA(c, cudaEventSynchronize(c->ev[2 * i + 1]));
      float t = 0.f;
      DQO_CUDA(c, cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]));
      c->last_ms[i] = t;
      c->pending[i] = false;
    }
  }
  for (int i = 0; i < n && i < DQO_PHASE_COUNT; ++i) ms[i] = c->last_ms[i];
  for (int i = DQO_PHASE_COUNT; i < n; ++i) ms[i] = -1.f;
  return DQO_OK;
}

int64_t dqo_launch_count(const dqo_ctx* c) { return c ? c->launches : 0; }

dqo_status dqo_get_counts(const dqo_ctx* c, int64_t* n_pairs, int64_t* n_visible, int32_t* n_tiles) {
  if (!c) return DQO_EINVAL;
  if (!c->have_fwd) return DQO_ESTATE;
  if (n_pairs) *n_pairs = c->m;
  if (n_visible) *n_visible = c->n_vis;
  if (n_tiles) *n_tiles = c->ntx * c->nty;
  return DQO_OK;
}

dqo_status dqo_quadric_project(dqo_ctx* c, int32_t nq, const float* params, int32_t nv, const float* P,
                               const int32_t* q_ptr, const int32_t* pair_v, int32_t npairs, float* conic,
                               float* bbox, uint8_t* valid, dqo_stream stream_) {
  if (!c || nq < 0 || nv < 0 || npairs < 0) return DQO_EINVAL;
  if (nq > 0 && (!params || !q_ptr)) return DQO_EINVAL;
  if (npairs > 0 && (!P || !pair_v || nv == 0)) return DQO_EINVAL;
  DQO_CUDA(c, cudaSetDevice(c->device));
  {
    PhaseTimer pt(c, DQO_PHASE_QUADRIC, reinterpret_cast<cudaStream_t>(stream_));
    DQO_CUDA(c, launch_quadric_project(nq, params, nv, P, q_ptr, pair_v, npairs, conic, bbox, valid,
                                       reinterpret_cast<cudaStream_t>(stream_)));
  }
  c->launches += nq > 0 ? 1 : 0;
  return DQO_OK;
}

dqo_status dqo_quadric_bbox_loss(dqo_ctx* c, int32_t nq, const float* params, int32_t nv, const float* P,
                                 const int32_t* q_ptr, const int32_t* pair_v, int32_t npairs, const float* obs,
                                 float* loss, float* dparams, dqo_stream stream_) {
  if (!c || nq < 0 || nv < 0 || npairs < 0) return DQO_EINVAL;
  if (nq > 0 && (!params || !q_ptr)) return DQO_EINVAL;
  if (npairs > 0 && (!P || !pair_v || !obs || nv == 0)) return DQO_EINVAL;
  DQO_CUDA(c, cudaSetDevice(c->device));
  {
    PhaseTimer pt(c, DQO_PHASE_QUADRIC, reinterpret_cast<cudaStream_t>(stream_));
    DQO_CUDA(c, launch_quadric_bbox_loss(nq, params, nv, P, q_ptr, pair_v, npairs, obs, loss, dparams,
                                         reinterpret_cast<cudaStream_t>(stream_)));
  }
  c->launches += nq > 0 ? 1 : 0;
  return DQO_OK;
}

dqo_status dqo_quadric_fit(dqo_ctx* c, int32_t nq, int32_t nv, const float* P, const int32_t* q_ptr,
                           const int32_t* pair_v, int32_t npairs, const float* obs, int32_t iters, float lr,
                           const float* start, float* init, float* params, float* loss, uint8_t* ok,
                           dqo_stream stream_) {
  if (!c || nq < 0 || nv < 0 || npairs < 0 || iters < 0 || !(lr >= 0.f)) return DQO_EINVAL;
  if (nq > 0 && !q_ptr) return DQO_EINVAL;
  if (npairs > 0 && (!P || !pair_v || !obs || nv == 0)) return DQO_EINVAL;
  DQO_CUDA(c, cudaSetDevice(c->device));
  {
    PhaseTimer pt(c, DQO_PHASE_QUADRIC, reinterpret_cast<cudaStream_t>(stream_));
    DQO_CUDA(c, launch_quadric_fit(nq, nv, P, q_ptr, pair_v, npairs, obs, iters, lr, start, init, params, loss,
                                   ok, reinterpret_cast<cudaStream_t>(stream_)));
  }
  c->launches += nq > 0 ? 1 : 0;
  return DQO_OK;
}

// ----------------------------------------------------------------------------- batched step

namespace {

dqo_status check_fits(const dqo_fit_batch* f) {
  if (!f) return DQO_OK;
  if (f->nq < 0 || f->nv < 0 || f->npairs < 0 || f->iters < 0 || !(f->lr >= 0.f)) return DQO_EINVAL;
  if (f->nq > 0 && !f->q_ptr) return DQO_EINVAL;
  if (f->npairs > 0 && (!f->P || !f->pair_v || !f->obs_bbox || f->nv == 0)) return DQO_EINVAL;
  return DQO_OK;
}

}  // namespace

// Two keyframes' gradient buffers are shared if any of their five arrays coincide.
bool grads_share(const dqo_gaussian_grads& a, const dqo_gaussian_grads& b) {
  const float* pa[5] = {a.means, a.log_scales, a.quats, a.opacity_logit, a.rgb};
  const float* pb[5] = {b.means, b.log_scales, b.quats, b.opacity_logit, b.rgb};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j)
      if (pa[i] && pa[i] == pb[j]) return true;
  return false;
}

dqo_status dqo_batch_step(dqo_ctx* c, const dqo_settings* s, int32_t nkf, const dqo_keyframe* kfs,
                          const dqo_fit_batch* fits, int32_t ctas_per_sm, int32_t schedule, dqo_stream stream_) {
  if (!c || !kfs || nkf < 1 || nkf > kMaxBatch || schedule < 0 || schedule > 2) return DQO_EINVAL;
  dqo_status st;
  if ((st = check_settings(s)) != DQO_OK) return st;
  if ((st = check_fits(fits)) != DQO_OK) return st;
  for (int k = 0; k < nkf; ++k) {
    if ((st = check_gaussians(&kfs[k].gaussians)) != DQO_OK) return st;
    if ((st = check_camera(&kfs[k].camera)) != DQO_OK) return st;
    if (!kfs[k].targets.gt_id || !kfs[k].targets.rgb) return DQO_EINVAL;
  }
  cudaStream_t s_ = reinterpret_cast<cudaStream_t>(stream_);
  DQO_CUDA(c, cudaSetDevice(c->device));
  dqo_ctx::Batch& B = c->b;

  // ---- joint layout: Gaussians, tiles and pixels of keyframe k at base / toff / poff
  RasterParams rp[kMaxBatch];
  int64_t base[kMaxBatch], poff[kMaxBatch];
  uint32_t toff[kMaxBatch + 1];
  int64_t N = 0, P = 0, max_n = 0;
  uint64_t T = 0;
  std::vector<int64_t> sig = {nkf, s->tile_w, s->tile_h};
  bool with_id = false;
  for (int k = 0; k < nkf; ++k) {
    const dqo_keyframe& kf = kfs[k];
    rp[k] = make_params(s, &kf.gaussians, &kf.camera);
    base[k] = N;
    N += kf.gaussians.n;
    max_n = std::max(max_n, kf.gaussians.n);
    toff[k] = (uint32_t)T;
    T += (uint64_t)rp[k].ntx * rp[k].nty;
    poff[k] = P;
    P += (int64_t)rp[k].W * rp[k].H;
    with_id = with_id || kf.out.id_map != nullptr;
    sig.push_back(kf.gaussians.n);
    sig.push_back(rp[k].W);
    sig.push_back(rp[k].H);
  }
  if (T >= (uint64_t(1) << 31) || N >= (int64_t(1) << 31)) return DQO_EINVAL;
  toff[nkf] = (uint32_t)T;
  const bool sizing = B.capacity == 0 || sig != B.sig;
  if (sizing) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DQO_CUDA(c, cudaStreamIsCapturing(s_, &cs));
    if (cs != cudaStreamCaptureStatusNone) return DQO_ESTATE;
    DQO_CUDA(c, ensure(B.p0, 16 * N));
    DQO_CUDA(c, ensure(B.p1, 16 * N));
    DQO_CUDA(c, ensure(B.p2, 16 * N));
    DQO_CUDA(c, ensure(B.rect, 8 * N));
    DQO_CUDA(c, ensure(B.ntiles, 4 * N));
    DQO_CUDA(c, ensure(B.zkey_a, 4 * N));
    DQO_CUDA(c, ensure(B.zkey_b, 4 * N));
    DQO_CUDA(c, ensure(B.zval_a, 4 * N));
    DQO_CUDA(c, ensure(B.zval_b, 4 * N));
    DQO_CUDA(c, ensure(B.gid, 4 * N));
    DQO_CUDA(c, ensure(B.offsets, 4 * N));
    DQO_CUDA(c, ensure(B.grad2d, 48 * N));
    DQO_CUDA(c, ensure(B.ranges, 8 * T));
    DQO_CUDA(c, ensure(B.tile_count, 4 * T));
    DQO_CUDA(c, ensure(B.tile_sched, 4 * (1 + 2 * kTileParts) * T));
    DQO_CUDA(c, ensure(B.loss_part, 12 * T));
    DQO_CUDA(c, ensure(B.T_final, 4 * P));
    DQO_CUDA(c, ensure(B.n_contrib, 4 * P));
    DQO_CUDA(c, ensure(B.dl_rgb, 12 * P));
    DQO_CUDA(c, ensure(B.dl_depth, 4 * P));
    DQO_CUDA(c, ensure(B.dl_ins, 4 * P));
    DQO_CUDA(c, ensure(B.depth_hist, 4 * radix_scratch_words(N)));
    DQO_CUDA(c, ensure(B.depth_scan_scratch, 8 * scan_scratch_words(radix_scratch_words(N))));
    DQO_CUDA(c, ensure(B.scan_scratch, 8 * std::max(scan_scratch_words(N), scan_emit_scratch_words(N))));
    DQO_CUDA(c, ensure(B.counters, 64));
    if (!B.host) DQO_CUDA(c, cudaMallocHost(reinterpret_cast<void**>(&B.host), 64));
    if (!B.side) DQO_CUDA(c, cudaStreamCreateWithFlags(&B.side, cudaStreamNonBlocking));
    if (!B.fork) DQO_CUDA(c, cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming));
    if (!B.join) DQO_CUDA(c, cudaEventCreateWithFlags(&B.join, cudaEventDisableTiming));
    if (!B.sms) DQO_CUDA(c, cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, c->device));
  }
  uint64_t* d_total = as<uint64_t>(B.counters);
  uint32_t* d_nvis = reinterpret_cast<uint32_t*>(d_total + 1);
  uint32_t* d_overflow = d_nvis + 1;
  uint32_t* d_queue = reinterpret_cast<uint32_t*>(d_total + 2);
  uint32_t* d_sort_err = d_queue + 2;  // byte 24: a sort's look-back wait gave up
  uint64_t* d_live = d_total + 4;      // byte 32: pairs the pair sort reads (all ones before the emission)
  const int rank_bits = bits_for((uint64_t)N);  // static bounds, so the step captures
  const int tile_bits = bits_for(T);
  const int end_bit = rank_bits + tile_bits;
  int64_t launches = 0;

  DQO_CUDA(c, cudaMemsetAsync(B.counters.p, 0, 32, s_));
  DQO_CUDA(c, cudaMemsetAsync(d_live, 0xFF, 8, s_));
  DQO_CUDA(c, cudaMemsetAsync(B.tile_count.p, 0, 4 * T, s_));   // the ranges are written from these
  // the sorts' and the scan's scratch, cleared up front so that the chain from the projection
  // to the blend runs kernel after kernel (programmatic launches, no copy engine between);
  // a sizing call allocates the pair sort's scratch later and lets the sort clear it
  DQO_CUDA(c, cudaMemsetAsync(B.depth_hist.p, 0, 4 * radix_scratch_used_words(N, 0, 32), s_));
  DQO_CUDA(c, cudaMemsetAsync(B.scan_scratch.p, 0, 8 * std::max(scan_scratch_words(N), scan_emit_scratch_words(N)),
                              s_));
  if (!sizing)
    DQO_CUDA(c, cudaMemsetAsync(B.hist.p, 0, 4 * radix_scratch_used_words((int64_t)B.capacity, rank_bits, end_bit),
                                s_));
  if (s->grads_zero) {
    // gradient buffers shared by several keyframes take atomic additions: clear them first
    // (once per buffer set); unshared ones are overwritten by the adjoint
    for (int k = 0; k < nkf; ++k) {
      bool shared = false, first = true;
      for (int j = 0; j < nkf; ++j) {
        if (j == k || !grads_share(kfs[j].grads, kfs[k].grads)) continue;
        shared = true;
        if (j < k) first = false;
      }
      if (!shared || !first) continue;
      const dqo_gaussian_grads& gr = kfs[k].grads;
      const size_t n = (size_t)kfs[k].gaussians.n;
      if (gr.means) DQO_CUDA(c, cudaMemsetAsync(gr.means, 0, 12 * n, s_));
      if (gr.log_scales) DQO_CUDA(c, cudaMemsetAsync(gr.log_scales, 0, 12 * n, s_));
      if (gr.quats) DQO_CUDA(c, cudaMemsetAsync(gr.quats, 0, 16 * n, s_));
      if (gr.opacity_logit) DQO_CUDA(c, cudaMemsetAsync(gr.opacity_logit, 0, 4 * n, s_));
      if (gr.rgb) DQO_CUDA(c, cudaMemsetAsync(gr.rgb, 0, 12 * n, s_));
    }
  }

  // ---- quadric fits on the side stream, concurrent with the keyframes
  const bool run_fits = fits && fits->nq > 0;
  if (run_fits) {
    DQO_CUDA(c, cudaEventRecord(B.fork, s_));
    DQO_CUDA(c, cudaStreamWaitEvent(B.side, B.fork, 0));
    DQO_CUDA(c, launch_quadric_fit(fits->nq, fits->nv, fits->P, fits->q_ptr, fits->pair_v, fits->npairs,
                                   fits->obs_bbox, fits->iters, fits->lr, fits->start, fits->init, fits->params,
                                   fits->loss, fits->ok, B.side));
    DQO_CUDA(c, cudaEventRecord(B.join, B.side));
    launches += 1;
  }

  // ---- projection of every keyframe's Gaussians into the joint arrays
  ProjBuffers pb;
  pb.p0 = as<float4>(B.p0);
  pb.p1 = as<float4>(B.p1);
  pb.p2 = as<float4>(B.p2);
  pb.rect = as<ushort4>(B.rect);
  pb.ntiles = as<uint32_t>(B.ntiles);
  pb.zkey = as<uint32_t>(B.zkey_a);
  pb.zval = as<uint32_t>(B.zval_a);
  pb.gid = as<uint32_t>(B.gid);
  pb.n_visible = d_nvis;
  pb.grad2d = as<float4>(B.grad2d);  // zeroed by the projection, for binned Gaussians only
  {
    PhaseTimer timer(c, DQO_PHASE_PROJECT, s_);
    PreTable pt;
    for (int k = 0; k < nkf; ++k) {
      pt.kf[k].rp = rp[k];
      pt.kf[k].g = kfs[k].gaussians;
      pt.kf[k].base = base[k];
    }
    DQO_CUDA(c, launch_preprocess_batch(pt, nkf, max_n, pb, s_));
    launches += 1;
  }
  // ---- depth order (one sort over all keyframes: the order restricted to a keyframe is
  // its (depth, index) order because its indices are contiguous); a sizing call then scans
  // the pair counts by depth rank here, to learn the pair total before it allocates (other
  // calls scan them inside the pair emission)
  int sel = 0;
  const uint32_t* order = nullptr;
  {
    PhaseTimer timer(c, DQO_PHASE_DEPTH_SORT, s_);
    DQO_CUDA(c, radix_sort_u32(as<uint32_t>(B.zkey_a), as<uint32_t>(B.zkey_b), as<uint32_t>(B.zval_a),
                               as<uint32_t>(B.zval_b), N, 32, as<uint32_t>(B.depth_hist), &sel, s_, nullptr,
                               d_sort_err, 0, true));
    order = sel ? as<uint32_t>(B.zval_b) : as<uint32_t>(B.zval_a);
    if (sizing) {
      DQO_CUDA(c, launch_exclusive_scan(as<uint32_t>(B.ntiles), as<uint32_t>(B.offsets), N,
                                        as<uint64_t>(B.scan_scratch), d_total, s_, d_sort_err, order, true));
      launches += scan_launches(N);
    }
    launches += radix_sort_launches(N, 32);
  }

  if (sizing) {
    DQO_CUDA(c, cudaMemcpyAsync(B.host, d_total, 8, cudaMemcpyDeviceToHost, s_));
    DQO_CUDA(c, cudaStreamSynchronize(s_));
    const uint64_t m = B.host[0];
    if (m >= (uint64_t(1) << 31)) return DQO_ENOMEM;
    const uint64_t cap = m + m / 4 + 65536;
    DQO_CUDA(c, ensure(B.pair_a, 8 * cap));
    DQO_CUDA(c, ensure(B.pair_b, 8 * cap));
    DQO_CUDA(c, ensure(B.list, 4 * cap));
    DQO_CUDA(c, ensure(B.hist, 4 * radix_scratch_words((int64_t)cap)));
    DQO_CUDA(c, ensure(B.scan_scratch, 8 * std::max({scan_scratch_words(N), scan_emit_scratch_words(N),
                                                     scan_scratch_words(radix_scratch_words((int64_t)cap))})));
    DQO_CUDA(c, ensure(B.hitrec, 4 * hit_record_words(cap, T)));
    B.capacity = cap;
    B.sig = sig;
  }
  const uint64_t cap = B.capacity;

  // ---- pairs of the joint tile numbering, pair sort, tile ranges (counts on the device)
  {
    PhaseTimer timer(c, DQO_PHASE_BINNING, s_);
    EmitTable et;
    for (int k = 0; k < nkf; ++k) {
      et.kf[k].base = base[k];
      et.kf[k].n = kfs[k].gaussians.n;
      et.kf[k].tile_off = toff[k];
      et.kf[k].ntx = rp[k].ntx;
    }
    const bool k32 = end_bit <= 32;
    // the pair sort's last pass writes the tile list and each tile's pair count, from which
    // the forward's tile schedule writes the ranges
    if (sizing)
      DQO_CUDA(c, launch_emit_pairs_batch(et, nkf, N, as<ushort4>(B.rect), as<uint32_t>(B.offsets), order,
                                          rank_bits, cap, B.pair_a.p, k32, d_overflow, d_total, d_live, s_));
    else
      DQO_CUDA(c, launch_scan_emit_pairs_batch(et, nkf, N, as<ushort4>(B.rect), order, rank_bits, cap, B.pair_a.p,
                                               k32, d_overflow, as<uint64_t>(B.scan_scratch), d_sort_err, d_total,
                                               d_live, s_));
    const PairOut po{order, as<uint32_t>(B.list), as<uint32_t>(B.tile_count), rank_bits, (uint32_t)T,
                     (uint32_t)N};
    int psel = 0;
    if (k32)
      DQO_CUDA(c, radix_sort_pairs_u32(as<uint32_t>(B.pair_a), as<uint32_t>(B.pair_b), (int64_t)cap, end_bit,
                                       as<uint32_t>(B.hist), &psel, s_, d_live, d_sort_err, rank_bits, po, !sizing));
    else
      DQO_CUDA(c, radix_sort_pairs_u64(as<uint64_t>(B.pair_a), as<uint64_t>(B.pair_b), (int64_t)cap, end_bit,
                                       as<uint32_t>(B.hist), &psel, s_, d_live, d_sort_err, rank_bits, po, !sizing));
    launches += 1 + radix_sort_launches((int64_t)cap, end_bit, rank_bits);
  }

  // ---- persistent forward + backward over all tiles, losses, projection adjoint
  {
    StepTable tt;
    PreBwdTable bt;
    for (int k = 0; k < nkf; ++k) {
      const dqo_keyframe& kf = kfs[k];
      const int64_t po = poff[k];
      BlendFwdArgs& a = tt.f[k];
      a.rp = rp[k];
      a.p0 = pb.p0;
      a.p1 = pb.p1;
      a.p2 = pb.p2;
      a.gid = pb.gid;
      a.ranges = as<uint2>(B.ranges) + toff[k];
      a.list = as<uint32_t>(B.list);
      a.t_rgb = kf.targets.rgb;
      a.t_depth = kf.targets.depth;
      a.t_gt = kf.targets.gt_id;
      a.o_rgb = kf.out.rgb;
      a.o_depth = kf.out.depth;
      a.o_alpha = kf.out.alpha;
      a.o_ins = kf.out.ins;
      a.o_id = kf.out.id_map;
      a.T_final = as<float>(B.T_final) + po;
      a.n_contrib = as<uint32_t>(B.n_contrib) + po;
      a.dl_rgb = as<float>(B.dl_rgb) + 3 * po;
      a.dl_depth = as<float>(B.dl_depth) + po;
      a.dl_ins = as<float>(B.dl_ins) + po;
      a.loss_part = as<float>(B.loss_part) + 3 * (int64_t)toff[k];
      a.o_mask = kf.out.update_mask;
      a.tile_order = as<uint32_t>(B.tile_sched) + toff[k];
      a.tile_cost = as<uint32_t>(B.tile_sched) + T + kTileParts * (uint64_t)toff[k];
      a.hitmask = as<uint32_t>(B.hitrec) + 8 * (uint64_t)toff[k];  // joint tile numbering
      BlendBwdArgs& bb = tt.b[k];
      bb.rp = rp[k];
      bb.p0 = pb.p0;
      bb.p1 = pb.p1;
      bb.p2 = pb.p2;
      bb.ranges = a.ranges;
      bb.list = a.list;
      bb.t_gt = kf.targets.gt_id;
      bb.T_final = a.T_final;
      bb.n_contrib = a.n_contrib;
      bb.g_rgb = a.dl_rgb;
      bb.g_depth = a.dl_depth;
      bb.g_alpha = nullptr;
      bb.g_ins = a.dl_ins;
      bb.grad2d = as<float>(B.grad2d);
      bb.tile_order = as<uint32_t>(B.tile_sched) + (1 + kTileParts) * T + kTileParts * (uint64_t)toff[k];
      bb.hitmask = a.hitmask;
      tt.tile_off[k] = toff[k];
      LossKf& lk = bt.loss[k];
      lk.part = a.loss_part;
      lk.tiles = (int)(toff[k + 1] - toff[k]);
      lk.lambda_ins = rp[k].lambda_ins;
      lk.scale = (float)(1.0 / ((double)rp[k].W * (double)rp[k].H));
      lk.loss = kf.out.loss;
      PreBwdArgs& pa = bt.kf[k];
      pa.rp = rp[k];
      pa.n = kf.gaussians.n;
      pa.means = kf.gaussians.means;
      pa.log_scales = kf.gaussians.log_scales;
      pa.quats = kf.gaussians.quats;
      pa.opacity_logit = kf.gaussians.opacity_logit;
      pa.ntiles = as<uint32_t>(B.ntiles) + base[k];
      pa.grad2d = as<float>(B.grad2d) + 12 * base[k];
      pa.d_means = kf.grads.means;
      pa.d_log_scales = kf.grads.log_scales;
      pa.d_quats = kf.grads.quats;
      pa.d_logit = kf.grads.opacity_logit;
      pa.d_rgb = kf.grads.rgb;
      // gradients are added atomically (keyframes may share buffers); with grads_zero a
      // keyframe whose buffers no other keyframe uses overwrites them, shared ones were
      // cleared at the start
      bool shared = false;
      for (int j = 0; j < nkf; ++j)
        if (j != k && grads_share(kfs[j].grads, kf.grads)) shared = true;
      pa.mode = s->grads_zero && !shared ? kGradStore : kGradAtomic;
    }
    tt.tile_off[nkf] = toff[nkf];
    tt.nkf = nkf;
    tt.tile_count = as<uint32_t>(B.tile_count);
    {
      PhaseTimer timer(c, DQO_PHASE_BLEND_STEP, s_);
      const BlendCommon cm{pb.p0, pb.p1, pb.p2, pb.gid, as<uint32_t>(B.list), as<float>(B.grad2d), s->alpha_clamp,
                           s->alpha_min, s->t_stop, s->og_filter ? 1 : 0};
      DQO_CUDA(c, launch_blend_step(tt, cm, d_queue, s->tile_w, with_id, ctas_per_sm, B.sms, schedule, s_));
    }
    {
      PhaseTimer timer(c, DQO_PHASE_PROJECT_BWD, s_);
      DQO_CUDA(c, launch_preprocess_backward_batch(bt, nkf, max_n, s_));
    }
    launches += 1 + (schedule == 0 ? 2 : schedule == 1 ? 4 : 2 * nkf + 2);
  }
  if (run_fits) DQO_CUDA(c, cudaStreamWaitEvent(s_, B.join, 0));
  c->launches += launches;
  return DQO_OK;
}

dqo_status dqo_batch_check(dqo_ctx* c, uint64_t* pairs, int* overflow) {
  if (!c) return DQO_EINVAL;
  if (pairs) *pairs = 0;
  if (overflow) *overflow = 0;
  if (!c->b.counters.p) return DQO_OK;
  DQO_CUDA(c, cudaSetDevice(c->device));
  DQO_CUDA(c, cudaDeviceSynchronize());
  uint64_t h[4] = {0, 0, 0, 0};
  DQO_CUDA(c, cudaMemcpy(h, c->b.counters.p, 32, cudaMemcpyDeviceToHost));
  const int over = (int)(h[1] >> 32) != 0;
  if (pairs) *pairs = h[0];
  if (overflow) *overflow = over;
  if (over) c->b.capacity = 0;  // the next step sizes again
  return (h[3] & 0xFFFFFFFFu) ? DQO_ETIMEOUT : DQO_OK;
}

dqo_status dqo_batch_tune(dqo_ctx* c, dqo_settings* s, int32_t nkf, const dqo_keyframe* kfs,
                          const dqo_fit_batch* fits, int32_t reps, int32_t* ctas_per_sm, int32_t* schedule, float* ms,
                          dqo_stream stream_) {
  if (!c || !s || !ctas_per_sm || !schedule || reps < 1) return DQO_EINVAL;
  static const int shapes[3][2] = {{16, 16}, {8, 32}, {32, 8}};
  cudaStream_t s_ = reinterpret_cast<cudaStream_t>(stream_);
  DQO_CUDA(c, cudaSetDevice(c->device));
  cudaEvent_t e0, e1;
  DQO_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DQO_ECUDA;
  }
  float best = 0.f;
  int best_i = -1;
  dqo_status st = DQO_OK;
  auto cand = [](int i, int* cps, int* sched) {
    const int j = i % 7;
    *sched = j < 3 ? DQO_SCHEDULE_FUSED : (j < 6 ? DQO_SCHEDULE_SPLIT : DQO_SCHEDULE_PER_KEYFRAME);
    *cps = j < 3 ? 2 + j : (j < 6 ? j - 1 : 0);
  };
  for (int i = 0; i < DQO_TUNE_CANDIDATES && st == DQO_OK; ++i) {
    dqo_settings t = *s;
    t.tile_w = shapes[i / 7][0];
    t.tile_h = shapes[i / 7][1];
    int cps, sched;
    cand(i, &cps, &sched);
    st = dqo_batch_step(c, &t, nkf, kfs, fits, cps, sched, stream_);  // warm-up (sizes the layout)
    if (st != DQO_OK) break;
    cudaEventRecord(e0, s_);
    for (int r = 0; r < reps && st == DQO_OK; ++r) st = dqo_batch_step(c, &t, nkf, kfs, fits, cps, sched, stream_);
    cudaEventRecord(e1, s_);
    if (st != DQO_OK) break;
    float t_ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess) {
      st = DQO_ECUDA;
      break;
    }
    t_ms /= (float)reps;
    if (ms) ms[i] = t_ms;
    if (best_i < 0 || t_ms < best) {
      best = t_ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DQO_OK) return st;
  s->tile_w = shapes[best_i / 7][0];
  s->tile_h = shapes[best_i / 7][1];
  cand(best_i, ctas_per_sm, schedule);
  return DQO_OK;
}

dqo_status dqo_quadric_canonical(int32_t nq, const float* params, float* out, dqo_stream stream_) {
  if (nq < 0 || (nq > 0 && (!params || !out))) return DQO_EINVAL;
  if (launch_quadric_canonical(nq, params, out, reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess)
    return DQO_ECUDA;
  return DQO_OK;
}

// ----------------------------------------------------------------------------- learned proposal

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kParamBytes = align_up(sizeof(float) * kMlpParams);
constexpr size_t kW128Bytes = align_up(2 * kMlpHidden * kMlpHidden);
constexpr size_t kW3Bytes = align_up(2 * kMlpOutPad * kMlpHidden);
constexpr size_t kStateBytes = 4 * kParamBytes + 2 * kW128Bytes + kW3Bytes + kAlign;

MlpState state_view(const void* state) {
  unsigned char* b = static_cast<unsigned char*>(const_cast<void*>(state));
  MlpState st;
  st.param = reinterpret_cast<float*>(b);
  st.grad = reinterpret_cast<float*>(b + kParamBytes);
  st.m1 = reinterpret_cast<float*>(b + 2 * kParamBytes);
  st.m2 = reinterpret_cast<float*>(b + 3 * kParamBytes);
  b += 4 * kParamBytes;
  st.w1b = reinterpret_cast<__nv_bfloat16*>(b);
  st.w2b = reinterpret_cast<__nv_bfloat16*>(b + kW128Bytes);
  b += 2 * kW128Bytes;
  st.w3b = reinterpret_cast<__nv_bfloat16*>(b);
  st.step = reinterpret_cast<int*>(b + kW3Bytes);
  return st;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Workspace for batches of up to n rows (n rounded up to 128); sets up the GEMM kernels'
// shared-memory limit on first use.
dqo_status mlp_work(dqo_ctx* c, int64_t n, MlpWork* wk) {
  if (!c->mlp_ready) {
    DQO_CUDA(c, mlp_gemm_setup());
    c->mlp_ready = true;
  }
  // the layout follows the largest batch seen, so the error flag keeps its place
  const int64_t nn = std::max((n + 127) / 128 * 128, c->mlp_n);
  const size_t big = align_up((size_t)nn * kMlpHidden * 2);
  const size_t part = align_up((size_t)(nn / 128) * kMlpParams * sizeof(float));
  const size_t bytes = 2 * big + kAlign + part;
  const bool grow = nn > c->mlp_n;
  DQO_CUDA(c, ensure(c->mlp_work, bytes));
  unsigned char* b = as<unsigned char>(c->mlp_work);
  wk->h1 = reinterpret_cast<__nv_bfloat16*>(b);
  wk->h2 = reinterpret_cast<__nv_bfloat16*>(b + big);
  wk->err = reinterpret_cast<int*>(b + 2 * big);
  wk->bar = reinterpret_cast<unsigned*>(b + 2 * big + 64);
  wk->gpart = reinterpret_cast<float*>(b + 2 * big + kAlign);
  if (grow) DQO_CUDA(c, cudaMemset(wk->err, 0, sizeof(int)));
  c->mlp_n = nn;
  return DQO_OK;
}

dqo_status check_batch(int64_t n, const uint16_t* X, const float* labels) {
  if (n <= 0 || n % 128 != 0 || n > (int64_t(1) << 30)) return DQO_EINVAL;
  if (!X || !labels || !aligned16(X) || !aligned16(labels)) return DQO_EINVAL;
  return DQO_OK;
}

}  // namespace

dqo_status dqo_mlp_features(int32_t nq, int32_t nv, const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                            int32_t npairs, const float* obs, const int32_t* counts, float length_scale,
                            uint16_t* X, uint16_t* XT, int64_t ldt, dqo_stream stream_) {
  if (nq < 0 || nv < 0 || npairs < 0 || !(length_scale > 0.f)) return DQO_EINVAL;
  if (nq == 0) return DQO_OK;
  if (!q_ptr || !X || !aligned16(X)) return DQO_EINVAL;
  if (npairs > 0 && (!P || !pair_v || !obs || nv == 0)) return DQO_EINVAL;
  if (XT && (ldt < nq || ldt % 8 != 0)) return DQO_EINVAL;
  if (launch_mlp_features(nq, nv, P, q_ptr, pair_v, npairs, obs, counts, 1.f / length_scale, X, XT, ldt,
                          reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess)
    return DQO_ECUDA;
  return DQO_OK;
}

size_t dqo_mlp_state_bytes(void) { return kStateBytes; }

dqo_status dqo_mlp_set_params(void* state, const float* params, dqo_stream stream_) {
  if (!state || !params || (reinterpret_cast<uintptr_t>(state) % kAlign) != 0) return DQO_EINVAL;
  if (launch_mlp_set(state_view(state), params, reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess)
    return DQO_ECUDA;
  return DQO_OK;
}

dqo_status dqo_mlp_get_params(const void* state, float* params, dqo_stream stream_) {
  if (!state || !params || (reinterpret_cast<uintptr_t>(state) % kAlign) != 0) return DQO_EINVAL;
  if (cudaMemcpyAsync(params, state_view(state).param, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice,
                      reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess)
    return DQO_ECUDA;
  return DQO_OK;
}

dqo_status dqo_mlp_forward(dqo_ctx* c, const void* state, int64_t n, const uint16_t* X, float* out,
                           dqo_stream stream_) {
  if (!c || !state || n < 0 || n > (int64_t(1) << 30) || (reinterpret_cast<uintptr_t>(state) % kAlign) != 0)
    return DQO_EINVAL;
  if (n == 0) return DQO_OK;
  if (!X || !out || !aligned16(X)) return DQO_EINVAL;
  DQO_CUDA(c, cudaSetDevice(c->device));
  MlpWork wk;
  dqo_status st = mlp_work(c, n, &wk);
  if (st != DQO_OK) return st;
  DQO_CUDA(c, launch_mlp_forward(state_view(state), wk, n, X, out, reinterpret_cast<cudaStream_t>(stream_)));
  c->launches += 3;
  return DQO_OK;
}

dqo_status dqo_mlp_gradients(dqo_ctx* c, void* state, int64_t n, const uint16_t* X, const float* labels,
                             const float* loss_w, float* grads, float* loss, dqo_stream stream_) {
  if (!c || !state || !loss_w || !grads || !loss || (reinterpret_cast<uintptr_t>(state) % kAlign) != 0 ||
      !aligned16(grads))
    return DQO_EINVAL;
  dqo_status st = check_batch(n, X, labels);
  if (st != DQO_OK) return st;
  DQO_CUDA(c, cudaSetDevice(c->device));
  MlpWork wk;
  if ((st = mlp_work(c, n, &wk)) != DQO_OK) return st;
  dqo_mlp_hparams hp{};
  for (int j = 0; j < 9; ++j) hp.loss_w[j] = loss_w[j];
  DQO_CUDA(c, launch_mlp_train(state_view(state), hp, true, 1, n, X, labels, loss, grads, wk,
                               reinterpret_cast<cudaStream_t>(stream_)));
  c->launches += 1;
  return DQO_OK;
}

dqo_status dqo_mlp_train_steps(dqo_ctx* c, void* state, const dqo_mlp_hparams* hp, int32_t steps, int64_t batch,
                               const uint16_t* X, const float* labels, float* losses, dqo_stream stream_) {
  if (!c || !state || !hp || steps < 0 || (reinterpret_cast<uintptr_t>(state) % kAlign) != 0) return DQO_EINVAL;
  if (!(hp->lr >= 0.f) || !(hp->lr_final >= 0.f) || !(hp->beta1 >= 0.f && hp->beta1 < 1.f) ||
      !(hp->beta2 >= 0.f && hp->beta2 < 1.f) || !(hp->eps > 0.f))
    return DQO_EINVAL;
  if (steps == 0) return DQO_OK;
  if (batch <= 0 || (int64_t)steps * batch > (int64_t(1) << 30)) return DQO_EINVAL;
  dqo_status st = check_batch(batch, X, labels);
  if (st != DQO_OK) return st;
  DQO_CUDA(c, cudaSetDevice(c->device));
  MlpWork wk;
  if ((st = mlp_work(c, batch, &wk)) != DQO_OK) return st;
  DQO_CUDA(c, launch_mlp_train(state_view(state), *hp, false, steps, batch, X, labels, losses, nullptr, wk,
                               reinterpret_cast<cudaStream_t>(stream_)));
  c->launches += 1;
  return DQO_OK;
}

dqo_status dqo_mlp_train_step(dqo_ctx* c, void* state, const dqo_mlp_hparams* hp, int64_t n, const uint16_t* X,
                              const float* labels, float* loss, dqo_stream stream_) {
  return dqo_mlp_train_steps(c, state, hp, 1, n, X, labels, loss, stream_);
}

dqo_status dqo_mlp_check(dqo_ctx* c, int* timed_out) {
  if (!c || !timed_out) return DQO_EINVAL;
  *timed_out = 0;
  if (!c->mlp_work.p) return DQO_OK;
  DQO_CUDA(c, cudaSetDevice(c->device));
  MlpWork wk;
  dqo_status st = mlp_work(c, c->mlp_n, &wk);
  if (st != DQO_OK) return st;
  int v = 0;
  DQO_CUDA(c, cudaMemcpy(&v, wk.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) DQO_CUDA(c, cudaMemset(wk.err, 0, sizeof(int)));
  *timed_out = v;
  return v ? DQO_ETIMEOUT : DQO_OK;
}

dqo_status dqo_wait_probe(dqo_ctx* c, dqo_stream stream_) {
  if (!c) return DQO_EINVAL;
  DQO_CUDA(c, cudaSetDevice(c->device));
  int* flag = nullptr;   // the probe's flag word and its grid-barrier counter
  DQO_CUDA(c, cudaMalloc(&flag, 2 * sizeof(int)));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  int v = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = launch_bounded_wait_probe(flag, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(flag);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->launches += 1;
  return v == 3 ? DQO_ETIMEOUT : DQO_OK;   // both waits gave up
}

}  // extern "C"
