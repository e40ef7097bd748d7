// Binning and sorting (K2-K5): exclusive scan, LSD radix sort (one kernel per 8-bit digit,
// decoupled look-back), pair emission and tile ranges.  The tile lists the blend kernels walk are ordered by (tile, depth, index):
//   1. the Gaussians are radix-sorted once by the bit pattern of their (positive) camera
//      depth, stable on the index, which gives each visible Gaussian a depth rank;
//   2. every (tile, Gaussian) pair gets the key (tile << rank_bits) | rank -- unique, so a
//      plain radix sort of these keys yields (tile, depth bits, index) order with no
//      values carried along;
//   3. tile ranges are read off the sorted keys and ranks mapped back to indices.
// Keys are 32-bit when tile and rank bits fit, else 64-bit.
#include <atomic>

#include "dqo_internal.cuh"

namespace dqo {
namespace {

// ---------------------------------------------------------------- block-wide scan helpers

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan across the CTA of one value per thread; returns the CTA total.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T& total) {
  __shared__ T warp_tot[kThreads / 32 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T inc = warp_inclusive_scan(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T t = lane < kThreads / 32 ? warp_tot[lane] : T(0);
    const T ti = warp_inclusive_scan(t);
    if (lane < kThreads / 32) warp_tot[lane] = ti - t;
    if (lane == kThreads / 32 - 1) warp_tot[kThreads / 32] = ti;  // spare slot: see size below
  }
  __syncthreads();
  const T ex = warp_tot[warp] + inc - v;
  total = warp_tot[kThreads / 32];
  __syncthreads();
  return ex;
}

__device__ __forceinline__ uint64_t scan_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Single-pass exclusive scan with decoupled look-back: CTAs take tiles of kScanTile values from
// an atomic counter, scan their tile, publish its sum (64-bit word: 2 flag bits, 62 value
// bits) and add their predecessors' published sums back to the first inclusive prefix;
// the last tile writes the total.  Waits give up after about a second (err).
constexpr uint64_t kScanAgg = 1ull << 62, kScanInc = 2ull << 62, kScanMask = (1ull << 62) - 1;

// Warp 0 of a look-back CTA: publishes tile `tile`'s sum tot, adds the predecessors' published
// sums back to the first inclusive prefix, 32 at a time (lane j reads tile p - j; the words
// up to the nearest unpublished one are added, and the walk ends at the nearest inclusive
// one), publishes the tile's inclusive prefix and returns its exclusive prefix on every
// lane.  Tiles are numbered in the order their CTAs started, so every wait is on a running
// CTA; a wait still gives up after about a second (err = 1, prefix incomplete).
__device__ __forceinline__ uint64_t scan_lookback(uint64_t* __restrict__ status, uint32_t tile, uint64_t tot,
                                                  uint32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  volatile uint64_t* st = status;
  if (lane == 0) st[tile] = (tile == 0 ? kScanInc : kScanAgg) | tot;
  uint64_t excl = 0;
  if (tile > 0) {
    int64_t p = (int64_t)tile - 1;
    const uint64_t t0 = scan_ns();
    uint32_t it = 0;
    for (;;) {
      const uint64_t w = p - lane >= 0 ? (uint64_t)st[p - lane] : (uint64_t)kScanInc;   // before tile 0: an empty prefix
      const uint64_t f = w & ~kScanMask;
      const uint32_t unready = __ballot_sync(0xFFFFFFFFu, f == 0);
      const uint32_t inc = __ballot_sync(0xFFFFFFFFu, f == kScanInc);
      const uint32_t stop = unready | inc;
      const int first = stop ? __ffs(stop) - 1 : 32;
      const bool finish = first < 32 && ((inc >> first) & 1u);
      const int take = finish ? first + 1 : first;
      uint64_t v = lane < take ? (w & kScanMask) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      excl += v;
      if (finish) break;
      p -= take;
      if (take == 0 && (++it & 63u) == 0u) {
        const bool late = __shfl_sync(0xFFFFFFFFu, lane == 0 && scan_ns() - t0 > 1000000000ull, 0);
        if (late) {
          if (lane == 0) atomicExch(err, 1u);
          break;
        }
      }
    }
    if (lane == 0) st[tile] = kScanInc | (excl + tot);
  }
  return excl;
}

__global__ void __launch_bounds__(kThreads) k_scan_lookback(const uint32_t* __restrict__ in,
                                                            const uint32_t* __restrict__ gather,
                                                            uint32_t* __restrict__ out, int64_t n,
                                                            uint64_t* __restrict__ status,
                                                            uint32_t* __restrict__ counter,
                                                            uint32_t* __restrict__ err, uint64_t* __restrict__ total) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t tile_s[kScanTile];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t base = (int64_t)tile * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    tile_s[k * kThreads + threadIdx.x] = i < n ? in[gather ? gather[i] : i] : 0u;
  }
  __syncthreads();
  uint32_t v[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = tile_s[threadIdx.x * kScanItems + k];
    sum += v[k];
  }
  uint32_t tot;
  uint32_t run = block_exclusive_scan<uint32_t>(sum, tot);
  if (threadIdx.x < 32) {
    const uint64_t excl = scan_lookback(status, tile, tot, err);
    if (threadIdx.x == 0) {
      s_prefix = excl;
      if (total && base + kScanTile >= n) *total = excl + tot;
    }
  }
  __syncthreads();
  run += (uint32_t)s_prefix;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile_s[threadIdx.x * kScanItems + k] = run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n) out[i] = tile_s[k * kThreads + threadIdx.x];
  }
}

// ---------------------------------------------------------------- LSD radix sort passes

// Element count: n, or the smaller of n and *n_dev when the count lives on the device
// (launches sized for a capacity n).
__device__ __forceinline__ int64_t live_count(int64_t n, const uint64_t* n_dev) {
  if (!n_dev) return n;
  const uint64_t d = *n_dev;
  return d < (uint64_t)n ? (int64_t)d : n;
}

// Single-pass-per-digit LSD radix sort with decoupled look-back.  One kernel counts the
// digits of every pass at once into global histograms; then each pass is one kernel whose
// CTAs take tile indices from an atomic counter (so a CTA's predecessors have all started),
// rank their keys locally and stably, publish their per-digit counts, and find their
// global offsets by looking back over their predecessors' published counts: a
// predecessor's word is an aggregate (its own count) or an inclusive prefix (everything up
// to and including it), flag and count in one 32-bit word.  Every CTA publishes before it
// waits, so each wait is on a CTA that is running; the wait still gives up after about a
// second and raises an error flag instead of hanging.

constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kCountMask = (1u << 30) - 1;
constexpr int kLookBatch = 8;   // predecessors a digit's look-back reads per round trip

// Digit histograms of every pass; the last block to finish turns them into each pass's
// exclusive digit offsets gex[pass][digit] (done: a block counter, zero before the launch).
template <typename K, int IPT>
__global__ void __launch_bounds__(kThreads) k_onesweep_hist(const K* __restrict__ keys, int64_t n_cap,
                                                            const uint64_t* __restrict__ n_dev, int begin_bit,
                                                            int passes, uint32_t* __restrict__ ghist,
                                                            uint32_t* __restrict__ gex, uint32_t* __restrict__ done) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t h[kMaxRadixPasses][kRadixBins];
  for (int i = threadIdx.x; i < passes * kRadixBins; i += kThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = live_count(n_cap, n_dev);
  const int64_t base = (int64_t)blockIdx.x * (kThreads * IPT);
  K key[IPT];
#pragma unroll
  for (int k = 0; k < IPT; ++k) {   // the loads first, all in flight together
    const int64_t i = base + k * kThreads + threadIdx.x;
    key[k] = i < n ? keys[i] : K(0);
  }
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int64_t i = base + k * kThreads + threadIdx.x;
    if (i < n)
      for (int p = 0; p < passes; ++p)
        atomicAdd(&h[p][(uint32_t)(key[k] >> (begin_bit + p * kRadixBits)) & (kRadixBins - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadixBins; i += kThreads) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(ghist + i, c);
  }
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int p = 0; p < passes; ++p) {   // kThreads == kRadixBins: thread t owns digit t
    uint32_t tot;
    gex[p * kRadixBins + threadIdx.x] =
        block_exclusive_scan<uint32_t>(__ldcg(ghist + p * kRadixBins + threadIdx.x), tot);
  }
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One pass.  gex_in: this pass's 256 global digit starts; status: [tiles][256] words, zero
// before the pass; counter: this pass's tile counter, zero before the pass.  rank (optional,
// with values): rank[value] = destination.  err: set to 1 if a look-back wait gave up.
template <typename K, bool kVals, int IPT>
__global__ void __launch_bounds__(kThreads, 3) k_onesweep_pass(const K* __restrict__ kin, K* __restrict__ kout,
                                                            const uint32_t* __restrict__ vin,
                                                            uint32_t* __restrict__ vout, int64_t n_cap,
                                                            const uint64_t* __restrict__ n_dev, int shift,
                                                            const uint32_t* __restrict__ gex_in,
                                                            uint32_t* __restrict__ status,
                                                            uint32_t* __restrict__ counter,
                                                            uint32_t* __restrict__ rank, uint32_t* __restrict__ err,
                                                            const PairOut po) {
  __shared__ uint32_t cnt[kThreads / 32][kRadixBins];
  __shared__ uint32_t s_base[kRadixBins], s_lstart[kRadixBins];
  __shared__ K s_key[kThreads * IPT];
  __shared__ uint32_t s_val[kVals ? kThreads * IPT : 1];
  __shared__ uint32_t s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = threadIdx.x;
  // the tile index and the counters do not depend on the previous kernel: taken while it
  // drains (the counter was cleared before the sort's first kernel)
  if (t == 0) s_tile = atomicAdd(counter, 1u);
  for (int d = t; d < (kThreads / 32) * kRadixBins; d += kThreads) (&cnt[0][0])[d] = 0;
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t n = live_count(n_cap, n_dev);
  // tiles past the live count (launches sized for a capacity) have nothing to do; every tile
  // after them is empty too, so no look-back ever reads their status
  if ((int64_t)tile * (kThreads * IPT) >= n && tile > 0) return;
  const uint32_t gex = gex_in[t];   // the digit's global start (exclusive scan of the histogram)
  const int64_t wbase = (int64_t)tile * (kThreads * IPT) + (int64_t)warp * 32 * IPT;
  K key[IPT];
  uint32_t val[IPT];
  uint32_t pos[IPT];
  const uint32_t lt = lanemask_lt();
  // every load of the tile first (all in flight together), then the ranking
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool ok = i < n;
    key[r] = ok ? kin[i] : K(0);
    if (kVals) val[r] = ok ? vin[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool ok = i < n;
    const uint32_t d = (uint32_t)(key[r] >> shift) & (kRadixBins - 1);
    const uint32_t active = __ballot_sync(0xFFFFFFFFu, ok);
    uint32_t peers = __match_any_sync(0xFFFFFFFFu, ok ? d : 0xFFFFFFFFu);
    peers &= active;
    const uint32_t before = cnt[warp][d];
    __syncwarp();
    if (ok) {
      pos[r] = before + __popc(peers & lt);
      const int leader = __ffs(peers) - 1;
      if (lane == leader) cnt[warp][d] = before + __popc(peers);
    } else {
      pos[r] = 0xFFFFFFFFu;
    }
    __syncwarp();
  }
  __syncthreads();
  // thread t owns digit t: offsets of the warps within the tile, and the tile's count
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    const uint32_t c = cnt[w][t];
    cnt[w][t] = total;
    total += c;
  }
  volatile uint32_t* st = status;
  st[(int64_t)tile * kRadixBins + t] = (tile == 0 ? kFlagInc : kFlagAgg) | total;
  // the digit's start within the tile (keys of the tile in digit order)
  uint32_t tile_n;
  s_lstart[t] = block_exclusive_scan<uint32_t>(total, tile_n);
  __syncthreads();   // every digit's start is read below
  // stage the tile's keys in digit order (local information only, so before the look-back,
  // which then holds few registers); each digit's run is written out contiguously below
  // (consecutive threads, consecutive addresses) instead of one scattered key per lane
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    if (pos[r] == 0xFFFFFFFFu) continue;
    const uint32_t d = (uint32_t)(key[r] >> shift) & (kRadixBins - 1);
    const uint32_t li = s_lstart[d] + cnt[warp][d] + pos[r];
    s_key[li] = key[r];
    if (kVals) s_val[li] = val[r];
  }
  uint32_t excl = 0;
  if (tile > 0) {
    // kLookBatch predecessors per round trip (independent loads in flight together): the
    // words up to the nearest unpublished one are added, the walk ends at the nearest
    // inclusive one
    int64_t p = (int64_t)tile - 1;
    const uint64_t t0 = global_ns();
    uint32_t it = 0;
    for (;;) {
      uint32_t w[kLookBatch];
#pragma unroll
      for (int k = 0; k < kLookBatch; ++k)
        w[k] = p - k >= 0 ? (uint32_t)st[(p - k) * kRadixBins + t] : (uint32_t)kFlagInc;   // before tile 0: empty
      int used = 0;
      bool done = false, stalled = false;
#pragma unroll
      for (int k = 0; k < kLookBatch; ++k) {
        if (done || stalled) continue;
        const uint32_t f = w[k] & ~kCountMask;
        if (f == 0u) {
          stalled = true;
          continue;
        }
        excl += w[k] & kCountMask;
        ++used;
        done = f == kFlagInc;
      }
      if (done) break;
      p -= used;
      if (used == 0 && (++it & 63u) == 0u && global_ns() - t0 > 1000000000ull) {
        atomicExch(err, 1u);
        break;
      }
    }
    st[(int64_t)tile * kRadixBins + t] = kFlagInc | (excl + total);
  }
  s_base[t] = gex + excl;
  __syncthreads();
  for (uint32_t j = t; j < tile_n; j += kThreads) {
    const K k = s_key[j];
    const uint32_t d = (uint32_t)(k >> shift) & (kRadixBins - 1);
    const uint32_t dst = s_base[d] + (j - s_lstart[d]);
    if (po.list) {
      // the last pass of a pair sort: the tile list, and per tile run of this CTA (its keys
      // are staged in digit order, so a tile's keys are contiguous here and at dst) the run
      // length, added as (last + 1) - first by the run's two ends; the sorted keys
      // themselves are not needed afterwards
      const uint32_t tile = (uint32_t)(k >> po.rank_bits);
      const uint32_t r = (uint32_t)(k & (((K)1 << po.rank_bits) - 1));
      if (tile >= po.tiles) continue;   // defensive: every live key was emitted in range
      if (dst < (uint32_t)n && r < po.n_order) po.list[dst] = po.order[r];
      if (j == 0 || (uint32_t)(s_key[j - 1] >> po.rank_bits) != tile) atomicAdd(po.counts + tile, 0u - j);
      if (j + 1 == tile_n || (uint32_t)(s_key[j + 1] >> po.rank_bits) != tile) atomicAdd(po.counts + tile, j + 1);
      continue;
    }
    kout[dst] = k;
    if (kVals) {
      const uint32_t v = s_val[j];
      vout[dst] = v;
      if (rank) rank[v] = dst;
    }
  }
}

// ---------------------------------------------------------------- binning helpers

__global__ void k_rank_scatter(const uint32_t* __restrict__ order, int64_t n, uint32_t* __restrict__ rank) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) rank[order[r]] = (uint32_t)r;
}

// The CTA writes the pairs of its Gaussians together: thread l holds one Gaussian's tile
// rectangle, first pair offset, pair count (0: none) and rank; pair k of a Gaussian is the
// tile (k / w, k % w) of its rectangle, row-major.  A Gaussian with at least kBigPairs pairs
// goes to a shared list that the whole CTA then writes one Gaussian at a time (consecutive
// threads, consecutive pairs), so the largest footprint costs its pairs / kThreads steps.
// The other Gaussians of a warp are numbered together, 0 .. small - 1 in lane order (a
// prefix over their counts), and each lane writes every 32nd: pair j belongs to the last lane
// whose prefix is <= j (a five-step search over the prefixes).  Called by every thread.
constexpr uint32_t kBigPairs = 64;

template <typename K>
struct BigEmit {
  uint64_t o;
  K rk;
  uint32_t cnt, w, t0, nt;
  float iw;
};

// row q = floor(k / w): (k + 1/2) / w is at least 1/(2w) from an integer, so the float
// product (relative error below 2^-22) rounds to q for k < 2^21; exact division past it
template <typename K>
__device__ __forceinline__ K pair_key(uint32_t k, uint32_t w, float iw, uint32_t t0, uint32_t nt, K rk,
                                      int rank_bits) {
  const uint32_t q = k < (1u << 21) ? __float2uint_rz(((float)k + 0.5f) * iw) : k / w;
  return ((K)(t0 + q * nt + (k - q * w)) << rank_bits) | rk;
}

template <typename K>
__device__ __forceinline__ void cta_emit(const ushort4 r, const uint64_t o, const uint32_t cnt, const K rk,
                                         uint32_t tile_off, int ntx, int rank_bits, K* __restrict__ keys) {
  __shared__ BigEmit<K> s_big[kThreads];
  __shared__ uint32_t s_nbig;
  const int lane = threadIdx.x & 31;
  const uint32_t w = cnt ? (uint32_t)(r.z - r.x) : 1u;
  const float inv_w = 1.f / (float)w;
  const uint32_t first_tile = tile_off + (uint32_t)r.y * (uint32_t)ntx + (uint32_t)r.x;
  if (threadIdx.x == 0) s_nbig = 0;
  __syncthreads();
  const bool big = cnt >= kBigPairs;
  if (big) s_big[atomicAdd(&s_nbig, 1u)] = BigEmit<K>{o, rk, cnt, w, first_tile, (uint32_t)ntx, inv_w};
  // the warp's small Gaussians
  const uint32_t sc = big ? 0u : cnt;
  uint32_t inc = sc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += u;
  }
  const uint32_t ex = inc - sc;                                // this lane's first small pair
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
  for (uint32_t base = 0; base < total; base += 32) {       // uniform over the warp
    const uint32_t j = base + lane;
    int own = 0;                                               // the last lane with prefix <= j
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
      if (__shfl_sync(0xFFFFFFFFu, ex, own + step) <= j) own += step;
    const uint32_t k = j - __shfl_sync(0xFFFFFFFFu, ex, own);
    const uint32_t wo = __shfl_sync(0xFFFFFFFFu, w, own);
    const float iw = __shfl_sync(0xFFFFFFFFu, inv_w, own);
    const uint32_t t0 = __shfl_sync(0xFFFFFFFFu, first_tile, own);
    const uint32_t nt = __shfl_sync(0xFFFFFFFFu, (uint32_t)ntx, own);
    const uint64_t oo = __shfl_sync(0xFFFFFFFFu, o, own);
    const K ro = __shfl_sync(0xFFFFFFFFu, rk, own);
    if (j < total) keys[oo + k] = pair_key<K>(k, wo, iw, t0, nt, ro, rank_bits);
  }
  // the CTA's large Gaussians, by every thread
  __syncthreads();
  const uint32_t nbig = s_nbig;
  for (uint32_t b = 0; b < nbig; ++b) {
    const BigEmit<K> e = s_big[b];
    for (uint32_t k = threadIdx.x; k < e.cnt; k += kThreads)
      keys[e.o + k] = pair_key<K>(k, e.w, e.iw, e.t0, e.nt, e.rk, rank_bits);
  }
}

// Pairs in depth order: thread r emits the pairs of the Gaussian of depth rank r,
// i = order[r], at offsets[r] (the exclusive scan of tile counts in rank order).  Pairs
// thus come out ordered by rank, and a stable sort on the tile bits alone groups them by
// tile with each tile's Gaussians front to back.
template <typename K>
__global__ void __launch_bounds__(kThreads) k_emit_pairs(const ushort4* __restrict__ rect,
                                                         const uint32_t* __restrict__ offsets,
                                                         const uint32_t* __restrict__ order, int64_t n, int ntx,
                                                         int rank_bits, K* __restrict__ keys) {
  pdl_wait();
  pdl_trigger();
  const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  ushort4 q = make_ushort4(0, 0, 0, 0);
  uint64_t o = 0;
  uint32_t cnt = 0;
  if (r < n) {
    q = rect[order[r]];
    if (q.z > q.x && q.w > q.y) {
      o = offsets[r];
      cnt = (uint32_t)(q.z - q.x) * (uint32_t)(q.w - q.y);
    }
  }
  cta_emit<K>(q, o, cnt, (K)r, 0u, ntx, rank_bits, keys);
}

// The same over a batch of keyframes (joint rank r of all keyframes' Gaussians; the
// Gaussian's keyframe k is found from the global index ranges [base, base + n)); its
// tiles are tile_off + ty * ntx + tx of the batch's joint tile numbering.  Pairs past
// `capacity` are not written; *overflow is set instead.  *live (all ones before) becomes
// the smaller of the pair count *total and the first pair not written: the count the pair
// sort reads, so that it sees only pairs of this call.
template <typename K>
__global__ void __launch_bounds__(kThreads) k_emit_pairs_batch(const __grid_constant__ EmitTable t, int nkf,
                                                               const ushort4* __restrict__ rect,
                                                               const uint32_t* __restrict__ offsets,
                                                               const uint32_t* __restrict__ order, int64_t n,
                                                               int rank_bits, uint64_t capacity, K* __restrict__ keys,
                                                               uint32_t* __restrict__ overflow,
                                                               const unsigned long long* __restrict__ total,
                                                               unsigned long long* __restrict__ live) {
  pdl_wait();
  pdl_trigger();
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMin(live, *total);
  const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  ushort4 q = make_ushort4(0, 0, 0, 0);
  uint64_t o = 0;
  uint32_t cnt = 0;
  int k = 0;
  if (r < n) {
    const int64_t gi = order[r];
    while (k + 1 < nkf && t.kf[k + 1].base <= gi) ++k;
    q = rect[gi];
    if (q.z > q.x && q.w > q.y) {
      o = offsets[r];
      cnt = (uint32_t)(q.z - q.x) * (uint32_t)(q.w - q.y);
      if (o + cnt > capacity) {
        atomicExch(overflow, 1u);
        atomicMin(live, (unsigned long long)o);
        cnt = 0;
      }
    }
  }
  cta_emit<K>(q, o, cnt, (K)r, t.kf[k].tile_off, t.kf[k].ntx, rank_bits, keys);
}

// k_emit_pairs_batch with the exclusive scan of the pair counts in the same kernel: CTA b
// of the look-back order (a ticket taken before the programmatic wait, so that every lower
// ticket's CTA has started) covers depth ranks [256 b, 256 b + 256), scans their counts,
// finds its first pair by decoupled look-back (scan_lookback) and writes the pairs.  The
// last CTA writes the pair total and bounds *live by it.  status: [ceil(n / 256)] words,
// then the ticket counter; all zero before the launch.  Eight CTAs per SM (32 registers)
// keep the indoor keyframe's 1172 CTAs resident together.
template <typename K>
__global__ void __launch_bounds__(kThreads, 8) k_scan_emit_pairs_batch(
    const __grid_constant__ EmitTable t, int nkf, const ushort4* __restrict__ rect,
    const uint32_t* __restrict__ order, int64_t n, int rank_bits, uint64_t capacity, K* __restrict__ keys,
    uint32_t* __restrict__ overflow, uint64_t* __restrict__ status, uint32_t* __restrict__ counter,
    uint32_t* __restrict__ err, unsigned long long* __restrict__ total, unsigned long long* __restrict__ live) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t r = (int64_t)tile * kThreads + threadIdx.x;
  ushort4 q = make_ushort4(0, 0, 0, 0);
  uint32_t cnt = 0;
  int k = 0;
  if (r < n) {
    const int64_t gi = order[r];
    while (k + 1 < nkf && t.kf[k + 1].base <= gi) ++k;
    q = rect[gi];
    if (q.z > q.x && q.w > q.y) cnt = (uint32_t)(q.z - q.x) * (uint32_t)(q.w - q.y);
  }
  uint32_t tot;
  const uint32_t run = block_exclusive_scan<uint32_t>(cnt, tot);
  if (threadIdx.x < 32) {
    const uint64_t excl = scan_lookback(status, tile, tot, err);
    if (threadIdx.x == 0) {
      s_prefix = excl;
      if ((int64_t)(tile + 1) * kThreads >= n) {
        *total = excl + tot;
        atomicMin(live, excl + tot);
      }
    }
  }
  __syncthreads();
  const uint64_t o = s_prefix + run;
  if (cnt && o + cnt > capacity) {
    atomicExch(overflow, 1u);
    atomicMin(live, (unsigned long long)o);
    cnt = 0;
  }
  cta_emit<K>(q, o, cnt, (K)r, t.kf[k].tile_off, t.kf[k].ntx, rank_bits, keys);
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_tile_ranges(const K* __restrict__ keys, int64_t m_cap,
                                                          const uint64_t* __restrict__ m_dev, int rank_bits,
                                                          const uint32_t* __restrict__ order,
                                                          uint2* __restrict__ ranges, uint32_t* __restrict__ list) {
  pdl_wait();
  pdl_trigger();
  const int64_t m = live_count(m_cap, m_dev);
  const int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= m) return;
  const K k = keys[p];
  const uint32_t tile = (uint32_t)(k >> rank_bits);
  list[p] = order[(uint32_t)(k & (((K)1 << rank_bits) - 1))];   // single keyframe: never overflows
  if (p == 0 || (uint32_t)(keys[p - 1] >> rank_bits) != tile) ranges[tile].x = (uint32_t)p;
  if (p == m - 1 || (uint32_t)(keys[p + 1] >> rank_bits) != tile) ranges[tile].y = (uint32_t)(p + 1);
}

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// SM count of the current device, read once per device.
int current_sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cached[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) return 1;
  cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Keys per CTA of a radix pass: 4096, or 2048 when a 4096-key grid would leave SMs idle.
inline int sort_items(int64_t n) { return n < int64_t(current_sm_count()) * 4096 ? 8 : 16; }

// Scratch of one sort (uint32 words): [passes][256] histograms, [passes][tiles][256] status
// words, [passes] tile counters and an error flag.
// po (optional): the last pass writes the tile list and per-tile counts instead of keys.
template <typename K, bool kVals, int IPT>
cudaError_t radix_passes(K* ka, K* kb, uint32_t* va, uint32_t* vb, int64_t n, int begin_bit, int end_bit,
                         uint32_t* scratch, int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* rank,
                         uint32_t* err_out, const PairOut* po, bool zeroed) {
  const unsigned nb = grid_for(n, kThreads * IPT);
  const int passes = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
  uint32_t* ghist = scratch;
  uint32_t* gex = ghist + (size_t)passes * kRadixBins;
  uint32_t* status = gex + (size_t)passes * kRadixBins;
  uint32_t* counters = status + (size_t)passes * nb * kRadixBins;
  uint32_t* done = counters + passes;
  uint32_t* err = err_out ? err_out : done + 1;
  if (!zeroed) {
    const cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * onesweep_scratch_words(nb, passes), s);
    if (e != cudaSuccess) return e;
  }
  launch_dep(k_onesweep_hist<K, IPT>, dim3(nb), dim3(kThreads), s, ka, n, n_dev, begin_bit, passes, ghist, gex,
             done);
  const PairOut none{nullptr, nullptr, nullptr, 0, 0u, 0u};
  K* kin = ka; K* kout = kb;
  uint32_t* vin = va; uint32_t* vout = vb;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    launch_dep(k_onesweep_pass<K, kVals, IPT>, dim3(nb), dim3(kThreads), s, kin, kout, vin, vout, n, n_dev,
                                                           begin_bit + p * kRadixBits, gex + p * kRadixBins,
                                                           status + (size_t)p * nb * kRadixBins, counters + p,
                                                           last ? rank : nullptr, err, last && po ? *po : none);
    std::swap(kin, kout);
    std::swap(vin, vout);
    *sel ^= 1;
  }
  return cudaGetLastError();
}

template <typename K, bool kVals>
cudaError_t radix_sort_impl(K* ka, K* kb, uint32_t* va, uint32_t* vb, int64_t n, int end_bit, uint32_t* hist,
                            int* sel, cudaStream_t s, const uint64_t* n_dev = nullptr, uint32_t* rank = nullptr,
                            uint32_t* err = nullptr, int begin_bit = 0, const PairOut* po = nullptr,
                            bool zeroed = false) {
  *sel = 0;
  if (begin_bit < 0 || end_bit > (int)(8 * sizeof(K))) return cudaErrorInvalidValue;
  if (n <= 1 || end_bit <= begin_bit) {  // already in order: ranks from the values as they stand
    if (po) return cudaErrorInvalidValue;  // pair sorts always have tile bits and capacity > 1
    if (rank && va && n > 0) k_rank_scatter<<<grid_for(n, kThreads), kThreads, 0, s>>>(va, n, rank);
    return cudaGetLastError();
  }
  if (end_bit - begin_bit > kMaxRadixPasses * kRadixBits) return cudaErrorInvalidValue;
  if (sort_items(n) == 8)
    return radix_passes<K, kVals, 8>(ka, kb, va, vb, n, begin_bit, end_bit, hist, sel, s, n_dev, rank, err, po,
                                     zeroed);
  return radix_passes<K, kVals, 16>(ka, kb, va, vb, n, begin_bit, end_bit, hist, sel, s, n_dev, rank, err, po,
                                    zeroed);
}

}  // namespace

// scratch: [tiles] look-back status words, a tile counter and an error flag (uint64 each)
size_t scan_scratch_words(int64_t n) { return (size_t)grid_for(n > 0 ? n : 1, kScanTile) + 2; }

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* scratch, uint64_t* total,
                                  cudaStream_t s, uint32_t* err, const uint32_t* gather, bool zeroed) {
  if (n <= 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
    return cudaSuccess;
  }
  const unsigned nb = grid_for(n, kScanTile);
  if (!zeroed) {
    const cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint64_t) * (nb + 2), s);
    if (e != cudaSuccess) return e;
  }
  uint32_t* counter = reinterpret_cast<uint32_t*>(scratch + nb);
  launch_dep(k_scan_lookback, dim3(nb), dim3(kThreads), s, in, gather, out, n, scratch, counter,
                                          err ? err : reinterpret_cast<uint32_t*>(scratch + nb + 1), total);
  return cudaGetLastError();
}

size_t radix_scratch_words(int64_t n) {
  const int64_t m = n > 0 ? n : 1;
  return onesweep_scratch_words(grid_for(m, kThreads * sort_items(m)), kMaxRadixPasses);
}

int64_t radix_sort_launches(int64_t n, int end_bit, int begin_bit) {
  if (n <= 1 || end_bit <= begin_bit) return 0;
  return 1 + (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;  // histograms, one kernel per pass
}

cudaError_t radix_sort_u32(uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a, uint32_t* vals_b, int64_t n,
                           int end_bit, uint32_t* scratch, int* sel, cudaStream_t s, uint32_t* rank, uint32_t* err,
                           int begin_bit, bool zeroed) {
  if (vals_a)
    return radix_sort_impl<uint32_t, true>(keys_a, keys_b, vals_a, vals_b, n, end_bit, scratch, sel, s, nullptr,
                                           rank, err, begin_bit, nullptr, zeroed);
  return radix_sort_impl<uint32_t, false>(keys_a, keys_b, nullptr, nullptr, n, end_bit, scratch, sel, s, nullptr,
                                          nullptr, err, begin_bit, nullptr, zeroed);
}

size_t radix_scratch_used_words(int64_t n, int begin_bit, int end_bit) {
  if (n <= 1 || end_bit <= begin_bit) return 0;
  return onesweep_scratch_words(grid_for(n, kThreads * sort_items(n)),
                                (end_bit - begin_bit + kRadixBits - 1) / kRadixBits);
}

cudaError_t radix_sort_u64(uint64_t* keys_a, uint64_t* keys_b, int64_t n, int end_bit, uint32_t* scratch, int* sel,
                           cudaStream_t s, const uint64_t* n_dev, uint32_t* err, int begin_bit) {
  return radix_sort_impl<uint64_t, false>(keys_a, keys_b, nullptr, nullptr, n, end_bit, scratch, sel, s, n_dev,
                                          nullptr, err, begin_bit);
}

cudaError_t launch_emit_pairs_u32(const ushort4* rect, const uint32_t* offsets, const uint32_t* order, int64_t n,
                                  int ntx, int rank_bits, uint32_t* keys, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_dep(k_emit_pairs<uint32_t>, dim3(grid_for(n, kThreads)), dim3(kThreads), s, rect, offsets, order, n, ntx,
             rank_bits, keys);
  return cudaGetLastError();
}

cudaError_t launch_emit_pairs_u64(const ushort4* rect, const uint32_t* offsets, const uint32_t* order, int64_t n,
                                  int ntx, int rank_bits, uint64_t* keys, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  launch_dep(k_emit_pairs<uint64_t>, dim3(grid_for(n, kThreads)), dim3(kThreads), s, rect, offsets, order, n, ntx,
             rank_bits, keys);
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges_u32(const uint32_t* keys, int64_t m, int rank_bits, const uint32_t* order,
                                   uint2* ranges, uint32_t* list, cudaStream_t s, const uint64_t* m_dev) {
  if (m == 0) return cudaSuccess;
  launch_dep(k_tile_ranges<uint32_t>, dim3(grid_for(m, kThreads)), dim3(kThreads), s, keys, m, m_dev, rank_bits, order,
             ranges,
                                                                       list);
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges_u64(const uint64_t* keys, int64_t m, int rank_bits, const uint32_t* order,
                                   uint2* ranges, uint32_t* list, cudaStream_t s, const uint64_t* m_dev) {
  if (m == 0) return cudaSuccess;
  launch_dep(k_tile_ranges<uint64_t>, dim3(grid_for(m, kThreads)), dim3(kThreads), s, keys, m, m_dev, rank_bits, order,
             ranges,
                                                                       list);
  return cudaGetLastError();
}

cudaError_t launch_emit_pairs_batch(const EmitTable& t, int nkf, int64_t n, const ushort4* rect,
                                    const uint32_t* offsets, const uint32_t* order, int rank_bits, uint64_t capacity,
                                    void* keys, bool k32, uint32_t* overflow, const uint64_t* total, uint64_t* live,
                                    cudaStream_t s) {
  if (nkf == 0 || n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, kThreads);
  if (k32)
    launch_dep(k_emit_pairs_batch<uint32_t>, dim3(grid), dim3(kThreads), s, t, nkf, rect, offsets, order, n, rank_bits,
               capacity, static_cast<uint32_t*>(keys), overflow, reinterpret_cast<const unsigned long long*>(total),
               reinterpret_cast<unsigned long long*>(live));
  else
    launch_dep(k_emit_pairs_batch<uint64_t>, dim3(grid), dim3(kThreads), s, t, nkf, rect, offsets, order, n, rank_bits,
               capacity, static_cast<uint64_t*>(keys), overflow, reinterpret_cast<const unsigned long long*>(total),
               reinterpret_cast<unsigned long long*>(live));
  return cudaGetLastError();
}

size_t scan_emit_scratch_words(int64_t n) { return (size_t)grid_for(n > 0 ? n : 1, kThreads) + 2; }

cudaError_t launch_scan_emit_pairs_batch(const EmitTable& t, int nkf, int64_t n, const ushort4* rect,
                                         const uint32_t* order, int rank_bits, uint64_t capacity, void* keys, bool k32,
                                         uint32_t* overflow, uint64_t* scratch, uint32_t* err, uint64_t* total,
                                         uint64_t* live, cudaStream_t s) {
  if (nkf == 0 || n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, kThreads);
  uint32_t* counter = reinterpret_cast<uint32_t*>(scratch + grid);
  if (!err) err = reinterpret_cast<uint32_t*>(scratch + grid + 1);
  auto* tot = reinterpret_cast<unsigned long long*>(total);
  auto* lv = reinterpret_cast<unsigned long long*>(live);
  if (k32)
    launch_dep(k_scan_emit_pairs_batch<uint32_t>, dim3(grid), dim3(kThreads), s, t, nkf, rect, order, n, rank_bits,
               capacity, static_cast<uint32_t*>(keys), overflow, scratch, counter, err, tot, lv);
  else
    launch_dep(k_scan_emit_pairs_batch<uint64_t>, dim3(grid), dim3(kThreads), s, t, nkf, rect, order, n, rank_bits,
               capacity, static_cast<uint64_t*>(keys), overflow, scratch, counter, err, tot, lv);
  return cudaGetLastError();
}

cudaError_t radix_sort_u32_dev(uint32_t* keys_a, uint32_t* keys_b, int64_t n, int end_bit, uint32_t* scratch,
                               int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* err, int begin_bit) {
  return radix_sort_impl<uint32_t, false>(keys_a, keys_b, nullptr, nullptr, n, end_bit, scratch, sel, s, n_dev,
                                          nullptr, err, begin_bit);
}

cudaError_t radix_sort_pairs_u32(uint32_t* keys_a, uint32_t* keys_b, int64_t n, int end_bit, uint32_t* scratch,
                                 int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* err, int begin_bit,
                                 const PairOut& po, bool zeroed) {
  return radix_sort_impl<uint32_t, false>(keys_a, keys_b, nullptr, nullptr, n, end_bit, scratch, sel, s, n_dev,
                                          nullptr, err, begin_bit, &po, zeroed);
}

cudaError_t radix_sort_pairs_u64(uint64_t* keys_a, uint64_t* keys_b, int64_t n, int end_bit, uint32_t* scratch,
                                 int* sel, cudaStream_t s, const uint64_t* n_dev, uint32_t* err, int begin_bit,
                                 const PairOut& po, bool zeroed) {
  return radix_sort_impl<uint64_t, false>(keys_a, keys_b, nullptr, nullptr, n, end_bit, scratch, sel, s, n_dev,
                                          nullptr, err, begin_bit, &po, zeroed);
}


}  // namespace dqo
