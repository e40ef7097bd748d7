// Learned quadric proposal: a perceptron 128 -> 128 -> 128 -> 9 with ReLU, its adjoint and
// its Adam update.  Every product runs on the 5th-generation tensor cores: tcgen05.mma of
// kind f16 with BF16 operands staged in shared memory and FP32 accumulators in tensor
// memory, issued by one thread per CTA; the epilogues (bias, ReLU, the regression loss,
// the ReLU derivative, the weight-gradient scatter) read the accumulators back with
// tcgen05.ld and are fused into the same kernel.
//
// One kernel shape covers every product of a training step: a CTA computes a 128-row tile
// D[128][N] = A[128][K] . B[N][K]^T (N = 16 or 128, K <= 128 per CTA) with both operands
// K-contiguous in global memory.  Forward layers tile the batch (A = activations,
// B = weights [out][in]); input gradients use the transposed weights; weight gradients
// take the batch as the K dimension (A = activations transposed, B = output gradients
// transposed, one CTA per 128 samples) and add their tile into the FP32 gradient with
// coalesced atomics.
#include <cuda_bf16.h>

#include "dqo_internal.cuh"

namespace dqo {
namespace {

constexpr int kTileM = 128;        // rows of a CTA tile = TMEM lanes
constexpr int kGemmThreads = 128;  // one thread per row in the epilogue
constexpr uint32_t kTmemCols = 128;
constexpr int kGemmSmem = 2 * kTileM * 128 * 2 + 1024;  // A and B tiles of K = 128, and headroom

// ----------------------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor core's (async proxy) reads
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase with the given parity, giving up after about one second.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) return false;
  }
}

// D[tmem] (+)= A[smem] . B[smem]^T, one K = 16 slice; enable_d = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t enable_d) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(enable_d)
      : "memory");
}
// Arrives on the mbarrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane (warp w reads lanes
// 32w..32w+31), waited for before the values are used.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------------------------- operand layout

// Operand tiles in shared memory use the canonical K-major layout without swizzle.  A tile
// of `rows` rows is a sequence of K/16 slices (one MMA each); a slice holds rows/8 groups,
// and a group two 8 x 8 core matrices (8 rows of 16 contiguous bytes) for K elements 0..7
// and 8..15 of the slice.  Descriptor: leading (K) byte offset 128 between the two core
// matrices of a group, stride (M/N) byte offset 256 between groups.  Either reading of the
// two offsets stays inside the slice.
__device__ __forceinline__ uint32_t tile_offset(int r, int k, int rows) {
  return (uint32_t)((k >> 4) * rows * 32 + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, LBO 128 B, SBO 256 B, fixed field 0b001
// at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1), B BF16
// (bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// rows x K tile from K-contiguous global rows (leading dimension ld elements, 16-byte
// aligned rows); rows at or past `valid_rows` are zero.  Each thread issues 8 loads before
// it stores any, so 8 pieces per thread are in flight at once.
__device__ __forceinline__ void load_tile(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int64_t ld,
                                          int rows, int valid_rows, int K) {
  constexpr int kUnroll = 8;
  const int per_row = K >> 3;
  const int total = rows * per_row;
  for (int base = threadIdx.x; base < total; base += kUnroll * blockDim.x) {
    uint4 v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = base + u * blockDim.x;
      const int r = i / per_row, kc = i - r * per_row;
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (i < total && r < valid_rows) v[u] = __ldg(reinterpret_cast<const uint4*>(src + (int64_t)r * ld + kc * 8));
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = base + u * blockDim.x;
      if (i < total) {
        const int r = i / per_row, kc = i - r * per_row;
        *reinterpret_cast<uint4*>(dst + tile_offset(r, kc * 8, rows)) = v[u];
      }
    }
  }
}

// The same tile with asynchronous 16-byte copies (cp.async: no register round trip, every
// piece in flight at once); rows at or past `valid_rows` are zero-filled.  The caller
// commits the group and waits for it (cp_async_wait_all) before the tile is read.
__device__ __forceinline__ void load_tile_async(unsigned char* dst, const __nv_bfloat16* __restrict__ src,
                                                int64_t ld, int rows, int valid_rows, int K) {
  const int per_row = K >> 3;
  const int total = rows * per_row;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int r = i / per_row, kc = i - r * per_row;
    const bool ok = r < valid_rows;
    const __nv_bfloat16* g = src + (int64_t)(ok ? r : 0) * ld + kc * 8;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + tile_offset(r, kc * 8, rows))),
                 "l"(g), "r"(ok ? 16 : 0)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Waits until at most n of this thread's committed groups are still in flight.
template <int n>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory"); }

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// ----------------------------------------------------------------------------- the GEMM kernel

enum : int { kEpiRelu = 0, kEpiOut = 1, kEpiReluGrad = 2, kEpiWgrad = 3 };

struct GemmArgs {
  // D[m][n] = sum_k A[m0 + m][k0 + k] B[n][k0 + k], k0 = blockIdx.y * K
  const __nv_bfloat16* A;
  int64_t lda;
  int M;  // valid rows of A (rows past it are zero)
  const __nv_bfloat16* B;
  int64_t ldb;
  int N;  // 16 or 128
  int K;  // per CTA, multiple of 16, <= 128
  // epilogue operands
  const float* bias;              // kEpiRelu, kEpiOut: [N]
  __nv_bfloat16* out;             // row-major [M][ldo]
  int64_t ldo;
  __nv_bfloat16* outT;            // transposed [N][ldt]
  int64_t ldt;
  const __nv_bfloat16* mask;      // kEpiReluGrad: activations [M][ldm], derivative = (h > 0)
  int64_t ldm;
  float* y;                       // kEpiOut: [M][9]
  const float* labels;            // kEpiOut: [M][9]; NULL = inference
  float inv_batch;
  float w[9];
  float* loss;                    // kEpiOut: += sum_rows sum_j w_j (y - label)^2 / batch
  float* dw;                      // kEpiWgrad: dw[n][m] += D[m][n] for n < dw_rows
  int dw_rows;
  float* db;                      // kEpiWgrad: db[n] += sum_k B[n][k0 + k]
  int* step_inc;                  // if set, block (0,0) adds 1 (the optimiser's step count)
  int* err;                       // set to 1 if the tensor-core wait timed out
};

template <int EPI>
__device__ __forceinline__ void epilogue(const GemmArgs& a, uint32_t trow, int m, bool row_ok) {
  if (EPI == kEpiOut) {
    float v[16];
    tmem_ld16(trow, v);
    float l = 0.f;
    if (row_ok) {
      float y[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) y[j] = v[j] + a.bias[j];
      if (a.y)
#pragma unroll
        for (int j = 0; j < 9; ++j) a.y[(int64_t)m * 9 + j] = y[j];
      if (a.labels) {
        __align__(16) __nv_bfloat16 d[16];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          const float e = y[j] - a.labels[(int64_t)m * 9 + j];
          l += a.w[j] * e * e;
          d[j] = __float2bfloat16_rn(2.f * a.w[j] * e * a.inv_batch);
        }
#pragma unroll
        for (int j = 9; j < 16; ++j) d[j] = __float2bfloat16_rn(0.f);
        if (a.out) {
          uint4* o = reinterpret_cast<uint4*>(a.out + (int64_t)m * a.ldo);
          o[0] = reinterpret_cast<const uint4*>(d)[0];
          o[1] = reinterpret_cast<const uint4*>(d)[1];
        }
        if (a.outT)
#pragma unroll
          for (int j = 0; j < 16; ++j) a.outT[(int64_t)j * a.ldt + m] = d[j];
      }
    }
    if (a.labels && a.loss) {
      l = warp_sum_f(l * a.inv_batch);
      if ((threadIdx.x & 31) == 0) atomicAdd(a.loss, l);
    }
    return;
  }
  for (int c = 0; c < a.N; c += 16) {
    float v[16];
    tmem_ld16(trow + (uint32_t)c, v);
    if (!row_ok) continue;
    if (EPI == kEpiWgrad) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c + j < a.dw_rows) atomicAdd(a.dw + (int64_t)(c + j) * kTileM + m, v[j]);
      continue;
    }
    __align__(16) __nv_bfloat16 h[16];
    if (EPI == kEpiRelu) {
#pragma unroll
      for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16_rn(fmaxf(v[j] + a.bias[c + j], 0.f));
    } else {  // kEpiReluGrad
      __align__(16) __nv_bfloat16 hm[16];
      const uint4* src = reinterpret_cast<const uint4*>(a.mask + (int64_t)m * a.ldm + c);
      reinterpret_cast<uint4*>(hm)[0] = src[0];
      reinterpret_cast<uint4*>(hm)[1] = src[1];
#pragma unroll
      for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16_rn(__bfloat162float(hm[j]) > 0.f ? v[j] : 0.f);
    }
    if (a.out) {
      uint4* o = reinterpret_cast<uint4*>(a.out + (int64_t)m * a.ldo + c);
      o[0] = reinterpret_cast<const uint4*>(h)[0];
      o[1] = reinterpret_cast<const uint4*>(h)[1];
    }
    if (a.outT)
#pragma unroll
      for (int j = 0; j < 16; ++j) a.outT[(int64_t)(c + j) * a.ldt + m] = h[j];
  }
}

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads) k_mlp_gemm(GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  pdl_wait();  // before any memory access or tensor-memory allocation
  pdl_trigger();
  const int t = threadIdx.x, w = t >> 5;
  const int m0 = blockIdx.x * kTileM;
  const int64_t k0 = (int64_t)blockIdx.y * a.K;
  unsigned char* sa = sm;
  unsigned char* sb = sm + kTileM * a.K * 2;
  if (a.step_inc && t == 0 && blockIdx.x == 0 && blockIdx.y == 0) atomicAdd(a.step_inc, 1);
  if (w == 0) {
    tmem_alloc(smem_u32(&tslot), kTmemCols);
    tmem_relinquish();
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  load_tile(sa, a.A + (int64_t)m0 * a.lda + k0, a.lda, kTileM, min(kTileM, a.M - m0), a.K);
  load_tile(sb, a.B + k0, a.ldb, a.N, a.N, a.K);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (t == 0) {
    const uint32_t idesc = idesc_bf16(kTileM, a.N);
    const uint32_t abase = smem_u32(sa), bbase = smem_u32(sb);
    for (int s = 0; s < (a.K >> 4); ++s)
      mma_bf16(tmem, smem_desc(abase + (uint32_t)(s * kTileM * 32)), smem_desc(bbase + (uint32_t)(s * a.N * 32)),
               idesc, s > 0 ? 1u : 0u);
    mma_commit(smem_u32(&mbar));
  }
  const bool done = mbar_wait_bounded(smem_u32(&mbar), 0);
  tc_fence_after();
  if (done) {
    const int m = m0 + t;
    epilogue<EPI>(a, tmem + ((uint32_t)(w * 32) << 16), m, m < a.M);
    if (EPI == kEpiWgrad && a.db && t < a.N) {  // bias gradient: row sums of this CTA's B chunk
      const __nv_bfloat16* row = a.B + (int64_t)t * a.ldb + k0;
      float s = 0.f;
      for (int k = 0; k < a.K; k += 8) {
        __align__(16) __nv_bfloat16 v8[8];
        *reinterpret_cast<uint4*>(v8) = __ldg(reinterpret_cast<const uint4*>(row + k));
#pragma unroll
        for (int j = 0; j < 8; ++j) s += __bfloat162float(v8[j]);
      }
      atomicAdd(a.db + t, s);
    }
  } else if (t == 0 && a.err) {
    atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------------------------- fused training step

// The eight products of a training step (forward, loss, input and weight gradients) for
// the 128 samples of one CTA, back to back in one kernel with every intermediate in shared
// memory: the same operands, the same BF16 rounding points and the same per-CTA weight-
// gradient tiles as the eight launches of launch_mlp_backward, which leave the
// activations in global memory instead.  A step is one launch of n / 128 CTAs + Adam.
// Shared memory: six 32 KB slots for 128 x 128 tiles, reused as the step goes on (the
// operands of a later product are copied asynchronously into a free slot while the
// current one runs), four 4 KB slots for the 16-wide tiles and the biases; tensor memory:
// 256 columns, the products alternating between the two halves.
constexpr int kFusedThreads = 128;
constexpr uint32_t kSlot = kTileM * 128 * 2;      // 32 KB
constexpr uint32_t kSmall = kTileM * kMlpOutPad * 2;  // 4 KB
constexpr int kBiasFloats = 2 * kMlpHidden + kMlpOutPad;
constexpr int kFusedSmem = 6 * kSlot + 4 * kSmall + kBiasFloats * 4 + 1024;
constexpr uint32_t kFusedCols = 256;

struct FusedArgs {
  MlpState st;
  const __nv_bfloat16* X;   // [n][128]
  const __nv_bfloat16* XT;  // [128][ldxt]
  int64_t ldxt;
  const float* labels;      // [n][9]
  float w[9];
  float inv_batch;
  float* loss;              // += sum of the batch's weighted squared errors / n
  int* step_inc;            // block 0 adds 1 (the optimiser's step count); may be NULL
  int* err;                 // set to 1 if a tensor-core wait timed out
  float* gpart;             // [gridDim.x][kMlpParams]: this CTA's gradient
};

// Thread m stores its 16 values of columns [c, c + 16) of row m into a K-major 128-row tile.
__device__ __forceinline__ void put_row16(unsigned char* tile, int m, int c, const __nv_bfloat16 (&h)[16]) {
  *reinterpret_cast<uint4*>(tile + tile_offset(m, c, kTileM)) = reinterpret_cast<const uint4*>(h)[0];
  *reinterpret_cast<uint4*>(tile + tile_offset(m, c + 8, kTileM)) = reinterpret_cast<const uint4*>(h)[1];
}
// ... and into the transposed K-major tile (rows = the columns c + j, K = the samples).
__device__ __forceinline__ void put_col16(unsigned char* tileT, int rowsT, int m, int c,
                                          const __nv_bfloat16 (&h)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    *reinterpret_cast<__nv_bfloat16*>(tileT + tile_offset(c + j, m, rowsT)) = h[j];
}

// D[tmem] = A[a] . B[b]^T over K (multiple of 16) for an N-wide B, issued by thread 0 and
// committed to the mbarrier; every thread then waits (bounded) for phase `ph`.
__device__ __forceinline__ bool fused_mma(uint32_t tmem, const unsigned char* a, const unsigned char* b, int N, int K,
                                          uint32_t bar, uint32_t ph) {
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_bf16(kTileM, N);
    const uint32_t abase = smem_u32(a), bbase = smem_u32(b);
    for (int s = 0; s < (K >> 4); ++s)
      mma_bf16(tmem, smem_desc(abase + (uint32_t)(s * kTileM * 32)), smem_desc(bbase + (uint32_t)(s * N * 32)),
               idesc, s > 0 ? 1u : 0u);
    mma_commit(bar);
  }
  const bool ok = mbar_wait_bounded(bar, ph);
  tc_fence_after();
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Row sums of a K-major tile's rows [0, rows) over its 128 samples (bias gradients).
__device__ __forceinline__ void bias_grad(const unsigned char* tileT, int rowsT, int rows, float* db) {
  const int t = threadIdx.x;
  if (t >= rows) return;
  float s = 0.f;
  for (int k = 0; k < kTileM; ++k)
    s += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tileT + tile_offset(t, k, rowsT)));
  db[t] = s;
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_mlp_train_fused(FusedArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  pdl_wait();
  pdl_trigger();
  const int t = threadIdx.x, w = t >> 5;
  const int64_t m0 = (int64_t)blockIdx.x * kTileM;
  const int m = (int)m0 + t;  // this thread's sample (the batch is a multiple of 128 rows)
  unsigned char* sA = sm;                  // X, then W2T
  unsigned char* sB = sm + kSlot;          // W1, then H2, then XT
  unsigned char* sC = sm + 2 * kSlot;      // H1, then G2T
  unsigned char* sD = sm + 3 * kSlot;      // H1T
  unsigned char* sE = sm + 4 * kSlot;      // H2T, then G1T
  unsigned char* sF = sm + 5 * kSlot;      // W2, then G2
  unsigned char* s0 = sm + 6 * kSlot;      // W3 [16][128]
  unsigned char* s1 = s0 + kSmall;         // dY [128][16]
  unsigned char* s2 = s1 + kSmall;         // dY^T [16][128]
  unsigned char* s3 = s2 + kSmall;         // W3^T [128][16]
  float* sbias = reinterpret_cast<float*>(s3 + kSmall);   // b1, b2, b3
  const MlpState& st = a.st;
  float* const gp = a.gpart + (int64_t)blockIdx.x * kMlpParams;   // this CTA's gradient
  if (a.step_inc && t == 0 && blockIdx.x == 0) atomicAdd(a.step_inc, 1);
  if (w == 0) {
    tmem_alloc(smem_u32(&tslot), kFusedCols);
    tmem_relinquish();
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  const uint32_t bar = smem_u32(&mbar);
  // the first product's operands, then W2 (in flight while the first product runs)
  load_tile_async(sA, a.X + m0 * kMlpIn, kMlpIn, kTileM, kTileM, 128);
  load_tile_async(sB, st.w1b, kMlpHidden, 128, 128, 128);
  load_tile_async(s0, st.w3b, kMlpHidden, kMlpOutPad, kMlpOutPad, 128);
  load_tile_async(s3, st.w3tb, kMlpOutPad, 128, 128, kMlpOutPad);
  cp_async_commit();
  load_tile_async(sF, st.w2b, kMlpHidden, 128, 128, 128);
  cp_async_commit();
  for (int i = t; i < kBiasFloats; i += kFusedThreads)
    sbias[i] = i < kMlpHidden ? st.param[kMlpB1 + i]
                              : (i < 2 * kMlpHidden ? st.param[kMlpB2 + i - kMlpHidden]
                                                    : st.param[kMlpB3 + i - 2 * kMlpHidden]);
  cp_async_wait_group<1>();
  __syncthreads();
  const uint32_t t0 = tslot, lane_off = (uint32_t)(w * 32) << 16;
  const uint32_t tA = t0 + lane_off, tB = t0 + 128u + lane_off;  // this thread's TMEM lane, two halves
  uint32_t ph = 0;
  bool ok = true;
  uint32_t mask1[4] = {0u, 0u, 0u, 0u}, mask2[4] = {0u, 0u, 0u, 0u};

  // ---- H1 = relu(X W1^T + b1): rows into sC, transposed into sD
  ok = fused_mma(t0, sA, sB, 128, 128, bar, ph);
  ph ^= 1u;
  if (ok) {
    for (int c = 0; c < 128; c += 16) {
      float v[16];
      tmem_ld16(tA + (uint32_t)c, v);
      __align__(16) __nv_bfloat16 h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        h[j] = __float2bfloat16_rn(fmaxf(v[j] + sbias[c + j], 0.f));
        if (__bfloat162float(h[j]) > 0.f) mask1[(c + j) >> 5] |= 1u << ((c + j) & 31);
      }
      put_row16(sC, t, c, h);
      put_col16(sD, kTileM, t, c, h);
    }
    // X is no longer needed: W2^T goes there while the next products run
    load_tile_async(sA, st.w2tb, kMlpHidden, 128, 128, 128);
    cp_async_commit();
  }
  // ---- H2 = relu(H1 W2^T + b2): rows into sB (W1 free), transposed into sE
  if (ok) {
    cp_async_wait_group<1>();   // W2
    ok = fused_mma(t0 + 128u, sC, sF, 128, 128, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    for (int c = 0; c < 128; c += 16) {
      float v[16];
      tmem_ld16(tB + (uint32_t)c, v);
      __align__(16) __nv_bfloat16 h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        h[j] = __float2bfloat16_rn(fmaxf(v[j] + sbias[kMlpHidden + c + j], 0.f));
        if (__bfloat162float(h[j]) > 0.f) mask2[(c + j) >> 5] |= 1u << ((c + j) & 31);
      }
      put_row16(sB, t, c, h);
      put_col16(sE, kTileM, t, c, h);
    }
  }
  // ---- Y = H2 W3^T + b3, the loss, dY = 2 w (y - label) / n: rows into s1, transposed into s2
  if (ok) {
    ok = fused_mma(t0, sB, s0, kMlpOutPad, 128, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    float v[16];
    tmem_ld16(tA, v);
    float l = 0.f;
    __align__(16) __nv_bfloat16 d[16];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const float y = v[j] + sbias[2 * kMlpHidden + j];
      const float e = y - a.labels[(int64_t)m * 9 + j];
      l += a.w[j] * e * e;
      d[j] = __float2bfloat16_rn(2.f * a.w[j] * e * a.inv_batch);
    }
#pragma unroll
    for (int j = 9; j < 16; ++j) d[j] = __float2bfloat16_rn(0.f);
    *reinterpret_cast<uint4*>(s1 + tile_offset(t, 0, kTileM)) = reinterpret_cast<const uint4*>(d)[0];
    *reinterpret_cast<uint4*>(s1 + tile_offset(t, 8, kTileM)) = reinterpret_cast<const uint4*>(d)[1];
    put_col16(s2, kMlpOutPad, t, 0, d);
    if (a.loss) {
      l = warp_sum_f(l * a.inv_batch);
      if ((t & 31) == 0) atomicAdd(a.loss, l);
    }
  }
  // ---- G2 = (dY W3) * (H2 > 0): rows into sF (W2 free), transposed into sC (H1 free)
  if (ok) {
    ok = fused_mma(t0 + 128u, s1, s3, 128, kMlpOutPad, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    // H2 is no longer needed: X^T goes there while the next products run
    load_tile_async(sB, a.XT + m0, a.ldxt, 128, 128, 128);
    cp_async_commit();
    for (int c = 0; c < 128; c += 16) {
      float v[16];
      tmem_ld16(tB + (uint32_t)c, v);
      __align__(16) __nv_bfloat16 h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        h[j] = __float2bfloat16_rn(((mask2[(c + j) >> 5] >> ((c + j) & 31)) & 1u) ? v[j] : 0.f);
      put_row16(sF, t, c, h);
      put_col16(sC, kTileM, t, c, h);
    }
  }
  // ---- dW3 += dY^T H2 (A = H2^T, B = dY^T), db3
  if (ok) {
    ok = fused_mma(t0, sE, s2, kMlpOutPad, 128, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    float v[16];
    tmem_ld16(tA, v);
#pragma unroll
    for (int j = 0; j < kMlpOutPad; ++j) gp[kMlpW3 + j * kTileM + t] = j < kMlpOut ? v[j] : 0.f;
    bias_grad(s2, kMlpOutPad, kMlpOutPad, gp + kMlpB3);
  }
  // ---- G1 = (G2 W2) * (H1 > 0): transposed into sE (H2^T free)
  if (ok) {
    cp_async_wait_group<1>();   // W2^T (X^T may still be in flight)
    ok = fused_mma(t0 + 128u, sF, sA, 128, 128, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    for (int c = 0; c < 128; c += 16) {
      float v[16];
      tmem_ld16(tB + (uint32_t)c, v);
      __align__(16) __nv_bfloat16 h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        h[j] = __float2bfloat16_rn(((mask1[(c + j) >> 5] >> ((c + j) & 31)) & 1u) ? v[j] : 0.f);
      put_col16(sE, kTileM, t, c, h);
    }
  }
  // ---- dW2 += G2^T H1 (A = H1^T, B = G2^T), db2
  if (ok) {
    ok = fused_mma(t0, sD, sC, 128, 128, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    for (int c = 0; c < 128; c += 16) {
      float v[16];
      tmem_ld16(tA + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) gp[kMlpW2 + (c + j) * kTileM + t] = v[j];
    }
    bias_grad(sC, kTileM, kMlpHidden, gp + kMlpB2);
  }
  // ---- dW1 += G1^T X (A = X^T, B = G1^T), db1
  if (ok) {
    cp_async_wait_all();        // X^T
    ok = fused_mma(t0 + 128u, sB, sE, 128, 128, bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    for (int c = 0; c < 128; c += 16) {
      float v[16];
      tmem_ld16(tB + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) gp[kMlpW1 + (c + j) * kTileM + t] = v[j];
    }
    bias_grad(sE, kTileM, kMlpHidden, gp + kMlpB1);
  }
  if (!ok && t == 0 && a.err) atomicExch(a.err, 1);
  cp_async_wait_all();          // no copy may still target shared memory when the CTA ends
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(t0, kFusedCols);
  }
}

// ----------------------------------------------------------------------------- features

// One thread per (quadric, view slot): decomposes P = K [R | t] and writes the slot's 16
// features (layout documented with dqo_mlp_features).
__global__ void k_mlp_features(int nq, int nv, const float* __restrict__ Pm, const int32_t* __restrict__ q_ptr,
                               const int32_t* __restrict__ pair_v, int npairs, const float* __restrict__ obs,
                               const int32_t* __restrict__ counts, float inv_scale, __nv_bfloat16* __restrict__ X,
                               __nv_bfloat16* __restrict__ XT, int64_t ldt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nq * kMlpViews) return;
  const int q = (int)(i / kMlpViews), j = (int)(i % kMlpViews);
  const int k0 = max(q_ptr[q], 0), k1 = min(q_ptr[q + 1], npairs);
  int use = min(k1 - k0, kMlpViews);
  if (counts) use = min(use, counts[q]);
  float f[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) f[k] = 0.f;
  const int vw = j < use ? pair_v[k0 + j] : -1;
  if (vw >= 0 && vw < nv) {
    const float* P = Pm + 12 * (int64_t)vw;
    float M0[3] = {P[0], P[1], P[2]}, M1[3] = {P[4], P[5], P[6]}, M2[3] = {P[8], P[9], P[10]};
    float p0 = P[3], p1 = P[7], p2 = P[11];
    const float det = M0[0] * (M1[1] * M2[2] - M1[2] * M2[1]) - M0[1] * (M1[0] * M2[2] - M1[2] * M2[0]) +
                      M0[2] * (M1[0] * M2[1] - M1[1] * M2[0]);
    const float n2 = sqrtf(M2[0] * M2[0] + M2[1] * M2[1] + M2[2] * M2[2]);
    if (det != 0.f && n2 > 0.f) {
      const float sc = (det > 0.f ? 1.f : -1.f) / n2;
#pragma unroll
      for (int k = 0; k < 3; ++k) { M0[k] *= sc; M1[k] *= sc; M2[k] *= sc; }
      p0 *= sc; p1 *= sc; p2 *= sc;
      // RQ by Gram-Schmidt from the last row: M = K R, K = [fx s cx; 0 fy cy; 0 0 1]
      const float* r3 = M2;
      const float cy = M1[0] * r3[0] + M1[1] * r3[1] + M1[2] * r3[2];
      float r2[3] = {M1[0] - cy * r3[0], M1[1] - cy * r3[1], M1[2] - cy * r3[2]};
      const float fy = sqrtf(r2[0] * r2[0] + r2[1] * r2[1] + r2[2] * r2[2]);
      const float cx = M0[0] * r3[0] + M0[1] * r3[1] + M0[2] * r3[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) r2[k] /= fy;
      const float sk = M0[0] * r2[0] + M0[1] * r2[1] + M0[2] * r2[2];
      float r1[3] = {M0[0] - cx * r3[0] - sk * r2[0], M0[1] - cx * r3[1] - sk * r2[1],
                     M0[2] - cx * r3[2] - sk * r2[2]};
      const float fx = sqrtf(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) r1[k] /= fx;
      // t = K^-1 p, camera centre C = -R^T t
      const float t3 = p2, t2 = (p1 - cy * t3) / fy, t1 = (p0 - sk * t2 - cx * t3) / fx;
      const float* b = obs + 4 * (int64_t)(k0 + j);
      const float yc = (0.5f * (b[1] + b[3]) - cy) / fy;
      const float xc = (0.5f * (b[0] + b[2]) - cx - sk * yc) / fx;
      f[0] = xc;
      f[1] = yc;
      f[2] = (b[2] - b[0]) / (2.f * fx);
      f[3] = (b[3] - b[1]) / (2.f * fy);
      float d[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) d[k] = xc * r1[k] + yc * r2[k] + r3[k];
      const float dn = 1.f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        f[4 + k] = r1[k];
        f[7 + k] = r2[k];
        f[10 + k] = d[k] * dn;
        f[13 + k] = -(t1 * r1[k] + t2 * r2[k] + t3 * r3[k]) * inv_scale;
      }
    }
  }
  __align__(16) __nv_bfloat16 h[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) h[k] = __float2bfloat16_rn(f[k]);
  uint4* o = reinterpret_cast<uint4*>(X + (int64_t)q * kMlpIn + 16 * j);
  o[0] = reinterpret_cast<const uint4*>(h)[0];
  o[1] = reinterpret_cast<const uint4*>(h)[1];
  if (XT)
#pragma unroll
    for (int k = 0; k < 16; ++k) XT[(int64_t)(16 * j + k) * ldt + q] = h[k];
}

// ----------------------------------------------------------------------------- Adam

// One thread per parameter: Adam (bias-corrected, step count from the state, learning rate
// on a cosine schedule from lr to lr_final over total_steps), gradient reset to zero, and
// the BF16 operand copies of the weights (W and, for W2 and W3, W^T) rewritten.
__global__ void k_mlp_adam(MlpState st, dqo_mlp_hparams hp, const float* __restrict__ gpart, int nb) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const int step = *st.step;
  float g = st.grad[i];
  for (int b = 0; b < nb; ++b) g += gpart[(int64_t)b * kMlpParams + i];   // in block order
  st.grad[i] = 0.f;
  const float m = hp.beta1 * st.m1[i] + (1.f - hp.beta1) * g;
  const float v = hp.beta2 * st.m2[i] + (1.f - hp.beta2) * g * g;
  st.m1[i] = m;
  st.m2[i] = v;
  const float prog = hp.total_steps > 0 ? fminf((float)(step - 1) / (float)hp.total_steps, 1.f) : 0.f;
  const float lr = hp.lr_final + 0.5f * (hp.lr - hp.lr_final) * (1.f + cospif(prog));
  const float mh = m / (1.f - powf(hp.beta1, (float)step));
  const float vh = v / (1.f - powf(hp.beta2, (float)step));
  const float p = st.param[i] - lr * mh / (sqrtf(vh) + hp.eps);
  st.param[i] = p;
  write_bf16_copies(st, i, p);
}

// out[i] = sum over the fused step's CTAs of their gradient entry i, in block order.
__global__ void k_mlp_sum_partials(const float* __restrict__ gpart, int nb, float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float g = 0.f;
  for (int b = 0; b < nb; ++b) g += gpart[(int64_t)b * kMlpParams + i];
  out[i] = g;
}

// Parameters -> state: master copy, BF16 copies, Adam moments and step reset.
__global__ void k_mlp_set(MlpState st, const float* __restrict__ params) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *st.step = 0;
  if (i >= kMlpParams) return;
  const float p = params[i];
  st.param[i] = p;
  st.grad[i] = 0.f;
  st.m1[i] = 0.f;
  st.m2[i] = 0.f;
  write_bf16_copies(st, i, p);
}

// The bounded wait of the tensor-core kernels on an mbarrier that nothing arrives at: it
// gives up after about one second and records that in *flag.
__global__ void k_bounded_wait_probe(int* __restrict__ flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
  __syncthreads();
  const bool done = mbar_wait_bounded(smem_u32(&bar), 0);
  if (!done && threadIdx.x == 0) atomicExch(flag, 1);
}

}  // namespace

// ----------------------------------------------------------------------------- launchers

cudaError_t launch_bounded_wait_probe(int* flag, cudaStream_t s) {
  k_bounded_wait_probe<<<1, 32, 0, s>>>(flag);
  return cudaGetLastError();
}

cudaError_t mlp_gemm_setup() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_mlp_gemm<kEpiRelu>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_gemm<kEpiOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_gemm<kEpiReluGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_gemm<kEpiWgrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem)))
    return e;
  return cudaFuncSetAttribute(k_mlp_train_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
}

namespace {

template <int EPI>
cudaError_t gemm(const GemmArgs& a, dim3 grid, cudaStream_t s) {
  // every launch takes the full shared-memory budget: at most three CTAs share an SM, so
  // their tensor-memory allocations (128 columns each) always fit in its 512 columns
  return launch_dep_smem(k_mlp_gemm<EPI>, grid, dim3(kGemmThreads), kGemmSmem, s, a);
}

GemmArgs base(const __nv_bfloat16* A, int64_t lda, int M, const __nv_bfloat16* B, int64_t ldb, int N, int K,
              int* err) {
  GemmArgs a{};
  a.A = A;
  a.lda = lda;
  a.M = M;
  a.B = B;
  a.ldb = ldb;
  a.N = N;
  a.K = K;
  a.err = err;
  return a;
}

}  // namespace

cudaError_t launch_mlp_features(int nq, int nv, const float* P, const int32_t* q_ptr, const int32_t* pair_v,
                                int npairs, const float* obs, const int32_t* counts, float inv_scale, uint16_t* X,
                                uint16_t* XT, int64_t ldt, cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  const int64_t n = (int64_t)nq * kMlpViews;
  k_mlp_features<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      nq, nv, P, q_ptr, pair_v, npairs, obs, counts, inv_scale, reinterpret_cast<__nv_bfloat16*>(X),
      reinterpret_cast<__nv_bfloat16*>(XT), ldt);
  return cudaGetLastError();
}

cudaError_t launch_mlp_set(const MlpState& st, const float* params, cudaStream_t s) {
  k_mlp_set<<<(kMlpParams + 255) / 256, 256, 0, s>>>(st, params);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(const MlpState& st, const dqo_mlp_hparams& hp, const float* gpart, int nb,
                            cudaStream_t s) {
  return launch_dep(k_mlp_adam, dim3((kMlpParams + 255) / 256), dim3(256), s, st, hp, gpart, nb);
}

cudaError_t launch_mlp_sum_partials(const float* gpart, int nb, float* out, cudaStream_t s) {
  return launch_dep(k_mlp_sum_partials, dim3((kMlpParams + 255) / 256), dim3(256), s, gpart, nb, out);
}

// Inference: X [n][128] -> y [n][9]; three launches.
cudaError_t launch_mlp_forward(const MlpState& st, const MlpWork& wk, int64_t n, const uint16_t* X_, float* y,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const __nv_bfloat16* X = reinterpret_cast<const __nv_bfloat16*>(X_);
  const dim3 grid((unsigned)((n + kTileM - 1) / kTileM), 1);
  cudaError_t e;
  GemmArgs a = base(X, kMlpIn, (int)n, st.w1b, kMlpHidden, 128, 128, wk.err);
  a.bias = st.param + kMlpB1;
  a.out = wk.h1;
  a.ldo = kMlpHidden;
  if ((e = gemm<kEpiRelu>(a, grid, s))) return e;
  a = base(wk.h1, kMlpHidden, (int)n, st.w2b, kMlpHidden, 128, 128, wk.err);
  a.bias = st.param + kMlpB2;
  a.out = wk.h2;
  a.ldo = kMlpHidden;
  if ((e = gemm<kEpiRelu>(a, grid, s))) return e;
  a = base(wk.h2, kMlpHidden, (int)n, st.w3b, kMlpHidden, kMlpOutPad, 128, wk.err);
  a.bias = st.param + kMlpB3;
  a.y = y;
  return gemm<kEpiOut>(a, grid, s);
}

// Loss and gradients of a batch (n % 128 == 0) in one launch of n / 128 CTAs (the eight
// products of launch_mlp_backward fused, intermediates in shared memory).  Each CTA's
// gradient goes to gpart[blockIdx]; the loss is ADDED to *loss.
cudaError_t launch_mlp_backward_fused(const MlpState& st, int* err, float* gpart, int64_t n, const uint16_t* X_,
                                      const uint16_t* XT_, int64_t ldxt, const float* labels, const float* loss_w,
                                      float* loss, int* step_inc, cudaStream_t s) {
  if (n <= 0 || n % kTileM || !gpart) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.st = st;
  a.gpart = gpart;
  a.X = reinterpret_cast<const __nv_bfloat16*>(X_);
  a.XT = reinterpret_cast<const __nv_bfloat16*>(XT_);
  a.ldxt = ldxt;
  a.labels = labels;
#pragma unroll
  for (int j = 0; j < 9; ++j) a.w[j] = loss_w[j];
  a.inv_batch = 1.f / (float)n;
  a.loss = loss;
  a.step_inc = step_inc;
  a.err = err;
  return launch_dep_smem(k_mlp_train_fused, dim3((unsigned)(n / kTileM)), dim3(kFusedThreads), kFusedSmem, s, a);
}

// Loss and gradients of a batch (n % 128 == 0): eight launches.  Gradients are ADDED to
// st.grad; the loss is ADDED to *loss.
cudaError_t launch_mlp_backward(const MlpState& st, const MlpWork& wk, int64_t n, const uint16_t* X_,
                                const uint16_t* XT_, int64_t ldxt, const float* labels, const float* loss_w,
                                float* loss, int* step_inc, cudaStream_t s) {
  const __nv_bfloat16* X = reinterpret_cast<const __nv_bfloat16*>(X_);
  const __nv_bfloat16* XT = reinterpret_cast<const __nv_bfloat16*>(XT_);
  const dim3 rows((unsigned)(n / kTileM), 1), ksplit(1, (unsigned)(n / kTileM));
  cudaError_t e;
  // forward, keeping activations in both layouts
  GemmArgs a = base(X, kMlpIn, (int)n, st.w1b, kMlpHidden, 128, 128, wk.err);
  a.bias = st.param + kMlpB1;
  a.out = wk.h1;
  a.ldo = kMlpHidden;
  a.outT = wk.h1t;
  a.ldt = n;
  a.step_inc = step_inc;
  if ((e = gemm<kEpiRelu>(a, rows, s))) return e;
  a = base(wk.h1, kMlpHidden, (int)n, st.w2b, kMlpHidden, 128, 128, wk.err);
  a.bias = st.param + kMlpB2;
  a.out = wk.h2;
  a.ldo = kMlpHidden;
  a.outT = wk.h2t;
  a.ldt = n;
  if ((e = gemm<kEpiRelu>(a, rows, s))) return e;
  a = base(wk.h2, kMlpHidden, (int)n, st.w3b, kMlpHidden, kMlpOutPad, 128, wk.err);
  a.bias = st.param + kMlpB3;
  a.labels = labels;
  a.inv_batch = 1.f / (float)n;
#pragma unroll
  for (int j = 0; j < 9; ++j) a.w[j] = loss_w[j];
  a.loss = loss;
  a.out = wk.dy;
  a.ldo = kMlpOutPad;
  a.outT = wk.dyt;
  a.ldt = n;
  if ((e = gemm<kEpiOut>(a, rows, s))) return e;
  // layer 3: dZ2 = (dY W3) * (H2 > 0), dW3 += dY^T H2
  a = base(wk.dy, kMlpOutPad, (int)n, st.w3tb, kMlpOutPad, 128, kMlpOutPad, wk.err);
  a.mask = wk.h2;
  a.ldm = kMlpHidden;
  a.out = wk.dz2;
  a.ldo = kMlpHidden;
  a.outT = wk.dz2t;
  a.ldt = n;
  if ((e = gemm<kEpiReluGrad>(a, rows, s))) return e;
  a = base(wk.h2t, n, kMlpHidden, wk.dyt, n, kMlpOutPad, kTileM, wk.err);
  a.dw = st.grad + kMlpW3;
  a.dw_rows = kMlpOut;
  a.db = st.grad + kMlpB3;
  if ((e = gemm<kEpiWgrad>(a, ksplit, s))) return e;
  // layer 2: dZ1 = (dZ2 W2) * (H1 > 0), dW2 += dZ2^T H1
  a = base(wk.dz2, kMlpHidden, (int)n, st.w2tb, kMlpHidden, 128, 128, wk.err);
  a.mask = wk.h1;
  a.ldm = kMlpHidden;
  a.out = wk.dz1;
  a.ldo = kMlpHidden;
  a.outT = wk.dz1t;
  a.ldt = n;
  if ((e = gemm<kEpiReluGrad>(a, rows, s))) return e;
  a = base(wk.h1t, n, kMlpHidden, wk.dz2t, n, 128, kTileM, wk.err);
  a.dw = st.grad + kMlpW2;
  a.dw_rows = kMlpHidden;
  a.db = st.grad + kMlpB2;
  if ((e = gemm<kEpiWgrad>(a, ksplit, s))) return e;
  // layer 1: dW1 += dZ1^T X
  a = base(XT, ldxt, kMlpIn, wk.dz1t, n, 128, kTileM, wk.err);
  a.dw = st.grad + kMlpW1;
  a.dw_rows = kMlpHidden;
  a.db = st.grad + kMlpB1;
  return gemm<kEpiWgrad>(a, ksplit, s);
}

}  // namespace dqo
