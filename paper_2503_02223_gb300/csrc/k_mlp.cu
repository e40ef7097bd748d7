// Learned quadric proposal: a perceptron 128 -> 128 -> 128 -> 9 with ReLU, its adjoint and
// its Adam update.  Every product runs on the 5th-generation tensor cores: tcgen05.mma of
// kind f16 with BF16 operands staged in shared memory and FP32 accumulators in tensor
// memory, issued by one thread per CTA; the epilogues (bias, ReLU, the regression loss,
// the ReLU derivative, the gradient stores) read the accumulators back with tcgen05.ld.
//
// Inference (k_mlp_gemm, one launch per layer): a CTA computes a 128-row tile
// D[128][N] = A[128][K] . B[N][K]^T (N = 16 or 128, K = 128), A = activations (row-major),
// B = the weights' BF16 copy.  Training (k_mlp_train): one persistent cooperative launch
// runs any number of Adam steps, gradients and optimiser inside.
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

// 64 consecutive FP32 accumulator columns of this thread's TMEM lane, one load and one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,"
      "%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------------------------- operand layout

// Every operand tile [R][C] (C contiguous in global memory, R and C multiples of 8) is kept
// in shared memory as a grid of 8 x 8 core matrices (8 rows of 16 contiguous bytes), column
// block by column block: core (r / 8, c / 8) at (c / 8) * 16 R + (r / 8) * 128 bytes, so a
// column block of 8 is one contiguous run of R rows of 16 bytes.  The same bytes are a valid
// tcgen05 operand both ways (no swizzle):
//   K-major (rows = M or N, columns = K): stride offset 128 B between the 8-row groups,
//     leading offset 16 R B between the two column blocks of a 16-wide K step, 32 R B per
//     K step;
//   MN-major (columns = M or N, rows = K): stride offset 16 R B between column blocks,
//     leading offset 128 B between the two 8-row groups of a K step, 256 B per K step
//     (bits 15 / 16 of the instruction descriptor).
// So a transposed operand (H1^T, X^T, W2^T, ...) is the stored tile read the other way.
// The BF16 weight copies of the state are kept in the same layout in global memory, so a
// weight tile is one contiguous copy.
__device__ __forceinline__ uint32_t grid_off(int r, int c, int R) {
  return (uint32_t)((c >> 3) * (R * 16) + r * 16 + (c & 7) * 2);
}

// One operand of a product: a grid tile of R rows read K-major or MN-major.
struct Opnd {
  uint32_t addr;
  int R;
  bool mn;
};
__device__ __forceinline__ uint64_t opnd_desc(const Opnd& o, int kstep) {
  const uint32_t wide = 16u * (uint32_t)o.R;
  const uint32_t lbo = o.mn ? 128u : wide, sbo = o.mn ? wide : 128u;
  const uint32_t a = o.addr + (uint32_t)kstep * (o.mn ? 256u : 2u * wide);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
// D[tmem][128][N] (+)= A . B^T over K (multiple of 16), kind f16: D F32 (bits 4-5 = 1), A
// and B BF16 (bits 7-9, 10-12 = 1), transposes at bits 15 / 16, N >> 3 at bit 17, M >> 4
// at bit 24.  Called by one thread.
__device__ __forceinline__ void issue_product(uint32_t tmem, const Opnd& A, const Opnd& B, int N, int K) {
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((A.mn ? 1u : 0u) << 15) | ((B.mn ? 1u : 0u) << 16) |
                         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
  for (int s = 0; s < (K >> 4); ++s) mma_bf16(tmem, opnd_desc(A, s), opnd_desc(B, s), idesc, s > 0 ? 1u : 0u);
}

// rows x 128 block of a row-major BF16 matrix (ld elements per row, 16-byte aligned rows)
// into a grid tile of R = rows; rows at or past `valid_rows` are zero.  Consecutive threads
// take consecutive rows of a column block (contiguous shared-memory stores); eight 16-byte
// loads per thread are in flight before the first store.
__device__ __forceinline__ void load_rows_grid(unsigned char* dst, const __nv_bfloat16* __restrict__ src,
                                               int64_t ld, int rows, int valid_rows) {
  constexpr int kUnroll = 8;
  const int total = rows * 16;
  for (int base = threadIdx.x; base < total; base += kUnroll * blockDim.x) {
    uint4 v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = base + u * blockDim.x;
      const int cb = i / rows, r = i - cb * rows;
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (i < total && r < valid_rows)
        v[u] = __ldg(reinterpret_cast<const uint4*>(src + (int64_t)r * ld + cb * 8));
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = base + u * blockDim.x;
      if (i < total) *reinterpret_cast<uint4*>(dst + 16 * i) = v[u];   // 16 i = grid_off(r, 8 cb, rows)
    }
  }
}
// Contiguous copy of `bytes` (multiple of 16) from global to shared memory, eight 16-byte
// loads per thread in flight before the first store.
__device__ __forceinline__ void copy_contig(unsigned char* dst, const void* __restrict__ src, int bytes) {
  constexpr int kUnroll = 8;
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  const int total = bytes / 16;
  for (int base = threadIdx.x; base < total; base += kUnroll * blockDim.x) {
    uint4 v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = base + u * blockDim.x;
      if (i < total) v[u] = __ldg(s4 + i);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = base + u * blockDim.x;
      if (i < total) reinterpret_cast<uint4*>(dst)[i] = v[u];
    }
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

enum : int { kEpiRelu = 0, kEpiOut = 1 };

struct GemmArgs {
  // D[m][n] = sum_k A[m0 + m][k] B[n][k], K = 128
  const __nv_bfloat16* A;         // row-major [M][lda]
  int64_t lda;
  int M;                          // valid rows of A (rows past it are zero)
  const __nv_bfloat16* B;         // weights [N][128] in the grid layout (a state copy)
  int N;                          // 16 or 128
  const float* bias;              // [N]
  __nv_bfloat16* out;             // kEpiRelu: row-major [M][ldo]
  int64_t ldo;
  float* y;                       // kEpiOut: [M][9]
  int* err;                       // set to 1 if the tensor-core wait timed out
};

template <int EPI>
__device__ __forceinline__ void epilogue(const GemmArgs& a, uint32_t trow, int m, bool row_ok) {
  if constexpr (EPI == kEpiOut) {
    float v[16];
    tmem_ld16(trow, v);
    if (row_ok)
#pragma unroll
      for (int j = 0; j < 9; ++j) a.y[(int64_t)m * 9 + j] = v[j] + a.bias[j];
  } else {
    for (int c = 0; c < a.N; c += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c, v);
      if (!row_ok) continue;
      __align__(16) __nv_bfloat16 h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) h[j] = __float2bfloat16_rn(fmaxf(v[j] + a.bias[c + j], 0.f));
      uint4* o = reinterpret_cast<uint4*>(a.out + (int64_t)m * a.ldo + c);
      o[0] = reinterpret_cast<const uint4*>(h)[0];
      o[1] = reinterpret_cast<const uint4*>(h)[1];
    }
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
  unsigned char* sa = sm;
  unsigned char* sb = sm + kTileM * 128 * 2;
  if (w == 0) {
    tmem_alloc(smem_u32(&tslot), kTmemCols);
    tmem_relinquish();
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  load_rows_grid(sa, a.A + (int64_t)m0 * a.lda, a.lda, kTileM, min(kTileM, a.M - m0));
  copy_contig(sb, a.B, a.N * 128 * 2);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (t == 0) {
    issue_product(tmem, Opnd{smem_u32(sa), kTileM, false}, Opnd{smem_u32(sb), a.N, false}, a.N, 128);
    mma_commit(smem_u32(&mbar));
  }
  const bool done = mbar_wait_bounded(smem_u32(&mbar), 0);
  tc_fence_after();
  if (done) {
    const int m = m0 + t;
    epilogue<EPI>(a, tmem + ((uint32_t)(w * 32) << 16), m, m < a.M);
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

// ----------------------------------------------------------------------------- training

// Training (k_mlp_train): one cooperative launch runs `steps` Adam steps on consecutive
// batches (or, in gradient mode, the loss gradient of one batch).  A step is
//   1. per 128-sample tile, the eight products of the forward and backward pass, with every
//      intermediate in shared memory, the tile's whole gradient written to its own slot;
//   2. a grid-wide barrier;
//   3. Adam on a slice of the parameters per CTA (the slots added in tile order, so the
//      result does not depend on timing), the BF16 weight copies rewritten;
//   4. a grid-wide barrier (the next step reads the new weights).
// The grid is every SM (one CTA each, by shared memory); CTA c takes tiles c, c + grid, ...
// of every step, and the next tile's samples and labels are copied in while the current
// tile runs.  The weights of a step arrive as three bulk copies of their grid-layout copies.
//
// Tile products (s = samples, h1 / h2 = hidden units; R1..R6 are the six rounds of
// tensor-core work, products of one round issued together):
//   R1 H1 = relu(X W1^T + b1)          R2 H2 = relu(H1 W2^T + b2)
//   R3 Y = H2 W3^T + b3, loss, dY      R4 G2 = (dY W3) * (H2 > 0);  dW3^T = H2^T dY
//   R5 G1 = (G2 W2) * (H1 > 0);  dW2^T = H1^T G2;  db2 = G2^T 1
//   R6 dW1^T = X^T G1;  db1 = G1^T 1
// The weight gradients come out transposed (one accumulator row per input unit), so a
// warp's stores of a column are 128 contiguous bytes.  db3 is a warp and block sum of dY.
//
// Two warps share each 32-lane quarter of tensor memory (warp w reads lanes 32 (w % 4) ..
// + 31) and take the columns [64 (w / 4), + 64) of a 128-column result, one 64-column
// load and one wait each.
constexpr int kTrainThreads = 256;
constexpr uint32_t kTileW = 128 * 128 * 2;
constexpr uint32_t kTile16 = 16 * 128 * 2;
constexpr uint32_t kLabBytes = kTileM * 9 * 4;
constexpr int kBiasFloats = 2 * kMlpHidden + kMlpOutPad;
constexpr uint32_t kOffX = 0,                          // X, two buffers
    kOffH1 = kOffX + 2 * kTileW, kOffS = kOffH1 + kTileW,  // S: W1, then H2, then G1
    kOffW2 = kOffS + kTileW, kOffG2 = kOffW2 + kTileW, kOffW3 = kOffG2 + kTileW, kOffDY = kOffW3 + kTile16,
    kOffOnes = kOffDY + kTile16, kOffLab = kOffOnes + kTile16,  // labels, two buffers
    kOffBias = kOffLab + 2 * kLabBytes, kOffDb3 = kOffBias + kBiasFloats * 4, kTrainBytes = kOffDb3 + 4 * 16 * 4;
constexpr int kTrainSmem = (int)kTrainBytes + 1024;   // the base is aligned to 1024 B inside
constexpr uint32_t kTrainCols = 512;

enum : int { kTrainAdam = 0, kTrainGrad = 1 };

struct TrainArgs {
  MlpState st;
  dqo_mlp_hparams hp;        // Adam (kTrainAdam); hp.loss_w weights the loss in both modes
  const __nv_bfloat16* X;    // [steps * tiles * 128][128]
  const float* labels;       // [steps * tiles * 128][9]
  float* losses;             // [steps]: += each step's loss; may be NULL
  float* grads;              // kTrainGrad: [kMlpParams], overwritten with the batch gradient
  float* gpart;              // [tiles][kMlpParams]: the tiles' gradients of the current step
  unsigned* bar;             // grid barrier counter, zero at the launch
  int* err;                  // set to 1 if a wait ran out
  int steps, tiles, mode;
  float inv_batch;
};

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global to shared
// memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Grid-wide barrier number k (1, 2, ...) of the launch: each CTA adds 1 to the counter and
// waits until it reaches k * gridDim.x.  Global writes before it (generic stores) are
// visible after it to loads and to bulk copies.  Returns false if the wait ran out (about
// a second).
__device__ bool grid_barrier(unsigned* bar, unsigned k) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = k * gridDim.x;
    const uint64_t t0 = global_ns();
    int ok = 1;
    for (uint32_t it = 0;; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if ((it & 15u) == 15u && global_ns() - t0 > 1000000000ull) {
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Makes the block's shared-memory writes visible to the tensor core and orders the
// previous tensor-memory reads before the products the caller issues next.
__device__ __forceinline__ void round_begin() {
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}
// Thread 0 commits the products it issued; every thread waits (bounded) for them.
__device__ __forceinline__ bool round_end(uint32_t bar, uint32_t ph) {
  if (threadIdx.x == 0) mma_commit(bar);
  const bool ok = mbar_wait_bounded(bar, ph);
  tc_fence_after();
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Thread m's 16 BF16 values for columns [c, c + 16) of row m of a grid tile of R rows.
__device__ __forceinline__ void put_grid16(unsigned char* tile, int R, int m, int c, const __nv_bfloat16 (&h)[16]) {
  *reinterpret_cast<uint4*>(tile + grid_off(m, c, R)) = reinterpret_cast<const uint4*>(h)[0];
  *reinterpret_cast<uint4*>(tile + grid_off(m, c + 8, R)) = reinterpret_cast<const uint4*>(h)[1];
}

// Epilogue of a 128 x 128 activation result: thread (row r, columns [c0, c0 + 64)) turns its
// accumulators into BF16 values (kRelu: ReLU of the sum with the bias, recording which are
// positive in `mask`; else the accumulators masked by the ReLU derivative `mask`) and stores
// them into row r of a grid tile.
template <bool kRelu>
__device__ __forceinline__ void act_epilogue(uint32_t taddr, const float* bias, uint32_t (&mask)[2],
                                             unsigned char* tile, int r, int c0) {
  float v[64];
  tmem_ld64(taddr, v);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __align__(16) __nv_bfloat16 h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = 16 * q + j;
      if (kRelu) {
        h[j] = __float2bfloat16_rn(fmaxf(v[k] + bias[c0 + k], 0.f));
        if (__bfloat162float(h[j]) > 0.f) mask[k >> 5] |= 1u << (k & 31);
      } else {
        h[j] = __float2bfloat16_rn(((mask[k >> 5] >> (k & 31)) & 1u) ? v[k] : 0.f);
      }
    }
    put_grid16(tile, kTileM, r, c0 + 16 * q, h);
  }
}
// Epilogue of a transposed weight gradient D[in][out] (row r = input unit): dw[out][in]
// for this thread's 64 output columns; a warp's store of one column is 128 contiguous bytes.
__device__ __forceinline__ void wgrad_store(uint32_t taddr, float* dw, int r, int c0) {
  float v[64];
  tmem_ld64(taddr, v);
#pragma unroll
  for (int j = 0; j < 64; ++j) dw[(c0 + j) * 128 + r] = v[j];
}

// The tile's samples and labels (job j of this CTA) into buffer j & 1, by cp.async (one
// commit group).  Rows of X are 16-byte aligned; the labels of a tile are 4608 contiguous
// bytes at a multiple of 4608.
__device__ __forceinline__ void load_tile_inputs(const TrainArgs& a, unsigned char* sbase, int64_t row0, int buf) {
  const uint32_t dx = smem_u32(sbase + kOffX + buf * kTileW), dl = smem_u32(sbase + kOffLab + buf * kLabBytes);
  const __nv_bfloat16* x = a.X + row0 * kMlpIn;
  for (int i = threadIdx.x; i < kTileM * 16; i += kTrainThreads) {
    const int cb = i >> 7, r = i & (kTileM - 1);   // grid_off(r, 8 cb, 128) = 16 i
    cp_async16(dx + 16u * (uint32_t)i, x + (int64_t)r * kMlpIn + cb * 8);
  }
  const float* lab = a.labels + row0 * 9;
  for (int i = threadIdx.x; i < (int)(kLabBytes / 16); i += kTrainThreads) cp_async16(dl + 16u * (uint32_t)i, lab + 4 * i);
  cp_async_commit();
}

__global__ void __launch_bounds__(kTrainThreads, 1) k_mlp_train(const __grid_constant__ TrainArgs a) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t mbar[3];   // products, W1, W2 + W3
  __shared__ uint32_t tslot;
  __shared__ int s_step0;
  pdl_wait();
  pdl_trigger();
  unsigned char* sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int g = w >> 2;              // column half of a 128-column result
  const int r = (w & 3) * 32 + lane; // accumulator row (TMEM lane) of this thread
  const int c0 = 64 * g;
  const int G = (int)gridDim.x, c = (int)blockIdx.x;
  const int my_tiles = c < a.tiles ? (a.tiles - 1 - c) / G + 1 : 0;
  const int jobs = my_tiles * a.steps;
  unsigned char* sH1 = sm + kOffH1;
  unsigned char* sS = sm + kOffS;
  unsigned char* sW2 = sm + kOffW2;
  unsigned char* sG2 = sm + kOffG2;
  unsigned char* sW3 = sm + kOffW3;
  unsigned char* sDY = sm + kOffDY;
  float* sbias = reinterpret_cast<float*>(sm + kOffBias);   // b1, b2, b3
  float* sdb3 = reinterpret_cast<float*>(sm + kOffDb3);     // [warp][16]
  const MlpState& st = a.st;
  const uint32_t bar_mma = smem_u32(&mbar[0]), bar_w1 = smem_u32(&mbar[1]), bar_w23 = smem_u32(&mbar[2]);
  if (jobs > 0 && w == 0) {
    tmem_alloc(smem_u32(&tslot), kTrainCols);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_w1, 1);
    mbar_init(bar_w23, 1);
    s_step0 = *st.step;
  }
  // the ones tile [16][128] (bias gradients) and the first job's inputs
  reinterpret_cast<uint4*>(sm + kOffOnes)[t] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  if (jobs > 0) load_tile_inputs(a, sm, (int64_t)c * kTileM, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t t0 = tslot, t1 = t0 + 256u, lane_off = (uint32_t)((w & 3) * 32) << 16;
  const uint32_t a0 = t0 + lane_off, a1 = t1 + lane_off;   // this thread's row in the two halves
  const Opnd H1{smem_u32(sH1), kTileM, false}, H1T{smem_u32(sH1), kTileM, true};
  const Opnd S{smem_u32(sS), kTileM, false}, ST{smem_u32(sS), kTileM, true};
  const Opnd W2{smem_u32(sW2), 128, false}, W2T{smem_u32(sW2), 128, true};
  const Opnd G2{smem_u32(sG2), kTileM, false}, G2T{smem_u32(sG2), kTileM, true};
  const Opnd W3{smem_u32(sW3), kMlpOutPad, false}, W3T{smem_u32(sW3), kMlpOutPad, true};
  const Opnd DY{smem_u32(sDY), kTileM, false}, DYT{smem_u32(sDY), kTileM, true};
  const Opnd ONES{smem_u32(sm + kOffOnes), 16, false};
  uint32_t ph = 0, ph_w1 = 0, ph_w23 = 0;
  bool w1_out = false, w23_out = false;   // bulk copies issued and not yet waited for
  bool ok = true;
  unsigned nbar = 0;
  int job = 0;
  for (int step = 0; step < a.steps && ok; ++step) {
    // ---- the step's biases (written by other CTAs' Adam: read through L2) and weights
    for (int i = t; i < kBiasFloats; i += kTrainThreads)
      sbias[i] = __ldcg(st.param + (i < kMlpHidden ? kMlpB1 + i
                                                   : (i < 2 * kMlpHidden ? kMlpB2 + i - kMlpHidden
                                                                         : kMlpB3 + i - 2 * kMlpHidden)));
    if (my_tiles > 0 && t == 0) {
      mbar_expect_tx(bar_w23, kTileW + kTile16);
      bulk_g2s(smem_u32(sW2), st.w2b, kTileW, bar_w23);
      bulk_g2s(smem_u32(sW3), st.w3b, kTile16, bar_w23);
    }
    w23_out = my_tiles > 0;
    for (int k = 0; k < my_tiles && ok; ++k, ++job) {
      const int tile = c + k * G;
      const int buf = job & 1;
      const Opnd X{smem_u32(sm + kOffX + buf * kTileW), kTileM, false}, XT{X.addr, kTileM, true};
      const float* slab = reinterpret_cast<const float*>(sm + kOffLab + buf * kLabBytes);
      float* const gp = a.gpart + (int64_t)tile * kMlpParams;
      if (t == 0) {
        mbar_expect_tx(bar_w1, kTileW);
        bulk_g2s(smem_u32(sS), st.w1b, kTileW, bar_w1);
      }
      w1_out = true;
      if (job + 1 < jobs) {
        // the next job's inputs: tile c + (k + 1) G of this step, or tile c of the next one
        const int nstep = k + 1 < my_tiles ? step : step + 1, ntile = k + 1 < my_tiles ? tile + G : c;
        load_tile_inputs(a, sm, ((int64_t)nstep * a.tiles + ntile) * kTileM, buf ^ 1);
        cp_async_wait_group<1>();
      } else {
        cp_async_wait_group<0>();
      }
      ok = __syncthreads_and(mbar_wait_bounded(bar_w1, ph_w1) ? 1 : 0) != 0;
      ph_w1 ^= 1u;
      w1_out = !ok;
      uint32_t mask1[2] = {0u, 0u}, mask2[2] = {0u, 0u};   // ReLU masks of this thread's 64 columns
      // ---- R1: H1 = relu(X W1^T + b1) [s][h1]
      round_begin();
      if (ok && t == 0) issue_product(t0, X, S, 128, kMlpIn);
      ok = ok && round_end(bar_mma, ph);
      ph ^= 1u;
      if (ok) act_epilogue<true>(a0 + (uint32_t)c0, sbias, mask1, sH1, r, c0);
      // ---- R2: H2 = relu(H1 W2^T + b2) [s][h2], into S (W1 is done)
      if (ok && w23_out) {
        ok = __syncthreads_and(mbar_wait_bounded(bar_w23, ph_w23) ? 1 : 0) != 0;
        ph_w23 ^= 1u;
        w23_out = !ok;
      }
      if (ok) {
        round_begin();
        if (t == 0) issue_product(t1, H1, W2, 128, kMlpHidden);
        ok = round_end(bar_mma, ph);
        ph ^= 1u;
      }
      if (ok) act_epilogue<true>(a1 + (uint32_t)c0, sbias + kMlpHidden, mask2, sS, r, c0);
      // ---- R3: Y = H2 W3^T + b3, the loss, dY = 2 w (y - label) / n [s][16], db3 (warps 0-3)
      if (ok) {
        round_begin();
        if (t == 0) issue_product(t0, S, W3, kMlpOutPad, kMlpHidden);
        ok = round_end(bar_mma, ph);
        ph ^= 1u;
      }
      if (ok && g == 0) {
        float v[16];
        tmem_ld16(a0, v);
        float l = 0.f;
        __align__(16) __nv_bfloat16 d[16];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          const float y = v[j] + sbias[2 * kMlpHidden + j];
          const float e = y - slab[r * 9 + j];
          l += a.hp.loss_w[j] * e * e;
          d[j] = __float2bfloat16_rn(2.f * a.hp.loss_w[j] * e * a.inv_batch);
        }
#pragma unroll
        for (int j = 9; j < 16; ++j) d[j] = __float2bfloat16_rn(0.f);
        put_grid16(sDY, kTileM, r, 0, d);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          const float s = warp_sum_f(__bfloat162float(d[j]));
          if (lane == 0) sdb3[w * kMlpOutPad + j] = s;
        }
        if (a.losses) {
          l = warp_sum_f(l * a.inv_batch);
          if (lane == 0) atomicAdd(a.losses + step, l);
        }
      }
      // ---- R4: G2 = (dY W3) * (H2 > 0) [s][h2]; dW3^T = H2^T dY [h2][16]
      if (ok) {
        round_begin();
        if (t == 0) {
          issue_product(t0, DY, W3T, 128, kMlpOutPad);
          issue_product(t1, ST, DYT, kMlpOutPad, kTileM);
        }
        ok = round_end(bar_mma, ph);
        ph ^= 1u;
      }
      if (ok) {
        act_epilogue<false>(a0 + (uint32_t)c0, nullptr, mask2, sG2, r, c0);
        if (g == 1) {
          float v[16];
          tmem_ld16(a1, v);
#pragma unroll
          for (int j = 0; j < kMlpOutPad; ++j) gp[kMlpW3 + j * kTileM + r] = j < kMlpOut ? v[j] : 0.f;
        } else if (r < kMlpOutPad) {
          gp[kMlpB3 + r] = r < kMlpOut ? sdb3[r] + sdb3[kMlpOutPad + r] + sdb3[2 * kMlpOutPad + r] +
                                             sdb3[3 * kMlpOutPad + r]
                                       : 0.f;
        }
      }
      // ---- R5: G1 = (G2 W2) * (H1 > 0) [s][h1], into S (H2 is done); dW2^T = H1^T G2; db2
      if (ok) {
        round_begin();
        if (t == 0) {
          issue_product(t0, G2, W2T, 128, kMlpHidden);
          issue_product(t1, H1T, G2T, 128, kTileM);
          issue_product(t1 + 128u, G2T, ONES, 16, kTileM);
        }
        ok = round_end(bar_mma, ph);
        ph ^= 1u;
      }
      if (ok) {
        act_epilogue<false>(a0 + (uint32_t)c0, nullptr, mask1, sS, r, c0);
        wgrad_store(a1 + (uint32_t)c0, gp + kMlpW2, r, c0);
        if (g == 1) {
          float v[16];
          tmem_ld16(a1 + 128u, v);
          gp[kMlpB2 + r] = v[0];
        }
      }
      // ---- R6: dW1^T = X^T G1 [in][h1]; db1 = G1^T 1
      if (ok) {
        round_begin();
        if (t == 0) {
          issue_product(t0, XT, ST, 128, kTileM);
          issue_product(t0 + 128u, ST, ONES, 16, kTileM);
        }
        ok = round_end(bar_mma, ph);
        ph ^= 1u;
      }
      if (ok) {
        wgrad_store(a0 + (uint32_t)c0, gp + kMlpW1, r, c0);
        if (g == 1) {
          float v[16];
          tmem_ld16(a0 + 128u, v);
          gp[kMlpB1 + r] = v[0];
        }
      }
    }
    // ---- every tile's gradient is written: Adam (or the gradient sum) on this CTA's slice.
    // Four threads per group of four parameters: part p adds the tiles [p T / 4, (p + 1) T / 4)
    // in order, the four parts are combined pairwise (the same order on every run).  The
    // slice's own optimiser state (no other CTA touches it) is loaded before the barrier.
    constexpr int kGroups = kMlpParams / 4;
    const int q0 = (int)((int64_t)c * kGroups / G), q1 = (int)((int64_t)(c + 1) * kGroups / G);
    const int span = 4 * (q1 - q0);
    const bool adam = a.mode == kTrainAdam;
    float4 pre_g0, pre_m1, pre_m2, pre_p;
    if (adam && t < span && (t & 3) == 0) {
      const int i = 4 * (q0 + (t >> 2));
      pre_g0 = *reinterpret_cast<const float4*>(st.grad + i);
      pre_m1 = *reinterpret_cast<const float4*>(st.m1 + i);
      pre_m2 = *reinterpret_cast<const float4*>(st.m2 + i);
      pre_p = *reinterpret_cast<const float4*>(st.param + i);
    }
    const int stepn = s_step0 + step + 1;
    const float prog = a.hp.total_steps > 0 ? fminf((float)(stepn - 1) / (float)a.hp.total_steps, 1.f) : 0.f;
    const float lr = a.hp.lr_final + 0.5f * (a.hp.lr - a.hp.lr_final) * (1.f + cospif(prog));
    const float bc1 = 1.f - powf(a.hp.beta1, (float)stepn), bc2 = 1.f - powf(a.hp.beta2, (float)stepn);
    if (ok) ok = grid_barrier(a.bar, ++nbar);
    if (!ok) break;
    {
      for (int base = 0; base < span; base += kTrainThreads) {
        const int idx = base + t;
        const bool act = idx < span;
        const int q = q0 + (idx >> 2), part = idx & 3;
        const int i = 4 * q;
        const int b0 = part * a.tiles / 4, b1 = (part + 1) * a.tiles / 4;
        float4 gs = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
          int b = b0;
          for (; b + 8 <= b1; b += 8) {
            float4 p[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
              p[u] = __ldcg(reinterpret_cast<const float4*>(a.gpart + (int64_t)(b + u) * kMlpParams + i));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              gs.x += p[u].x;
              gs.y += p[u].y;
              gs.z += p[u].z;
              gs.w += p[u].w;
            }
          }
          for (; b < b1; ++b) {
            const float4 p = __ldcg(reinterpret_cast<const float4*>(a.gpart + (int64_t)b * kMlpParams + i));
            gs.x += p.x;
            gs.y += p.y;
            gs.z += p.z;
            gs.w += p.w;
          }
        }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
          gs.x += __shfl_xor_sync(0xFFFFFFFFu, gs.x, o);
          gs.y += __shfl_xor_sync(0xFFFFFFFFu, gs.y, o);
          gs.z += __shfl_xor_sync(0xFFFFFFFFu, gs.z, o);
          gs.w += __shfl_xor_sync(0xFFFFFFFFu, gs.w, o);
        }
        if (!act || part != 0) continue;
        if (a.mode == kTrainGrad) {
          *reinterpret_cast<float4*>(a.grads + i) = gs;
          continue;
        }
        const bool pre = base == 0;   // the state of the first round was loaded before the barrier
        const float4 g0 = pre ? pre_g0 : *reinterpret_cast<const float4*>(st.grad + i);   // added from outside
        *reinterpret_cast<float4*>(st.grad + i) = make_float4(0.f, 0.f, 0.f, 0.f);
        const float gv[4] = {g0.x + gs.x, g0.y + gs.y, g0.z + gs.z, g0.w + gs.w};
        float4 m1 = pre ? pre_m1 : *reinterpret_cast<const float4*>(st.m1 + i);
        float4 m2 = pre ? pre_m2 : *reinterpret_cast<const float4*>(st.m2 + i);
        float4 pp = pre ? pre_p : *reinterpret_cast<const float4*>(st.param + i);
        float* m1v = &m1.x;
        float* m2v = &m2.x;
        float* pv = &pp.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          m1v[e] = a.hp.beta1 * m1v[e] + (1.f - a.hp.beta1) * gv[e];
          m2v[e] = a.hp.beta2 * m2v[e] + (1.f - a.hp.beta2) * gv[e] * gv[e];
          pv[e] = pv[e] - lr * (m1v[e] / bc1) / (sqrtf(m2v[e] / bc2) + a.hp.eps);
          write_bf16_copies(st, i + e, pv[e]);
        }
        *reinterpret_cast<float4*>(st.m1 + i) = m1;
        *reinterpret_cast<float4*>(st.m2 + i) = m2;
        *reinterpret_cast<float4*>(st.param + i) = pp;
      }
    }
    if (a.mode == kTrainGrad) break;
    if (step + 1 < a.steps) ok = grid_barrier(a.bar, ++nbar);   // the next step reads the new weights
  }
  if (!ok && t == 0 && a.err) atomicExch(a.err, 1);
  if (ok && a.mode == kTrainAdam && c == 0 && t == 0) *st.step = s_step0 + a.steps;
  // nothing may still target shared memory or tensor memory when the CTA ends
  cp_async_wait_all();
  if (t == 0) {
    if (w1_out) mbar_wait_bounded(bar_w1, ph_w1);
    if (w23_out) mbar_wait_bounded(bar_w23, ph_w23);
  }
  tc_fence_before();
  __syncthreads();
  if (jobs > 0 && w == 0) {
    tc_fence_after();
    tmem_dealloc(t0, kTrainCols);
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

// ----------------------------------------------------------------------------- state

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

// The bounded waits of the tensor-core kernels: on an mbarrier that nothing arrives at
// (bit 0 of *flag when it gives up, after about one second), then the training kernel's
// grid barrier with a count that one CTA never reaches (bit 1).
__global__ void k_bounded_wait_probe(int* __restrict__ flag, unsigned* __restrict__ counter) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
  __syncthreads();
  const bool done = mbar_wait_bounded(smem_u32(&bar), 0);
  if (!done && threadIdx.x == 0) atomicOr(flag, 1);
  if (!grid_barrier(counter, 2u) && threadIdx.x == 0) atomicOr(flag, 2);
}

}  // namespace

// ----------------------------------------------------------------------------- launchers

cudaError_t launch_bounded_wait_probe(int* flag, cudaStream_t s) {
  k_bounded_wait_probe<<<1, 32, 0, s>>>(flag, reinterpret_cast<unsigned*>(flag + 1));
  return cudaGetLastError();
}

cudaError_t mlp_gemm_setup() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_mlp_gemm<kEpiRelu>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_gemm<kEpiOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem)))
    return e;
  return cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
}

namespace {

template <int EPI>
cudaError_t gemm(const GemmArgs& a, dim3 grid, cudaStream_t s) {
  // every launch takes the full shared-memory budget: at most three CTAs share an SM, so
  // their tensor-memory allocations (128 columns each) always fit in its 512 columns
  return launch_dep_smem(k_mlp_gemm<EPI>, grid, dim3(kGemmThreads), kGemmSmem, s, a);
}

GemmArgs base(const __nv_bfloat16* A, int64_t lda, int M, const __nv_bfloat16* B, int N, int* err) {
  GemmArgs a{};
  a.A = A;
  a.lda = lda;
  a.M = M;
  a.B = B;
  a.N = N;
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

// Inference: X [n][128] -> y [n][9]; three launches.
cudaError_t launch_mlp_forward(const MlpState& st, const MlpWork& wk, int64_t n, const uint16_t* X_, float* y,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const __nv_bfloat16* X = reinterpret_cast<const __nv_bfloat16*>(X_);
  const dim3 grid((unsigned)((n + kTileM - 1) / kTileM), 1);
  cudaError_t e;
  GemmArgs a = base(X, kMlpIn, (int)n, st.w1b, 128, wk.err);
  a.bias = st.param + kMlpB1;
  a.out = wk.h1;
  a.ldo = kMlpHidden;
  if ((e = gemm<kEpiRelu>(a, grid, s))) return e;
  a = base(wk.h1, kMlpHidden, (int)n, st.w2b, 128, wk.err);
  a.bias = st.param + kMlpB2;
  a.out = wk.h2;
  a.ldo = kMlpHidden;
  if ((e = gemm<kEpiRelu>(a, grid, s))) return e;
  a = base(wk.h2, kMlpHidden, (int)n, st.w3b, kMlpOutPad, wk.err);
  a.bias = st.param + kMlpB3;
  a.y = y;
  return gemm<kEpiOut>(a, grid, s);
}

// Training launch: `steps` Adam steps on consecutive batches of `batch` rows (grad_mode:
// the gradient of one batch into grads).  One cooperative launch of one CTA per SM (the
// kernel's grid barriers need every CTA resident); the barrier counter and the per-step
// losses are cleared first.
cudaError_t launch_mlp_train(const MlpState& st, const dqo_mlp_hparams& hp, bool grad_mode, int steps,
                             int64_t batch, const uint16_t* X_, const float* labels, float* losses, float* grads,
                             const MlpWork& wk, cudaStream_t s) {
  if (steps <= 0 || batch <= 0 || batch % kTileM || (grad_mode && (steps != 1 || !grads))) return cudaErrorInvalidValue;
  // the grid: the device's SMs x resident CTAs of this kernel per SM (one, by shared memory)
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_train, kTrainThreads, kTrainSmem)))
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = sms * per_sm;
  if ((e = cudaMemsetAsync(wk.bar, 0, sizeof(unsigned), s))) return e;
  if (losses && (e = cudaMemsetAsync(losses, 0, sizeof(float) * steps, s))) return e;
  TrainArgs a{};
  a.st = st;
  a.hp = hp;
  a.X = reinterpret_cast<const __nv_bfloat16*>(X_);
  a.labels = labels;
  a.losses = losses;
  a.grads = grads;
  a.gpart = wk.gpart;
  a.bar = wk.bar;
  a.err = wk.err;
  a.steps = steps;
  a.tiles = (int)(batch / kTileM);
  a.mode = grad_mode ? kTrainGrad : kTrainAdam;
  a.inv_batch = 1.f / (float)batch;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kTrainThreads);
  cfg.dynamicSmemBytes = kTrainSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mlp_train, a);
}

}  // namespace dqo
