// Learned quadric proposal: a perceptron 128 -> 128 -> 128 -> 9 with ReLU, its adjoint and
// its Adam update.  Every product runs on the 5th-generation tensor cores: tcgen05.mma of
// kind f16 with BF16 operands staged in shared memory and FP32 accumulators in tensor
// memory, issued by one thread per CTA; the epilogues (bias, ReLU, the regression loss,
// the ReLU derivative, the gradient stores) read the accumulators back with tcgen05.ld.
//
// Inference (k_mlp_gemm, one launch per layer): a CTA computes a 128-row tile
// D[128][N] = A[128][K] . B[N][K]^T (N = 16 or 128, K = 128) with both operands
// K-contiguous in global memory (A = activations, B = weights [out][in]).  Training
// (k_mlp_train_fused): the whole step of 128 samples per CTA in one kernel, then Adam.
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
  // D[m][n] = sum_k A[m0 + m][k] B[n][k]
  const __nv_bfloat16* A;
  int64_t lda;
  int M;  // valid rows of A (rows past it are zero)
  const __nv_bfloat16* B;
  int64_t ldb;
  int N;  // 16 or 128
  int K;  // multiple of 16, <= 128
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
  unsigned char* sb = sm + kTileM * a.K * 2;
  if (w == 0) {
    tmem_alloc(smem_u32(&tslot), kTmemCols);
    tmem_relinquish();
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  load_tile(sa, a.A + (int64_t)m0 * a.lda, a.lda, kTileM, min(kTileM, a.M - m0), a.K);
  load_tile(sb, a.B, a.ldb, a.N, a.N, a.K);
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
// the 128 samples of one CTA, in one kernel with every intermediate in shared memory.
//
// Layout: every tile [R][C] (C contiguous in global memory) is stored as a plain grid of
// 8 x 8 core matrices, core (r / 8, c / 8) at (r / 8) * 16 C + (c / 8) * 128 bytes, each core
// 8 rows of 16 contiguous bytes.  The same bytes are a valid tcgen05 operand both ways:
// K-major (rows = M or N, K = the columns: leading offset 128 B between the two K cores of
// a 16-wide K step, stride offset 16 C B between row groups, 256 B per K step) and MN-major
// (M or N = the columns, K = the rows: stride offset 128 B between column groups, leading
// offset 16 C B between the two K cores, 32 C B per K step; bits 15 / 16 of the instruction
// descriptor).  So a transposed operand (H1^T, X^T, W2^T, ...) is the stored tile read the
// other way, and no transposed copy is written.
//
// Bias gradients come out of the weight-gradient products: the X and H1 tiles carry 16
// extra columns of ones (C = 144), so G1^T [X | 1] and G2^T [H1 | 1] give dW1 | db1 and
// dW2 | db2 in one product each (column 128 of the result is the row sum); db3 is a warp
// and block sum of dY.  Products that do not depend on each other (G2 and dW3; G1 and
// dW2) are issued together into the two halves of a 512-column tensor-memory allocation
// (one CTA per SM: the shared memory allows no second).
//
// Two warps share each 32-lane quarter of tensor memory (one accumulator row per lane):
// warp w reads lanes 32 (w % 4) .. + 31 and the columns [64 (w / 4), + 64) of a 128-column
// result, so every epilogue is split across 256 threads; each thread loads its 64 columns
// with one tensor-memory load and one wait.
//
// Shared memory (bytes): X | 1 (36 K, all step) | H1 | 1 (36 K) | W1, then H2, then G1
// (32 K) | W2 (32 K) | G2 (32 K) | W3 [16][128] (4 K) | dY [128][16] (4 K) | b1 b2 b3 |
// db3 per warp | the CTA's labels [128][9].
constexpr int kFusedThreads = 256;
constexpr int kXC = kMlpIn + 16;        // columns of the X and H1 tiles: the values, then ones
constexpr uint32_t kTileX = kTileM * kXC * 2;
constexpr uint32_t kTileW = 128 * 128 * 2;
constexpr uint32_t kTile16 = 128 * kMlpOutPad * 2;
constexpr int kBiasFloats = 2 * kMlpHidden + kMlpOutPad;
constexpr uint32_t kOffX = 0, kOffH1 = kOffX + kTileX, kOffS = kOffH1 + kTileX, kOffW2 = kOffS + kTileW,
                   kOffG2 = kOffW2 + kTileW, kOffW3 = kOffG2 + kTileW, kOffDY = kOffW3 + kTile16,
                   kOffBias = kOffDY + kTile16, kOffDb3 = kOffBias + kBiasFloats * 4,
                   kOffLab = kOffDb3 + 4 * kMlpOutPad * 4, kFusedBytes = kOffLab + kTileM * 9 * 4;
constexpr int kFusedSmem = (int)kFusedBytes + 1024;
constexpr uint32_t kFusedCols = 512;

struct FusedArgs {
  MlpState st;
  const __nv_bfloat16* X;   // [n][128]
  const float* labels;      // [n][9]
  float w[9];
  float inv_batch;
  float* loss;              // += sum of the batch's weighted squared errors / n
  int* step_inc;            // block 0 adds 1 (the optimiser's step count); may be NULL
  int* err;                 // set to 1 if a tensor-core wait timed out
  float* gpart;             // [gridDim.x][kMlpParams]: this CTA's gradient
};

// Byte offset of element (r, c) of a grid-layout tile of C columns.
__device__ __forceinline__ uint32_t grid_off(int r, int c, int C) {
  return (uint32_t)((r >> 3) * (C >> 3) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}
// rows x K block of a row-major global matrix (ld elements, 16-byte aligned rows) into
// columns [0, K) of a grid tile of C columns, by cp.async (committed by the caller).
__device__ __forceinline__ void load_grid_async(unsigned char* dst, const __nv_bfloat16* __restrict__ src,
                                                int64_t ld, int rows, int K, int C) {
  const int per_row = K >> 3;
  for (int i = threadIdx.x; i < rows * per_row; i += blockDim.x) {
    const int r = i / per_row, kc = i - r * per_row;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + grid_off(r, kc * 8, C))),
                 "l"(src + (int64_t)r * ld + kc * 8)
                 : "memory");
  }
}
// Thread m's 16 values for columns [c, c + 16) of row m of a grid tile of C columns.
__device__ __forceinline__ void put_grid16(unsigned char* tile, int C, int m, int c, const __nv_bfloat16 (&h)[16]) {
  *reinterpret_cast<uint4*>(tile + grid_off(m, c, C)) = reinterpret_cast<const uint4*>(h)[0];
  *reinterpret_cast<uint4*>(tile + grid_off(m, c + 8, C)) = reinterpret_cast<const uint4*>(h)[1];
}

// One operand of a product: a grid tile read K-major (rows = M or N) or MN-major (columns =
// M or N, rows = K).
struct Opnd {
  uint32_t addr;
  int C;
  bool mn;
};
__device__ __forceinline__ uint64_t opnd_desc(const Opnd& o, int kstep) {
  const uint32_t lbo = o.mn ? 16u * (uint32_t)o.C : 128u, sbo = o.mn ? 128u : 16u * (uint32_t)o.C;
  const uint32_t a = o.addr + (uint32_t)kstep * (o.mn ? 32u * (uint32_t)o.C : 256u);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
// D[tmem][128][N] = A . B^T over K (multiple of 16); called by thread 0.
__device__ __forceinline__ void issue_product(uint32_t tmem, const Opnd& A, const Opnd& B, int N, int K) {
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((A.mn ? 1u : 0u) << 15) | ((B.mn ? 1u : 0u) << 16) |
                         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
  for (int s = 0; s < (K >> 4); ++s) mma_bf16(tmem, opnd_desc(A, s), opnd_desc(B, s), idesc, s > 0 ? 1u : 0u);
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

// Epilogue of a 128-row activation tile: thread (row r, half g) turns its 64 accumulator
// columns into BF16 values (ReLU of the sum with the bias when `bias` is set, else the
// accumulator masked by the ReLU derivative `mask`), stores them into row r of a grid tile
// of C columns, and (with the bias) records which are positive in `mask`.
template <bool kRelu>
__device__ __forceinline__ void act_epilogue(uint32_t taddr, const float* bias, uint32_t (&mask)[2],
                                             unsigned char* tile, int C, int r, int c0) {
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
    put_grid16(tile, C, r, c0 + 16 * q, h);
  }
}
// Epilogue of a weight-gradient result [128][128 | ones]: thread (row r, half g) stores its
// 64 columns into row r of the gradient block dw [128][128]; half 1 also stores column 128
// (the row sum: the bias gradient) into db[r].
__device__ __forceinline__ void wgrad_epilogue(uint32_t taddr, float* dw, float* db, int r, int g) {
  float v[64];
  tmem_ld64(taddr + (uint32_t)(64 * g), v);
  float4* d4 = reinterpret_cast<float4*>(dw + (int64_t)r * 128 + 64 * g);
#pragma unroll
  for (int q = 0; q < 16; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  if (g == 1) {
    float b[16];
    tmem_ld16(taddr + 128u, b);
    db[r] = b[0];
  }
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_mlp_train_fused(FusedArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  pdl_wait();
  pdl_trigger();
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int g = w >> 2;              // column half of a 128-column result
  const int r = (w & 3) * 32 + lane; // accumulator row (TMEM lane) of this thread
  const int c0 = 64 * g;
  const int64_t m0 = (int64_t)blockIdx.x * kTileM;
  unsigned char* sX = sm + kOffX;
  unsigned char* sH1 = sm + kOffH1;
  unsigned char* sS = sm + kOffS;    // W1, then H2, then G1
  unsigned char* sW2 = sm + kOffW2;
  unsigned char* sG2 = sm + kOffG2;
  unsigned char* sW3 = sm + kOffW3;
  unsigned char* sDY = sm + kOffDY;
  float* sbias = reinterpret_cast<float*>(sm + kOffBias);   // b1, b2, b3
  float* sdb3 = reinterpret_cast<float*>(sm + kOffDb3);     // [warp][16]
  const float* slab = reinterpret_cast<const float*>(sm + kOffLab);
  const MlpState& st = a.st;
  float* const gp = a.gpart + (int64_t)blockIdx.x * kMlpParams;   // this CTA's gradient
  if (a.step_inc && t == 0 && blockIdx.x == 0) atomicAdd(a.step_inc, 1);
  if (w == 0) {
    tmem_alloc(smem_u32(&tslot), kFusedCols);
    tmem_relinquish();
  }
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  const uint32_t bar = smem_u32(&mbar);
  load_grid_async(sX, a.X + m0 * kMlpIn, kMlpIn, kTileM, kMlpIn, kXC);
  load_grid_async(sS, st.w1b, kMlpIn, kMlpHidden, kMlpIn, 128);
  cp_async_commit();
  load_grid_async(sW2, st.w2b, kMlpHidden, kMlpHidden, kMlpHidden, 128);
  load_grid_async(sW3, st.w3b, kMlpHidden, kMlpOutPad, kMlpHidden, 128);
  {
    // the CTA's labels: 128 x 9 floats, contiguous and 16-byte aligned (m0 is a multiple of 128)
    const float* lab = a.labels + m0 * 9;
    for (int i = t; i < kTileM * 9 / 4; i += kFusedThreads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sm + kOffLab + 16 * i)),
                   "l"(lab + 4 * i)
                   : "memory");
  }
  cp_async_commit();
  {
    // the ones columns [128, 144) of the X and H1 tiles: two 16-byte rows per tile row
    const uint4 ones = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    for (int i = t; i < 4 * kTileM; i += kFusedThreads) {
      unsigned char* tile = (i & 2) ? sH1 : sX;
      *reinterpret_cast<uint4*>(tile + grid_off(i >> 2, kMlpIn + 8 * (i & 1), kXC)) = ones;
    }
  }
  for (int i = t; i < kBiasFloats; i += kFusedThreads)
    sbias[i] = i < kMlpHidden ? st.param[kMlpB1 + i]
                              : (i < 2 * kMlpHidden ? st.param[kMlpB2 + i - kMlpHidden]
                                                    : st.param[kMlpB3 + i - 2 * kMlpHidden]);
  cp_async_wait_group<1>();
  __syncthreads();
  const uint32_t t0 = tslot, t1 = t0 + 256u, lane_off = (uint32_t)((w & 3) * 32) << 16;
  const uint32_t a0 = t0 + lane_off, a1 = t1 + lane_off;   // this thread's row in the two halves
  const Opnd X{smem_u32(sX), kXC, false}, XT{smem_u32(sX), kXC, true};
  const Opnd H1{smem_u32(sH1), kXC, false}, H1T{smem_u32(sH1), kXC, true};
  const Opnd S{smem_u32(sS), 128, false}, ST{smem_u32(sS), 128, true};
  const Opnd W2{smem_u32(sW2), 128, false}, W2T{smem_u32(sW2), 128, true};
  const Opnd G2{smem_u32(sG2), 128, false}, G2T{smem_u32(sG2), 128, true};
  const Opnd W3{smem_u32(sW3), 128, false}, W3T{smem_u32(sW3), 128, true};
  const Opnd DY{smem_u32(sDY), kMlpOutPad, false}, DYT{smem_u32(sDY), kMlpOutPad, true};
  uint32_t ph = 0;
  bool ok = true;
  uint32_t mask1[2] = {0u, 0u}, mask2[2] = {0u, 0u};   // ReLU masks of this thread's 64 columns

  // ---- H1 = relu(X W1^T + b1) [samples][h1]
  round_begin();
  if (t == 0) issue_product(t0, X, S, 128, kMlpIn);
  ok = round_end(bar, ph);
  ph ^= 1u;
  if (ok) {
    act_epilogue<true>(a0 + (uint32_t)c0, sbias, mask1, sH1, kXC, r, c0);
    cp_async_wait_all();   // W2, W3, labels
  }
  // ---- H2 = relu(H1 W2^T + b2) [samples][h2], into the W1 slot
  if (ok) {
    round_begin();
    if (t == 0) issue_product(t1, H1, W2, 128, kMlpHidden);
    ok = round_end(bar, ph);
    ph ^= 1u;
  }
  if (ok) act_epilogue<true>(a1 + (uint32_t)c0, sbias + kMlpHidden, mask2, sS, 128, r, c0);
  // ---- Y = H2 W3^T + b3, the loss, dY = 2 w (y - label) / n [samples][16], db3 (warps 0-3)
  if (ok) {
    round_begin();
    if (t == 0) issue_product(t0, S, W3, kMlpOutPad, kMlpHidden);
    ok = round_end(bar, ph);
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
      l += a.w[j] * e * e;
      d[j] = __float2bfloat16_rn(2.f * a.w[j] * e * a.inv_batch);
    }
#pragma unroll
    for (int j = 9; j < 16; ++j) d[j] = __float2bfloat16_rn(0.f);
    put_grid16(sDY, kMlpOutPad, r, 0, d);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const float s = warp_sum_f(__bfloat162float(d[j]));
      if (lane == 0) sdb3[w * kMlpOutPad + j] = s;
    }
    if (a.loss) {
      l = warp_sum_f(l * a.inv_batch);
      if (lane == 0) atomicAdd(a.loss, l);
    }
  }
  // ---- G2 = (dY W3) * (H2 > 0) [samples][h2] and dW3 = dY^T H2 [h2][16] (transposed)
  if (ok) {
    round_begin();
    if (t == 0) {
      issue_product(t0, DY, W3T, 128, kMlpOutPad);
      issue_product(t1, ST, DYT, kMlpOutPad, kTileM);
    }
    ok = round_end(bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    act_epilogue<false>(a0 + (uint32_t)c0, nullptr, mask2, sG2, 128, r, c0);
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
  // ---- G1 = (G2 W2) * (H1 > 0) [samples][h1], into the H2 slot; dW2 | db2 = G2^T [H1 | 1]
  if (ok) {
    round_begin();
    if (t == 0) {
      issue_product(t0, G2, W2T, 128, kMlpHidden);
      issue_product(t1, G2T, H1T, kXC, kTileM);
    }
    ok = round_end(bar, ph);
    ph ^= 1u;
  }
  if (ok) {
    act_epilogue<false>(a0 + (uint32_t)c0, nullptr, mask1, sS, 128, r, c0);
    wgrad_epilogue(a1, gp + kMlpW2, gp + kMlpB2, r, g);
  }
  // ---- dW1 | db1 = G1^T [X | 1] [h1][in + 1]
  if (ok) {
    round_begin();
    if (t == 0) issue_product(t0, ST, XT, kXC, kTileM);
    ok = round_end(bar, ph);
    ph ^= 1u;
  }
  if (ok) wgrad_epilogue(a0, gp + kMlpW1, gp + kMlpB1, r, g);
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
// g0 + the fused step's per-CTA gradient entries i, added in block order; eight loads in
// flight at a time.
__device__ __forceinline__ float sum_partials(const float* __restrict__ gpart, int nb, int i, float g0) {
  float g = g0;
  int b = 0;
  for (; b + 8 <= nb; b += 8) {
    float p[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) p[u] = __ldcg(gpart + (int64_t)(b + u) * kMlpParams + i);
#pragma unroll
    for (int u = 0; u < 8; ++u) g += p[u];
  }
  for (; b < nb; ++b) g += __ldcg(gpart + (int64_t)b * kMlpParams + i);
  return g;
}

__global__ void k_mlp_adam(MlpState st, dqo_mlp_hparams hp, const float* __restrict__ gpart, int nb) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const int step = *st.step;
  const float g = sum_partials(gpart, nb, i, st.grad[i]);
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
  out[i] = sum_partials(gpart, nb, i, 0.f);
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
// products of a training step fused, intermediates in shared memory).  Each CTA's
// gradient goes to gpart[blockIdx]; the loss is ADDED to *loss.
cudaError_t launch_mlp_backward_fused(const MlpState& st, int* err, float* gpart, int64_t n, const uint16_t* X_,
                                      const float* labels, const float* loss_w, float* loss, int* step_inc,
                                      cudaStream_t s) {
  if (n <= 0 || n % kTileM || !gpart) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.st = st;
  a.gpart = gpart;
  a.X = reinterpret_cast<const __nv_bfloat16*>(X_);
  a.labels = labels;
#pragma unroll
  for (int j = 0; j < 9; ++j) a.w[j] = loss_w[j];
  a.inv_batch = 1.f / (float)n;
  a.loss = loss;
  a.step_inc = step_inc;
  a.err = err;
  return launch_dep_smem(k_mlp_train_fused, dim3((unsigned)(n / kTileM)), dim3(kFusedThreads), kFusedSmem, s, a);
}

}  // namespace dqo
