// Learned sampling proposal (an extension of the method; the paper has no learning): a small MLP
// whose products run on the tensor cores in BF16 with FP32 accumulation, FP32 master weights and
// Adam state, and a training loop that stays on the device.
//
// Network.  dims[0] -> dims[1] -> ... -> dims[L]; ReLU after every layer but the last.  Inputs:
// the environment's features (obstacle boxes, start, goal), eight standard normals z, zeros.  The
// first six outputs o are squashed into the state box: position 0.5 + 0.5 tanh(o), velocity
// vmax tanh(o).  Loss over the row's targets y_0 .. y_{n-1} (the states along a solution path, in
// path order), averaged over the batch: winner takes all, min_p |s - y_p|^2, or path-indexed,
// |s - y(u)|^2 with u = Phi(z_0) and y(u) the point at fraction u of the polyline by node index.
//
// Parameters live in one flat FP32 vector (per layer W (out x in, row-major) then b), with Adam's
// moments and a BF16 copy beside it, so one launch updates every layer.
//
// Products, all on the 5th-generation tensor cores (k_gemm_tc, tcgen05.mma with TMEM accumulators,
// operands brought in by TMA tensor copies):
//   forward   pre_l  = h_l W_l^T     A = h_l (K-major), B = W_l (K-major)
//   backward  dh_l   = g_l W_l       A = g_l (K-major), B = W_l^T (K-major copy kept by Adam)
//             dW_l   = g_l^T h_l     A = g_l, B = h_l, both MN-major (consecutive m or n in memory),
//                                    split over K (the batch); db_l from the same products
// so no activation or gradient is ever transposed in memory.  The epilogues are fused: bias + ReLU
// to BF16, bias to FP32, ReLU mask of the layer below to BF16, or plain FP32 partial sums (split K).
// The weight-gradient partials of the S splits stay separate and the Adam launch adds them in a
// fixed order, so a training step is deterministic.
//
// Device-side step counter.  ctl[0] counts the Adam steps taken; the batch assembly of step t
// draws with t, the loss kernel advances the counter, and Adam corrects its moments with the new
// count.  Nothing in a step depends on a host value that changes between steps, so one step is
// captured once as a CUDA graph and replayed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pump_internal.cuh"

namespace pump {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kLatent = 8;
constexpr int kOutUsed = 6;
constexpr int kMaxSplit = 32;
constexpr int kLossThreads = 256;
constexpr int kLossBlocksMax = 1024;

enum Epi : int {
  kEpiBiasRelu = 0,  // out_bf16 = bf16(relu(acc + bias))
  kEpiBias = 1,      // out_f32 = acc + bias
  kEpiMask = 2,      // out_bf16 = bf16(acc * (mask > 0))
  kEpiPartial = 3,   // out_f32[split] = acc
};

struct GemmArgs {
  const bf16* A;  // K-major: M x K (lda = row stride); M-major: K x M (lda = row stride)
  const bf16* B;  // K-major: N x K;                    N-major: K x N
  int lda, ldb;
  int M, N, K;
  int kchunk;     // split z covers k in [z kchunk, min(K, (z + 1) kchunk))
  const float* bias;
  const bf16* mask;
  bf16* out_bf16;
  float* out_f32;
  int ldo;               // output row stride (elements)
  int64_t split_stride;  // offset between the splits' outputs (kEpiPartial)
  float* colsum;         // kEpiPartial with an M-major A: also sum_k A[k][m] per split (bias gradient), or null
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------------------------
// GEMM on the 5th-generation tensor cores: C[M x N] = A[M x K] B[N x K]^T, both operands K-major
// BF16, accumulator FP32 in tensor memory.  A block owns 128 rows (the accumulator's 128 TMEM
// lanes) and tileN <= 256 columns (TMEM columns); K goes 64 at a time through kTcStages shared
// buffers.  The tensor memory accelerator copies each operand's 64-wide K step as one box of
// 128-byte rows in the 128-byte swizzled layout (16-byte chunks of row r XOR-permuted by r mod 8,
// 8-row groups 1024 B apart), the layout the descriptors name; a K = 16 step of the products starts
// 32 B further along the rows.  Rows past the end and K past the end arrive as zeros.  One thread drives the loop: it
// starts the copies (completion counted in bytes on a per-buffer "full" mbarrier), issues the
// tcgen05.mma instructions (M 128, N tileN, K 16), commits them to the buffer's "empty" mbarrier,
// and refills the buffer once that one has fired; the last commit tells the epilogue that the
// accumulator is complete.  Every mbarrier wait is bounded: on expiry the block records an error,
// skips its epilogue and still frees its tensor memory.  The epilogue reads the accumulator with
// tcgen05.ld (warp w: lanes 32w .. 32w + 31, 16 columns at a time) and applies the fused
// operations listed at the top of this file.
constexpr int kTcM = 128, kTcNMax = 256, kTcK = 64, kTcStages = 4, kTcThreads = 128;
constexpr int kTcStageBytes = (kTcM + kTcNMax) * kTcK * 2;  // 48 KB
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024;   // + alignment
constexpr long long kTcSpin = 1ll << 26;                    // mbarrier polls before giving up

struct TcArgs {
  int M, N, K, tileN, cols;  // cols: TMEM columns of a block (power of 2, >= 32, >= tileN)
  const float* bias;
  const bf16* mask;
  bf16* out_bf16;
  float* out_f32;
  int ldo;
  int* err;
  // weight-gradient form (MN-major operands, kEpiPartial): split z covers k in [z kchunk,
  // (z + 1) kchunk) (kchunk a multiple of kTcK) and writes out_f32 + z split_stride; blocks of the
  // first N tile also write the split's column sums of A to colsum + z split_stride
  int kchunk;
  int64_t split_stride;
  float* colsum;
};

constexpr int kTcMnBox = 64;          // M/N elements of one MN-major box (128 B rows)
constexpr int kTcMnBoxBytes = kTcK * kTcMnBox * 2;  // 8 KB: 64 K rows of 128 B
constexpr int kTcOnes = 16;           // extra accumulator columns of the column sums (N step)

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled layout: start
// address, leading offset 16 B (not used by this layout), 8-row groups 1024 B apart, version 1,
// layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Descriptor of an MN-major operand in the 128-byte swizzled layout: each box holds 64 K rows of
// 64 M (or N) elements (128 B), so 8-row K groups are 1024 B apart (stride offset) and successive
// 64-wide M/N blocks kTcMnBoxBytes apart (leading offset); a K = 16 step starts 16 rows (2048 B)
// further on.
__device__ __forceinline__ uint64_t tc_desc_mn(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kTcMnBoxBytes >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kTcSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// One K step of both operands into a buffer: A rows m0 .. m0+127, B rows n0 .. n0+tileN-1, K groups
// kc*8 .. kc*8+7; the full mbarrier expects the two boxes' bytes.
__device__ __forceinline__ void tc_load(const CUtensorMap* tmA, const CUtensorMap* tmB, uint32_t sa, uint32_t sb,
                                        uint32_t full, int m0, int n0, int kc, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          sa),
      "l"((uint64_t)tmA), "r"(kc * kTcK), "r"(m0), "r"(full)
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          sb),
      "l"((uint64_t)tmB), "r"(kc * kTcK), "r"(n0), "r"(full)
      : "memory");
}

// One K step of MN-major operands: A (M 128) as two 64-wide boxes, B as tileN / 64 boxes, each box
// 64 K rows from k; the full mbarrier expects every box's bytes.
__device__ __forceinline__ void tc_load_mn(const CUtensorMap* tmA, const CUtensorMap* tmB, uint32_t sa, uint32_t sb,
                                           uint32_t full, int m0, int n0, int k, int nbox_b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full), "r"(bytes) : "memory");
#pragma unroll
  for (int h = 0; h < kTcM / kTcMnBox; ++h)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            sa + h * kTcMnBoxBytes),
        "l"((uint64_t)tmA), "r"(m0 + h * kTcMnBox), "r"(k), "r"(full)
        : "memory");
  for (int j = 0; j < nbox_b; ++j)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            sb + j * kTcMnBoxBytes),
        "l"((uint64_t)tmB), "r"(n0 + j * kTcMnBox), "r"(k), "r"(full)
        : "memory");
}

// kMN: the weight-gradient form, C = A^T B over the batch with A (K x M) and B (K x N) stored
// MN-major (row k holds consecutive m or n): the TMA boxes are 64 K rows x 64 M/N elements, the
// descriptors MN-major (tc_desc_mn) and the instruction descriptor transposes both operands.
// Blocks of the first N tile append a 64-wide block of BF16 ones to their B tile and run the
// products kTcOnes columns wider: accumulator column tileN then holds sum_k A[k][m] (the bias
// gradient), summed by the same tensor-core products.
template <int kEpi, bool kMN = false, int kSt = kTcStages>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, const TcArgs g) {
  extern __shared__ uint8_t tc_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[kSt], empty[kSt], done;
  __shared__ int ok_all;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * g.tileN;
  const int nt = min(g.tileN, g.N - n0);
  // K range: the whole of K, or split blockIdx.z of the weight-gradient form
  const int kb = kMN ? blockIdx.z * g.kchunk : 0;
  const int ke = kMN ? min(g.K, kb + g.kchunk) : g.K;
  const int nk = ke > kb ? (ke - kb + kTcK - 1) / kTcK : 0;
  const bool sums = kMN && g.colsum != nullptr && blockIdx.x == 0;  // this block adds the ones block
  const int nbox_b = g.tileN / kTcMnBox;
  const uint32_t bytes = (uint32_t)(kTcM + g.tileN) * kTcK * 2;  // TMA bytes per K step
  const uint32_t b_bytes = (uint32_t)(g.tileN + (kMN ? kTcMnBox : 0)) * kTcK * 2;
  const uint32_t stage = ((uint32_t)kTcM * kTcK * 2 + b_bytes + 1023) & ~1023u;  // buffer stride
  const int nmma = sums ? g.tileN + kTcOnes : g.tileN;  // N of the products (weight-gradient form)
  if (kMN && sums) {
    // the ones block after each buffer's B boxes (never written by the copies)
    const uint32_t one2 = 0x3F803F80u;
    for (int b = 0; b < kSt; ++b) {
      uint32_t* o = reinterpret_cast<uint32_t*>(smem + b * stage + kTcM * kTcK * 2 + nbox_b * kTcMnBoxBytes);
      for (int q = tid; q < kTcMnBoxBytes / 4; q += kTcThreads) o[q] = one2;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor cores
  }
  if (tid == 0) {
    for (int b = 0; b < kSt; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&empty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    ok_all = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(g.cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    // kind::f16: D F32, A and B BF16, both K-major (or both MN-major: transpose bits 15, 16),
    // N = nmma, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (kMN ? (1u << 15) | (1u << 16) : 0u) |
                           ((uint32_t)((kMN ? nmma : nt) >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t base = smem_addr(smem);
    bool ok = true;
    for (int c = 0; c < kSt && c < nk; ++c) {
      const uint32_t sa = base + c * stage;
      if (kMN)
        tc_load_mn(&tmA, &tmB, sa, sa + kTcM * kTcK * 2, smem_addr(&full[c]), m0, n0, kb + c * kTcK, nbox_b, bytes);
      else
        tc_load(&tmA, &tmB, sa, sa + kTcM * kTcK * 2, smem_addr(&full[c]), m0, n0, c, bytes);
    }
    for (int c = 0; c < nk && ok; ++c) {
      const int st = c % kSt;
      const uint32_t ph = (uint32_t)((c / kSt) & 1);
      if (!mbar_wait(smem_addr(&full[st]), ph)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t a0 = base + st * stage, b0 = a0 + kTcM * kTcK * 2;
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        const uint64_t da = kMN ? tc_desc_mn(a0 + kk * 2048) : tc_desc(a0 + kk * 32);
        const uint64_t db = kMN ? tc_desc_mn(b0 + kk * 2048) : tc_desc(b0 + kk * 32);
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(&empty[st])));
      if (c + kSt < nk) {
        if (!mbar_wait(smem_addr(&empty[st]), ph)) {
          ok = false;
          break;
        }
        if (kMN)
          tc_load_mn(&tmA, &tmB, a0, b0, smem_addr(&full[st]), m0, n0, kb + (c + kSt) * kTcK, nbox_b, bytes);
        else
          tc_load(&tmA, &tmB, a0, b0, smem_addr(&full[st]), m0, n0, c + kSt, bytes);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(&done)));
    if (!ok) ok_all = 0;
  }
  __syncthreads();
  if (!mbar_wait(smem_addr(&done), 0u)) atomicExch(&ok_all, 0);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (ok_all && kMN && nk == 0) {
    // an empty split (K past the end): zero partials
    const int r = m0 + warp * 32 + lane;
    if (r < g.M) {
      float* out = g.out_f32 + blockIdx.z * g.split_stride + (size_t)r * g.ldo + n0;
      for (int c = 0; c < nt; ++c) out[c] = 0.f;
      if (sums) g.colsum[blockIdx.z * g.split_stride + r] = 0.f;
    }
  } else if (ok_all && kMN) {
    const int r = m0 + warp * 32 + lane;
    float* out = g.out_f32 + blockIdx.z * g.split_stride + (size_t)r * g.ldo + n0;
    for (int c00 = 0; c00 < nt; c00 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
            "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c00));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
      if (r < g.M) {
        if (c00 + 16 <= nt && (g.ldo & 3) == 0 && (n0 & 3) == 0) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(out + c00 + j) = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                                    __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c00 + j < nt) out[c00 + j] = __uint_as_float(v[j]);
        }
      }
    }
    if (sums) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
            "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)g.tileN));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
      if (r < g.M) g.colsum[blockIdx.z * g.split_stride + r] = __uint_as_float(v[0]);
    }
  } else if (ok_all) {
    const int r = m0 + warp * 32 + lane;
    for (int c00 = 0; c00 < nt; c00 += 32) {
      uint32_t vv[2][16];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (c00 + 16 * h < nt)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];\n"
              : "=r"(vv[h][0]), "=r"(vv[h][1]), "=r"(vv[h][2]), "=r"(vv[h][3]), "=r"(vv[h][4]), "=r"(vv[h][5]),
                "=r"(vv[h][6]), "=r"(vv[h][7]), "=r"(vv[h][8]), "=r"(vv[h][9]), "=r"(vv[h][10]), "=r"(vv[h][11]),
                "=r"(vv[h][12]), "=r"(vv[h][13]), "=r"(vv[h][14]), "=r"(vv[h][15])
              : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c00 + 16 * h)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
      if (r >= g.M) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
      if (c00 + 16 * h >= nt) break;
      const uint32_t* v = vv[h];
      const int col = n0 + c00 + 16 * h;
      const size_t o = (size_t)r * g.ldo + col;
      if (kEpi == kEpiBias) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(g.out_f32 + o + j) =
              make_float4(__uint_as_float(v[j]) + g.bias[col + j], __uint_as_float(v[j + 1]) + g.bias[col + j + 1],
                          __uint_as_float(v[j + 2]) + g.bias[col + j + 2], __uint_as_float(v[j + 3]) + g.bias[col + j + 3]);
      } else {
        uint32_t pk[8];
        if (kEpi == kEpiBiasRelu) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(__uint_as_float(v[j]) + g.bias[col + j], 0.f),
                                                           fmaxf(__uint_as_float(v[j + 1]) + g.bias[col + j + 1], 0.f));
            pk[j / 2] = *reinterpret_cast<const uint32_t*>(&h);
          }
        } else {  // kEpiMask
          const uint4 m4a = *reinterpret_cast<const uint4*>(g.mask + o);
          const uint4 m4b = *reinterpret_cast<const uint4*>(g.mask + o + 8);
          const bf16* mk = reinterpret_cast<const bf16*>(&m4a);
          const bf16* mk2 = reinterpret_cast<const bf16*>(&m4b);
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const float k0 = __bfloat162float(j < 8 ? mk[j] : mk2[j - 8]);
            const float k1 = __bfloat162float(j < 8 ? mk[j + 1] : mk2[j - 7]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(k0 > 0.f ? __uint_as_float(v[j]) : 0.f,
                                                           k1 > 0.f ? __uint_as_float(v[j + 1]) : 0.f);
            pk[j / 2] = *reinterpret_cast<const uint32_t*>(&h);
          }
        }
        *reinterpret_cast<uint4*>(g.out_bf16 + o) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(g.out_bf16 + o + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
      }
    }
  } else if (tid == 0) {
    atomicExch(g.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(g.cols));
}

__global__ void k_to_bf16(const float* __restrict__ in, int64_t n, bf16* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = __float2bfloat16_rn(in[k]);
}

__global__ void k_bf16_to_f32(const bf16* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = __bfloat162float(in[k]);
}

// Sum of the S gradient partials (for reading the gradient out).
__global__ void k_sum_parts(const float* __restrict__ part, int S, int64_t P, float* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    float t = 0.f;
    for (int s = 0; s < S; ++s) t += part[(int64_t)s * P + k];
    out[k] = t;
  }
}

// Box-Muller on the two 24-bit fields of a 64-bit word (bits 63..40 -> u1, 39..16 -> u2).
__device__ __forceinline__ void normal_pair(uint64_t w, float* z0, float* z1) {
  const float u1 = ((float)(uint32_t)(w >> 40) + 0.5f) * 5.9604644775390625e-08f;
  const float u2 = ((float)(uint32_t)((w >> 16) & 0xFFFFFFull) + 0.5f) * 5.9604644775390625e-08f;
  const float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  *z0 = r * cs;
  *z1 = r * sn;
}

// Network inputs of B rows: row r = [feat[env_r] (F), z_r (8), zeros] as BF16 (width d0).  Draw
// set (t, stream): z_r from Philox4x64-10 counter (t, r, stream, 0), key (seed, 1); with
// n_env > 0, env_r from counter (t, r, stream + 1, 0): floor((word0 >> 32) n_env / 2^32), else 0.
// t = ctl[0] when ctl is given, else 0.  Block: 16 rows.
__global__ void k_assemble(const float* __restrict__ feat, int F, int n_env, int d0, int B, uint64_t seed,
                           uint64_t stream_id, const int64_t* __restrict__ ctl, bf16* __restrict__ x,
                           int32_t* __restrict__ env_out) {
  __shared__ float z[16][kLatent];
  __shared__ int e[16];
  const int row0 = blockIdx.x * 16;
  if (threadIdx.x < 32) {
    const int rr = threadIdx.x & 15, r = row0 + rr;
    const uint64_t t = ctl ? (uint64_t)ctl[0] : 0ull;
    uint64_t o[4];
    if (threadIdx.x < 16) {
      philox4x64(t, (uint64_t)r, stream_id, 0ull, seed, 1ull, o);
#pragma unroll
      for (int j = 0; j < 4; ++j) normal_pair(o[j], &z[rr][2 * j], &z[rr][2 * j + 1]);
    } else {
      int env = 0;
      if (n_env > 0) {
        philox4x64(t, (uint64_t)r, stream_id + 1, 0ull, seed, 1ull, o);
        env = (int)(((o[0] >> 32) * (uint64_t)n_env) >> 32);
      }
      e[rr] = env;
      if (env_out && r < B) env_out[r] = env;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int rr = warp; rr < 16; rr += nwarp) {
    const int r = row0 + rr;
    if (r >= B) break;
    const float* f = feat + (size_t)e[rr] * F;
    bf16* xr = x + (size_t)r * d0;
    // eight columns per lane, one 16-byte store (d0 is a multiple of 16)
    for (int c0 = lane * 8; c0 < d0; c0 += 256) {
      uint32_t pk[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = c0 + j + h;
          v[h] = c < F ? f[c] : (c < F + kLatent ? z[rr][c - F] : 0.f);
        }
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
        pk[j / 2] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      *reinterpret_cast<uint4*>(xr + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

__device__ __forceinline__ float squash(float o, int j, float vmax) {
  return j < 3 ? 0.5f + 0.5f * tanhf(o) : vmax * tanhf(o);
}

__global__ void k_squash(const float* __restrict__ o, int B, int ld, float vmax, float* __restrict__ states) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B * kOutUsed) return;
  const int r = q / kOutUsed, j = q % kOutUsed;
  states[q] = squash(o[(size_t)r * ld + j], j, vmax);
}

struct LossArgs {
  int kind;          // 0 winner takes all, 1 path-indexed
  const bf16* x;     // network inputs (kind 1 reads the first latent at column latent_col)
  int d0, latent_col;
};

// Loss and its gradient.  Row r uses target set env[r] (r without env): targets
// tg[set][0 .. ntg[set]) of 6 floats.  Kind 0 takes the nearest target (first on ties); kind 1
// the point at fraction u = Phi(z_0) of the targets' polyline: a = u (n - 1),
// i = min(floor(a), n - 2), y = y_i + (a - i)(y_{i+1} - y_i).  Writes g = bf16(d mean loss / d o)
// (B x ld, zero past column 6) and, after a fixed-order reduction,
// trace[ctl[0] - ctl[1]] = mean loss (the blocks' sums added by the last block to finish in a fixed
// order: thread t adds blocks t, t + 256, ..., then a tree over the threads); then advances ctl[0].
__global__ void __launch_bounds__(kLossThreads) k_loss(const float* __restrict__ o, int B, int ld, float vmax,
                                                       const float* __restrict__ tg, const int32_t* __restrict__ ntg,
                                                       int T, const int32_t* __restrict__ env, const LossArgs la,
                                                       bf16* __restrict__ gout, int64_t* __restrict__ ctl,
                                                       float* __restrict__ trace, int trace_cap,
                                                       float* __restrict__ part, unsigned int* __restrict__ ticket) {
  __shared__ float red[kLossThreads];
  __shared__ bool last;
  float local = 0.f;
  for (int r = blockIdx.x * kLossThreads + threadIdx.x; r < B; r += gridDim.x * kLossThreads) {
    const int set = env ? env[r] : r;
    const float* q0 = tg + (size_t)set * T * kOutUsed;
    const int n = min(ntg[set], T);
    float s[kOutUsed], y[kOutUsed];
    for (int j = 0; j < kOutUsed; ++j) s[j] = squash(o[(size_t)r * ld + j], j, vmax);
    bool has = n > 0;
    float loss = 0.f;
    if (has && la.kind == 0) {
      int best = 0;
      float bd = 0.f;
      for (int p = 0; p < n; ++p) {
        float d = 0.f;
        for (int j = 0; j < kOutUsed; ++j) {
          const float u = s[j] - q0[p * kOutUsed + j];
          d += u * u;
        }
        if (p == 0 || d < bd) {
          best = p;
          bd = d;
        }
      }
      for (int j = 0; j < kOutUsed; ++j) y[j] = q0[best * kOutUsed + j];
      loss = bd;
    } else if (has) {
      const float z0 = __bfloat162float(la.x[(size_t)r * la.d0 + la.latent_col]);
      const float u = normcdff(z0);
      int i = 0;
      float f = 0.f;
      if (n > 1) {
        const float a = u * (float)(n - 1);
        i = min((int)floorf(a), n - 2);
        f = a - (float)i;
      }
      for (int j = 0; j < kOutUsed; ++j) {
        const float y0 = q0[i * kOutUsed + j];
        y[j] = n > 1 ? y0 + f * (q0[(i + 1) * kOutUsed + j] - y0) : y0;
        const float d = s[j] - y[j];
        loss += d * d;
      }
    }
    local += loss;
    // the row's gradient: the used columns, then zeros, eight BF16 per 16-byte store (ld is a
    // multiple of 16)
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      float gv[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = j + h;
        gv[h] = 0.f;
        if (has && c < kOutUsed) {
          const float th = tanhf(o[(size_t)r * ld + c]);
          const float ds = (c < 3 ? 0.5f : vmax) * (1.f - th * th);
          gv[h] = 2.f * (s[c] - y[c]) * ds / (float)B;
        }
      }
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(gv[0], gv[1]);
      pk[j / 2] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    uint4* gr = reinterpret_cast<uint4*>(gout + (size_t)r * ld);
    gr[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    for (int q = 1; q < ld / 8; ++q) gr[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  red[threadIdx.x] = local;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  // the last block to finish adds the blocks' sums in block order, records and advances
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    // thread t adds blocks t, t + 256, ... in that order, then a fixed tree over the threads
    __threadfence();
    float v = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kLossThreads) v += ((volatile float*)part)[b];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const float sum = red[0];
      const int64_t idx = ctl[0] - ctl[1];
      if (trace && idx >= 0 && idx < trace_cap) trace[idx] = sum / (float)B;
      ctl[0] += 1;
      *ticket = 0u;
    }
  }
}

// Where each layer's W lives in the flat vector (for the transposed BF16 copy).
constexpr int kMaxLayers = 16;
struct LayerTable {
  int L;
  int64_t offW[kMaxLayers];
  int in[kMaxLayers], out[kMaxLayers];
};

// BF16 copies of parameter k: wb[k], and for a weight W_l[r][c] also wbt[offW_l + c out_l + r]
// (W_l^T, K-major for the input-gradient product).
__device__ __forceinline__ void write_bf16(int64_t k, float wk, bf16* __restrict__ wb, bf16* __restrict__ wbt,
                                           const LayerTable& T) {
  const bf16 q = __float2bfloat16_rn(wk);
  wb[k] = q;
  for (int l = 0; l < T.L; ++l) {
    const int64_t d = k - T.offW[l];
    if (d >= 0 && d < (int64_t)T.in[l] * T.out[l]) {
      const int r = (int)(d / T.in[l]), c = (int)(d - (int64_t)r * T.in[l]);
      wbt[T.offW[l] + (int64_t)c * T.out[l] + r] = q;
      break;
    }
  }
}

__global__ void k_weights_bf16(const float* __restrict__ w, int64_t P, bf16* __restrict__ wb, bf16* __restrict__ wbt,
                               const LayerTable T) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    write_bf16(k, w[k], wb, wbt, T);
}

// Adam over the flat parameter vector (Kingma and Ba, 2015): gradient = sum of the S partials,
// step count t = ctl[0] (already advanced by the loss), then the BF16 copies.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ part, int S, int64_t P, float* __restrict__ m,
                       float* __restrict__ v, const int64_t* __restrict__ ctl, float lr, bf16* __restrict__ wb,
                       bf16* __restrict__ wbt, const LayerTable T) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float t = (float)ctl[0];
  const float c1 = 1.f - powf(b1, t), c2 = 1.f - powf(b2, t);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    float gk = 0.f;
    for (int s = 0; s < S; ++s) gk += part[(int64_t)s * P + k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    w[k] = wk;
    write_bf16(k, wk, wb, wbt, T);
  }
}

int grid_for(int64_t n, int threads, int cap = 1184) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

}  // namespace
}  // namespace pump

using pump::bf16;
using pump::LayerTable;

struct pump_mlp {
  int L = 0;
  std::vector<int> dims;
  std::vector<int64_t> offW, offb;  // offsets of W_l and b_l in the flat vector
  int64_t P = 0;
  float* w = nullptr;      // FP32 master parameters (flat)
  float* m1 = nullptr;     // Adam first moments
  float* m2 = nullptr;     // Adam second moments
  bf16* wb = nullptr;      // BF16 copy of w
  bf16* wbt = nullptr;     // BF16 W_l^T per layer (K-major operand of the input gradient)
  int* tc_err = nullptr;   // a tensor-core block gave up waiting
  int host_err = 0;        // a launch could not be prepared (tensor map)
  LayerTable table{};
  int64_t* ctl = nullptr;  // [0] Adam steps taken, [1] trace base
  float* lpart = nullptr;          // per-block loss sums
  unsigned int* lticket = nullptr; // blocks of the loss kernel finished
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  // scratch for up to `cap` rows
  int cap = 0;
  std::vector<bf16*> act;  // act[l]: layer l input (B x dims[l]), l < L
  bf16* gA = nullptr;      // gradients w.r.t. pre-activations (B x maxd), two buffers
  bf16* gB = nullptr;
  float* out = nullptr;    // last layer's outputs (B x dims[L])
  float* xf = nullptr;     // FP32 staging (B x max(dims[0], dims[L]))
  float* part = nullptr;   // gradient partials (kMaxSplit x P)
  float* gsum = nullptr;   // summed gradient (P)
  int32_t* env = nullptr;  // row -> target set (B)
  float* tg_rows = nullptr;  // per-row targets for pump_mlp_train_step (cap x T x 6)
  int32_t* ntg_rows = nullptr;
  int tg_rows_T = 0;
  std::vector<void*> scratch;
  // training set
  float* feat = nullptr;
  float* tg = nullptr;
  int32_t* ntg = nullptr;
  int F = 0, n_env = 0, T = 0;
  // mean losses of the steps of one call
  float* trace = nullptr;
  int trace_cap = 0;
  // captured training step
  cudaGraphExec_t step_exec = nullptr;
  int step_batch = 0;
  uint64_t step_seed = 0;
  float step_lr = 0.f, step_vmax = 0.f;
  int step_launches = 0;
  // loss
  int loss_kind = 0, latent_col = 0;
};

namespace {

using namespace pump;

template <typename T>
T* dmalloc(size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (T*)p;
}

void drop_graph(pump_mlp* m) {
  if (m->step_exec) cudaGraphExecDestroy(m->step_exec);
  m->step_exec = nullptr;
  m->step_batch = 0;
}

void free_scratch(pump_mlp* m) {
  for (void* p : m->scratch) cudaFree(p);
  m->scratch.clear();
  m->act.clear();
  m->gA = m->gB = nullptr;
  m->out = m->xf = m->part = m->gsum = m->tg_rows = nullptr;
  m->env = m->ntg_rows = nullptr;
  m->tg_rows_T = 0;
  m->cap = 0;
}

int ensure_batch(pump_mlp* m, int B) {
  if (B <= m->cap) return PUMP_OK;
  cudaStreamSynchronize(m->s);
  drop_graph(m);
  free_scratch(m);
  int maxd = 0;
  for (int d : m->dims) maxd = std::max(maxd, d);
  auto take = [&](void* p) {
    if (p) m->scratch.push_back(p);
    return p != nullptr;
  };
  bool ok = true;
  for (int l = 0; l < m->L; ++l) {
    m->act.push_back(dmalloc<bf16>((size_t)B * m->dims[l]));
    ok &= take(m->act.back());
  }
  ok &= take(m->gA = dmalloc<bf16>((size_t)B * maxd));
  ok &= take(m->gB = dmalloc<bf16>((size_t)B * maxd));
  ok &= take(m->out = dmalloc<float>((size_t)B * m->dims[m->L]));
  ok &= take(m->xf = dmalloc<float>((size_t)B * std::max(m->dims[0], m->dims[m->L])));
  ok &= take(m->part = dmalloc<float>((size_t)kMaxSplit * m->P));
  ok &= take(m->gsum = dmalloc<float>((size_t)m->P));
  ok &= take(m->env = dmalloc<int32_t>((size_t)B));
  if (!ok) {
    free_scratch(m);
    return PUMP_ERR_OOM;
  }
  m->cap = B;
  return PUMP_OK;
}

int ensure_trace(pump_mlp* m, int n) {
  if (m->trace_cap >= n && m->trace) return PUMP_OK;
  PUMP_CUDA_TRY(cudaStreamSynchronize(m->s));
  drop_graph(m);
  if (m->trace) cudaFree(m->trace);
  m->trace_cap = std::max(n, 1024);
  m->trace = dmalloc<float>((size_t)m->trace_cap);
  if (!m->trace) {
    m->trace_cap = 0;
    return PUMP_ERR_OOM;
  }
  return PUMP_OK;
}

// Splits of the weight-gradient products over the batch (256 rows or more each, at most
// kMaxSplit), each a multiple of the tensor-core K step: small batches still spread over the SMs.
int n_splits(int B) { return std::max(1, std::min(kMaxSplit, B / 256)); }
int split_chunk(int B, int S) { return ((B + S - 1) / S + kTcK - 1) / kTcK * kTcK; }

void note_err(pump_mlp* m, int rc) {
  if (rc && !m->host_err) m->host_err = rc;
}

// Tensor map of a K-major BF16 operand (rows x K, row stride K): box of 64 K elements (128 B) x
// box_rows rows, written to shared memory in the 128-byte swizzled layout.
int tensor_map(CUtensorMap* map, const bf16* X, int rows, int K, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !encode) {
      encode = nullptr;
      return PUMP_ERR_CUDA;
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)X, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PUMP_OK : PUMP_ERR_CUDA;
}

// Tensor map of an MN-major BF16 operand (K rows x MN, row stride MN): boxes of 64 MN elements
// (128 B) x 64 K rows in the 128-byte swizzled layout.
int tensor_map_mn(CUtensorMap* map, const bf16* X, int MN, int K) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !encode) {
      encode = nullptr;
      return PUMP_ERR_CUDA;
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)MN, (cuuint64_t)K};
  const cuuint64_t strides[1] = {(cuuint64_t)MN * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcMnBox, (cuuint32_t)kTcK};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)X, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PUMP_OK : PUMP_ERR_CUDA;
}

// Weight gradient on the tensor cores: C[M x N] = A^T B summed over K (the batch) in S splits of
// `chunk` rows, A = g (K x M) and B = h (K x N) MN-major; partial z to of + z split_stride (row
// stride ldo) and the column sums of A (the bias gradient) to colsum + z split_stride.  N tile 128.
int gemm_tc_wgrad(pump_mlp* m, const bf16* A, const bf16* B, int M, int N, int K, int S, int chunk, float* of,
                  int ldo, int64_t split_stride, float* colsum, cudaStream_t s, int* launches) {
  constexpr int tileN = 128;
  constexpr int stage = ((kTcM * kTcK * 2 + (tileN + kTcMnBox) * kTcK * 2) + 1023) & ~1023;
  constexpr int smem = kTcStages * stage + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<kEpiPartial, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  CUtensorMap ta, tb;
  int rc = tensor_map_mn(&ta, A, M, K);
  if (!rc) rc = tensor_map_mn(&tb, B, N, K);
  if (rc) return rc;
  int cols = 32;
  while (cols < tileN + kTcOnes) cols <<= 1;
  TcArgs a{M, N, K, tileN, cols, nullptr, nullptr, nullptr, of, ldo, m->tc_err, chunk, split_stride, colsum};
  k_gemm_tc<kEpiPartial, true><<<dim3((N + tileN - 1) / tileN, (M + kTcM - 1) / kTcM, S), kTcThreads, smem, s>>>(
      ta, tb, a);
  ++*launches;
  return PUMP_OK;
}

// Tensor-core GEMM (K-major A and B): N tile 256, 128 or 64, the widest that still gives about one
// block per SM.
template <int kEpi>
int gemm_tc(pump_mlp* m, const bf16* A, const bf16* B, int M, int N, int K, const float* bias, const bf16* mask,
            bf16* ob, float* of, int ldo, cudaStream_t s, int* launches) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<kEpi, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    cudaFuncSetAttribute(k_gemm_tc<kEpi, false, kTcStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    attr = true;
  }
  const int mt = (M + kTcM - 1) / kTcM, sms = num_sms();
  int tileN = kTcNMax;
  while (tileN > 64 && (long long)mt * ((N + tileN - 1) / tileN) < sms) tileN >>= 1;
  tileN = std::min(tileN, N);
  CUtensorMap ta, tb;
  int rc = tensor_map(&ta, A, M, K, kTcM);
  if (!rc) rc = tensor_map(&tb, B, N, K, tileN);
  if (rc) return rc;
  int cols = 32;
  while (cols < tileN) cols <<= 1;
  const int stage = ((kTcM + tileN) * kTcK * 2 + 1023) & ~1023;
  TcArgs a{M, N, K, tileN, cols, bias, mask, ob, of, ldo, m->tc_err, 0, 0, nullptr};
  // a short K (at most 8 steps) needs two buffers: then two blocks share an SM, one's epilogue
  // beside the other's copies and products
  if (K <= 8 * kTcK)
    k_gemm_tc<kEpi, false, 2><<<dim3((N + tileN - 1) / tileN, mt), kTcThreads, 2 * stage + 1024, s>>>(ta, tb, a);
  else
    k_gemm_tc<kEpi, false, kTcStages><<<dim3((N + tileN - 1) / tileN, mt), kTcThreads, kTcStages * stage + 1024, s>>>(
        ta, tb, a);
  ++*launches;
  return PUMP_OK;
}

// Forward pass over B rows of act[0]; outputs (FP32) in m->out.
void forward(pump_mlp* m, int B, cudaStream_t s, int* launches) {
  for (int l = 0; l < m->L; ++l) {
    GemmArgs a{};
    a.A = m->act[l];
    a.lda = m->dims[l];
    a.B = m->wb + m->offW[l];
    a.ldb = m->dims[l];
    a.M = B;
    a.N = m->dims[l + 1];
    a.K = m->dims[l];
    a.kchunk = a.K;
    a.bias = m->w + m->offb[l];
    a.ldo = a.N;
    if (l + 1 < m->L)
      note_err(m, gemm_tc<kEpiBiasRelu>(m, a.A, a.B, B, a.N, a.K, a.bias, nullptr, m->act[l + 1], nullptr, a.N, s,
                                        launches));
    else
      note_err(m, gemm_tc<kEpiBias>(m, a.A, a.B, B, a.N, a.K, a.bias, nullptr, nullptr, m->out, a.N, s, launches));
  }
}

// Backward pass from g = m->gA (B x dims[L], BF16); gradient partials into m->part.
void backward(pump_mlp* m, int B, cudaStream_t s, int* launches) {
  const int S = n_splits(B), chunk = split_chunk(B, S);
  bf16* g = m->gA;
  bf16* gn = m->gB;
  for (int l = m->L - 1; l >= 0; --l) {
    const int in = m->dims[l], out = m->dims[l + 1];
    // dW_l = g^T h_l and db_l = column sums of g, on the tensor cores (MN-major operands)
    note_err(m, gemm_tc_wgrad(m, g, m->act[l], out, in, B, S, chunk, m->part + m->offW[l], in, m->P,
                              m->part + m->offb[l], s, launches));
    if (l > 0) {
      // g_{l-1} = (g W_l) * [h_l > 0]: B operand W_l^T (in x out, K-major)
      note_err(m, gemm_tc<kEpiMask>(m, g, m->wbt + m->offW[l], B, in, out, nullptr, m->act[l], gn, nullptr, in, s,
                                    launches));
      std::swap(g, gn);
    }
  }
}

void adam(pump_mlp* m, int B, float lr, cudaStream_t s, int* launches) {
  k_adam<<<grid_for(m->P, 256), 256, 0, s>>>(m->w, m->part, n_splits(B), m->P, m->m1, m->m2, m->ctl, lr, m->wb,
                                             m->wbt, m->table);
  ++*launches;
}

// Inputs (FP32, host or device, B x dims[0]) -> act[0].
int stage_input(pump_mlp* m, const float* x, int B, int* launches) {
  const size_t n = (size_t)B * m->dims[0];
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->xf, x, sizeof(float) * n, cudaMemcpyDefault, m->s));
  k_to_bf16<<<grid_for((int64_t)n, 256), 256, 0, m->s>>>(m->xf, (int64_t)n, m->act[0]);
  ++*launches;
  return PUMP_OK;
}

int loss_blocks(int B) { return std::max(1, std::min(kLossBlocksMax, (B + kLossThreads - 1) / kLossThreads)); }

LossArgs loss_args(const pump_mlp* m) {
  LossArgs a{};
  a.kind = m->loss_kind;
  a.x = m->act[0];
  a.d0 = m->dims[0];
  a.latent_col = m->latent_col;
  return a;
}

// One training step on the stored training set (graph-capturable): draws, forward, loss,
// backward, Adam.
void train_step_kernels(pump_mlp* m, int B, uint64_t seed, float lr, float vmax, cudaStream_t s, int* launches) {
  k_assemble<<<(B + 15) / 16, 128, 0, s>>>(m->feat, m->F, m->n_env, m->dims[0], B, seed, 0ull, m->ctl, m->act[0],
                                           m->env);
  ++*launches;
  forward(m, B, s, launches);
  k_loss<<<loss_blocks(B), kLossThreads, 0, s>>>(m->out, B, m->dims[m->L], vmax, m->tg, m->ntg, m->T, m->env,
                                                  loss_args(m), m->gA, m->ctl, m->trace, m->trace_cap, m->lpart,
                                                  m->lticket);
  ++*launches;
  backward(m, B, s, launches);
  adam(m, B, lr, s, launches);
}

void count_launches(int64_t n) {
  for (int64_t k = 0; k < n; ++k) note_launch();
}

// Order the library's stream after the caller's.
int enter(pump_mlp* m, void* stream) {
  PUMP_CUDA_TRY(cudaEventRecord(m->ev, (cudaStream_t)stream));
  PUMP_CUDA_TRY(cudaStreamWaitEvent(m->s, m->ev, 0));
  return PUMP_OK;
}

int finish(pump_mlp* m) {
  PUMP_CUDA_TRY(cudaStreamSynchronize(m->s));
  PUMP_CUDA_TRY(cudaGetLastError());
  if (m->host_err) {
    const int rc = m->host_err;
    m->host_err = 0;
    return rc;
  }
  int e = 0;
  PUMP_CUDA_TRY(cudaMemcpy(&e, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    cudaMemset(m->tc_err, 0, sizeof(int));
    return PUMP_ERR_TIMEOUT;
  }
  return PUMP_OK;
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int pump_mlp_create(int32_t n_layers, const int32_t* dims, uint64_t seed, pump_mlp** out) {
  if (!out || !dims || n_layers < 1 || n_layers > 16) return PUMP_ERR_INVALID_ARG;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] < 16 || dims[l] > 4096 || dims[l] % 16) return PUMP_ERR_INVALID_ARG;
  pump_mlp* m = new (std::nothrow) pump_mlp();
  if (!m) return PUMP_ERR_OOM;
  m->L = n_layers;
  m->dims.assign(dims, dims + n_layers + 1);
  for (int l = 0; l < n_layers; ++l) {
    m->offW.push_back(m->P);
    m->P += (int64_t)dims[l] * dims[l + 1];
    m->offb.push_back(m->P);
    m->P += dims[l + 1];
  }
  m->w = dmalloc<float>(m->P);
  m->m1 = dmalloc<float>(m->P);
  m->m2 = dmalloc<float>(m->P);
  m->wb = dmalloc<bf16>(m->P);
  m->ctl = dmalloc<int64_t>(2);
  m->wbt = dmalloc<bf16>(m->P);
  m->tc_err = dmalloc<int>(1);
  if (m->tc_err) cudaMemset(m->tc_err, 0, sizeof(int));
  m->table.L = n_layers;
  for (int l = 0; l < n_layers; ++l) {
    m->table.offW[l] = m->offW[l];
    m->table.in[l] = dims[l];
    m->table.out[l] = dims[l + 1];
  }
  m->lpart = dmalloc<float>(kLossBlocksMax);
  m->lticket = dmalloc<unsigned int>(1);
  if (m->lticket) cudaMemset(m->lticket, 0, sizeof(unsigned int));
  if (!m->w || !m->m1 || !m->m2 || !m->wb || !m->wbt || !m->tc_err || !m->ctl || !m->lpart || !m->lticket ||
      cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming) != cudaSuccess) {
    pump_mlp_destroy(m);
    return PUMP_ERR_OOM;
  }
  // He-uniform weights from a seeded splitmix64 stream, zero biases
  std::vector<float> h((size_t)m->P, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < n_layers; ++l) {
    const double lim = std::sqrt(6.0 / (double)dims[l]);
    for (int64_t k = 0; k < (int64_t)dims[l] * dims[l + 1]; ++k)
      h[m->offW[l] + k] = (float)((((double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * lim);
  }
  const int rc = pump_mlp_set_params(m, h.data(), m->P);
  if (rc) {
    pump_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return PUMP_OK;
}

int64_t pump_mlp_param_count(const pump_mlp* m) { return m ? m->P : -1; }

int pump_mlp_set_params(pump_mlp* m, const float* params, int64_t count) {
  if (!m || !params || count != m->P) return PUMP_ERR_INVALID_ARG;
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->w, params, sizeof(float) * m->P, cudaMemcpyDefault, m->s));
  PUMP_CUDA_TRY(cudaMemsetAsync(m->m1, 0, sizeof(float) * m->P, m->s));
  PUMP_CUDA_TRY(cudaMemsetAsync(m->m2, 0, sizeof(float) * m->P, m->s));
  PUMP_CUDA_TRY(cudaMemsetAsync(m->ctl, 0, sizeof(int64_t) * 2, m->s));
  k_weights_bf16<<<grid_for(m->P, 256), 256, 0, m->s>>>(m->w, m->P, m->wb, m->wbt, m->table);
  count_launches(1);
  return finish(m);
}

int pump_mlp_get_params(pump_mlp* m, float* params, int64_t count, int64_t* steps) {
  if (!m || !params || count != m->P) return PUMP_ERR_INVALID_ARG;
  PUMP_CUDA_TRY(cudaMemcpyAsync(params, m->w, sizeof(float) * m->P, cudaMemcpyDefault, m->s));
  int64_t ctl[2] = {0, 0};
  PUMP_CUDA_TRY(cudaMemcpyAsync(ctl, m->ctl, sizeof(ctl), cudaMemcpyDeviceToHost, m->s));
  const int rc = finish(m);
  if (!rc && steps) *steps = ctl[0];
  return rc;
}

int pump_mlp_forward(pump_mlp* m, const float* x, int32_t B, float* y, void* stream) {
  if (!m || !x || !y || B < 1) return PUMP_ERR_INVALID_ARG;
  int rc = ensure_batch(m, B);
  if (!rc) rc = enter(m, stream);
  int n = 0;
  if (!rc) rc = stage_input(m, x, B, &n);
  if (rc) return rc;
  forward(m, B, m->s, &n);
  count_launches(n);
  PUMP_CUDA_TRY(cudaMemcpyAsync(y, m->out, sizeof(float) * (size_t)B * m->dims[m->L], cudaMemcpyDefault, m->s));
  return finish(m);
}

int pump_mlp_gradients(pump_mlp* m, const float* x, int32_t B, const float* dy, float* grads, int64_t count,
                       void* stream) {
  if (!m || !x || !dy || !grads || B < 1 || count != m->P) return PUMP_ERR_INVALID_ARG;
  int rc = ensure_batch(m, B);
  if (!rc) rc = enter(m, stream);
  int n = 0;
  if (!rc) rc = stage_input(m, x, B, &n);
  if (rc) return rc;
  forward(m, B, m->s, &n);
  const size_t no = (size_t)B * m->dims[m->L];
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->xf, dy, sizeof(float) * no, cudaMemcpyDefault, m->s));
  k_to_bf16<<<grid_for((int64_t)no, 256), 256, 0, m->s>>>(m->xf, (int64_t)no, m->gA);
  ++n;
  backward(m, B, m->s, &n);
  k_sum_parts<<<grid_for(m->P, 256), 256, 0, m->s>>>(m->part, n_splits(B), m->P, m->gsum);
  ++n;
  count_launches(n);
  PUMP_CUDA_TRY(cudaMemcpyAsync(grads, m->gsum, sizeof(float) * m->P, cudaMemcpyDefault, m->s));
  return finish(m);
}

int pump_mlp_train_step(pump_mlp* m, const float* x, int32_t B, const float* targets, const int32_t* n_targets,
                        int32_t T, float lr, float vmax, float* mean_loss, void* stream) {
  if (!m || !x || !targets || !n_targets || B < 1 || T < 1 || !(lr > 0.f) || !(vmax > 0.f))
    return PUMP_ERR_INVALID_ARG;
  int rc = ensure_batch(m, B);
  if (!rc) rc = ensure_trace(m, 1);
  if (rc) return rc;
  if (m->tg_rows_T != T || !m->tg_rows) {
    PUMP_CUDA_TRY(cudaStreamSynchronize(m->s));
    for (void* p : {(void*)m->tg_rows, (void*)m->ntg_rows}) {
      auto it = std::find(m->scratch.begin(), m->scratch.end(), p);
      if (p && it != m->scratch.end()) {
        cudaFree(p);
        m->scratch.erase(it);
      }
    }
    m->tg_rows = dmalloc<float>((size_t)m->cap * T * kOutUsed);
    m->ntg_rows = dmalloc<int32_t>((size_t)m->cap);
    if (m->tg_rows) m->scratch.push_back(m->tg_rows);
    if (m->ntg_rows) m->scratch.push_back(m->ntg_rows);
    if (!m->tg_rows || !m->ntg_rows) {
      m->tg_rows_T = 0;
      return PUMP_ERR_OOM;
    }
    m->tg_rows_T = T;
  }
  rc = enter(m, stream);
  int n = 0;
  if (!rc) rc = stage_input(m, x, B, &n);
  if (rc) return rc;
  PUMP_CUDA_TRY(
      cudaMemcpyAsync(m->tg_rows, targets, sizeof(float) * (size_t)B * T * kOutUsed, cudaMemcpyDefault, m->s));
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->ntg_rows, n_targets, sizeof(int32_t) * B, cudaMemcpyDefault, m->s));
  // the step's mean loss goes to trace[0]: base = the current step count
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->ctl + 1, m->ctl, sizeof(int64_t), cudaMemcpyDeviceToDevice, m->s));
  forward(m, B, m->s, &n);
  k_loss<<<loss_blocks(B), kLossThreads, 0, m->s>>>(m->out, B, m->dims[m->L], vmax, m->tg_rows, m->ntg_rows, T,
                                                     nullptr, loss_args(m), m->gA, m->ctl, m->trace, m->trace_cap,
                                                     m->lpart, m->lticket);
  ++n;
  backward(m, B, m->s, &n);
  adam(m, B, lr, m->s, &n);
  count_launches(n);
  float l = 0.f;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&l, m->trace, sizeof(float), cudaMemcpyDeviceToHost, m->s));
  rc = finish(m);
  if (!rc && mean_loss) *mean_loss = l;
  return rc;
}

int pump_mlp_set_loss(pump_mlp* m, int32_t kind, int32_t latent_col) {
  if (!m || kind < 0 || kind > 1 || latent_col < 0 || latent_col >= m->dims[0]) return PUMP_ERR_INVALID_ARG;
  PUMP_CUDA_TRY(cudaStreamSynchronize(m->s));
  drop_graph(m);
  m->loss_kind = kind;
  m->latent_col = latent_col;
  return PUMP_OK;
}

int pump_mlp_set_data(pump_mlp* m, const float* feat, int32_t F, int32_t n_env, const float* targets,
                      const int32_t* n_targets, int32_t T) {
  if (!m || (!feat && F > 0) || !targets || !n_targets || n_env < 1 || T < 1 || F < 0 || F + kLatent > m->dims[0])
    return PUMP_ERR_INVALID_ARG;
  PUMP_CUDA_TRY(cudaStreamSynchronize(m->s));
  drop_graph(m);
  for (void* p : {(void*)m->feat, (void*)m->tg, (void*)m->ntg})
    if (p) cudaFree(p);
  m->feat = dmalloc<float>((size_t)n_env * std::max(F, 1));
  m->tg = dmalloc<float>((size_t)n_env * T * kOutUsed);
  m->ntg = dmalloc<int32_t>((size_t)n_env);
  if (!m->feat || !m->tg || !m->ntg) {
    for (void* p : {(void*)m->feat, (void*)m->tg, (void*)m->ntg})
      if (p) cudaFree(p);
    m->feat = m->tg = nullptr;
    m->ntg = nullptr;
    m->n_env = 0;
    return PUMP_ERR_OOM;
  }
  m->F = F;
  m->n_env = n_env;
  m->T = T;
  if (F > 0)
    PUMP_CUDA_TRY(cudaMemcpyAsync(m->feat, feat, sizeof(float) * (size_t)n_env * F, cudaMemcpyDefault, m->s));
  PUMP_CUDA_TRY(
      cudaMemcpyAsync(m->tg, targets, sizeof(float) * (size_t)n_env * T * kOutUsed, cudaMemcpyDefault, m->s));
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->ntg, n_targets, sizeof(int32_t) * n_env, cudaMemcpyDefault, m->s));
  return finish(m);
}

int pump_mlp_assemble(pump_mlp* m, int32_t B, int64_t t, uint64_t seed, float* x, int32_t* env) {
  if (!m || !x || B < 1 || t < 0 || !m->feat) return PUMP_ERR_INVALID_ARG;
  int rc = ensure_batch(m, B);
  if (rc) return rc;
  int64_t saved[2] = {0, 0};
  PUMP_CUDA_TRY(cudaMemcpyAsync(saved, m->ctl, sizeof(saved), cudaMemcpyDeviceToHost, m->s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(m->s));
  const int64_t tmp[2] = {t, saved[1]};
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->ctl, tmp, sizeof(tmp), cudaMemcpyHostToDevice, m->s));
  k_assemble<<<(B + 15) / 16, 128, 0, m->s>>>(m->feat, m->F, m->n_env, m->dims[0], B, seed, 0ull, m->ctl, m->act[0],
                                              m->env);
  const size_t n = (size_t)B * m->dims[0];
  k_bf16_to_f32<<<grid_for((int64_t)n, 256), 256, 0, m->s>>>(m->act[0], (int64_t)n, m->xf);
  count_launches(2);
  PUMP_CUDA_TRY(cudaMemcpyAsync(x, m->xf, sizeof(float) * n, cudaMemcpyDefault, m->s));
  if (env) PUMP_CUDA_TRY(cudaMemcpyAsync(env, m->env, sizeof(int32_t) * B, cudaMemcpyDefault, m->s));
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->ctl, saved, sizeof(saved), cudaMemcpyHostToDevice, m->s));
  return finish(m);
}

int pump_mlp_train(pump_mlp* m, int32_t B, int32_t steps, float lr, float vmax, uint64_t seed, float* loss_trace,
                   void* stream) {
  if (!m || B < 1 || steps < 0 || !(lr > 0.f) || !(vmax > 0.f) || !m->feat) return PUMP_ERR_INVALID_ARG;
  int rc = ensure_batch(m, B);
  if (!rc) rc = ensure_trace(m, steps);
  if (!rc) rc = enter(m, stream);
  if (rc) return rc;
  // losses of this call go to trace[0 .. steps): base = the current step count
  PUMP_CUDA_TRY(cudaMemcpyAsync(m->ctl + 1, m->ctl, sizeof(int64_t), cudaMemcpyDeviceToDevice, m->s));
  if (m->step_exec && (m->step_batch != B || m->step_seed != seed || m->step_lr != lr || m->step_vmax != vmax))
    drop_graph(m);
  if (!m->step_exec && steps > 0) {
    cudaGraph_t graph = nullptr;
    int n = 0;
    PUMP_CUDA_TRY(cudaStreamBeginCapture(m->s, cudaStreamCaptureModeThreadLocal));
    train_step_kernels(m, B, seed, lr, vmax, m->s, &n);
    const cudaError_t ce = cudaStreamEndCapture(m->s, &graph);
    if (ce != cudaSuccess || !graph) {
      cudaGetLastError();
      return PUMP_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&m->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      m->step_exec = nullptr;
      return PUMP_ERR_CUDA;
    }
    m->step_batch = B;
    m->step_seed = seed;
    m->step_lr = lr;
    m->step_vmax = vmax;
    m->step_launches = n;
  }
  for (int k = 0; k < steps; ++k) PUMP_CUDA_TRY(cudaGraphLaunch(m->step_exec, m->s));
  count_launches((int64_t)m->step_launches * steps);
  if (loss_trace && steps > 0)
    PUMP_CUDA_TRY(cudaMemcpyAsync(loss_trace, m->trace, sizeof(float) * steps, cudaMemcpyDefault, m->s));
  return finish(m);
}

int pump_mlp_propose(pump_mlp* m, const float* feat, int32_t F, int32_t count, uint64_t seed, float vmax,
                     float* states, void* stream) {
  if (!m || (!feat && F > 0) || !states || count < 1 || F < 0 || F + kLatent > m->dims[0] || !(vmax > 0.f))
    return PUMP_ERR_INVALID_ARG;
  const int B = (count + 15) / 16 * 16;
  int rc = ensure_batch(m, B);
  if (!rc) rc = enter(m, stream);
  if (rc) return rc;
  if (F > 0) PUMP_CUDA_TRY(cudaMemcpyAsync(m->xf, feat, sizeof(float) * F, cudaMemcpyDefault, m->s));
  int n = 0;
  k_assemble<<<B / 16, 128, 0, m->s>>>(m->xf, F, 0, m->dims[0], B, seed, 2ull, nullptr, m->act[0], nullptr);
  ++n;
  forward(m, B, m->s, &n);
  k_squash<<<(count * kOutUsed + 255) / 256, 256, 0, m->s>>>(m->out, count, m->dims[m->L], vmax, m->xf);
  ++n;
  count_launches(n);
  PUMP_CUDA_TRY(cudaMemcpyAsync(states, m->xf, sizeof(float) * (size_t)count * kOutUsed, cudaMemcpyDefault, m->s));
  return finish(m);
}

void pump_mlp_destroy(pump_mlp* m) {
  if (!m) return;
  if (m->s) cudaStreamSynchronize(m->s);
  drop_graph(m);
  free_scratch(m);
  for (void* p : {(void*)m->w, (void*)m->m1, (void*)m->m2, (void*)m->wb, (void*)m->ctl, (void*)m->feat, (void*)m->tg,
                  (void*)m->ntg, (void*)m->trace, (void*)m->lpart, (void*)m->lticket, (void*)m->wbt,
                  (void*)m->tc_err})
    if (p) cudaFree(p);
  if (m->ev) cudaEventDestroy(m->ev);
  if (m->s) cudaStreamDestroy(m->s);
  delete m;
}

}  // extern "C"
