// Learned-start inference on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The warm-start network's two hidden layers for 128-row tiles in one
// persistent CTA of eight warps: the weights of both layers stay in shared
// memory for the whole launch (W1: 64 x 256, W2: 256 x 256, BF16), each
// 128 x 64 input tile is staged with cp.async (zero-fill past the last row),
// and one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// N = 256) into 256 TMEM columns, committed to an mbarrier.  The first MMA's
// epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32 (w mod 4) .. +31, the tile's rows, and columns 128 (w div 4) .. +127) and
// writes relu(acc + b1) as BF16 straight into shared memory in the operand
// layout of the second MMA (over the input tile, which the first MMA has
// consumed); the second MMA's epilogue folds the output layer in,
// out = sum_c bf16(relu(acc_c + b2_c)) w3_c + b3 (the two column halves added
// through shared memory).  The hidden activations never leave the SM.
//
// Operand layout in shared memory: K-major, no swizzle, 8 x 16-byte core
// matrices; core matrix (r8, k8) of an R-row operand sits at byte
// (k8 * R/8 + r8) * 128, so the descriptor's stride between row groups (SBO)
// is 128 B and between K groups (LBO) is 16 R bytes.  Every wait on the
// mbarrier is bounded; a timeout sets *err and the CTA stops, releasing its
// TMEM.
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "rlt2_internal.h"

namespace rlt2 {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kN = 256;          // layer width (TMEM columns)
constexpr int kRowsPerTile = 128;  // M of the MMA = TMEM lanes
constexpr int kThreads = 256;
constexpr long long kWaitLimit = 1ll << 22;  // non-blocking mbarrier polls before giving up (~0.1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4
// (16-29), SBO >> 4 (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// (7-9 = 1) and B (10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22),
// M >> 4 (24-28).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRowsPerTile >> 4) << 24);

__device__ __forceinline__ uint32_t core_off(int r, int k8, int R) {
  return (uint32_t)((k8 * (R / 8) + (r >> 3)) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Both hidden layers of the network for 128-row tiles in one persistent CTA:
// the weights of both layers stay in shared memory (W1: 64 x 256, W2: 256 x
// 256, 160 KB), the 128 x 64 input tile is staged with cp.async, the first
// MMA's epilogue writes relu(acc + b1) as BF16 straight into shared memory in
// the K-major operand layout of the second MMA (over the input tile, which the
// first MMA has consumed), and the second MMA's epilogue folds the output
// layer in.  The hidden activations never leave the SM.
struct UmmaMlpArgs {
  long long rows;
  const bf16* X;  // [rows][64]
  const bf16* W1;  // [64][256]
  const float* b1;
  const bf16* W2;  // [256][256]
  const float* b2;
  const float* w3;
  const float* b3;
  float* out;
  int* err;
  int withhold_commit;  // diagnostics: issue no MMA and no commit, so the first wait runs out
};

__device__ __forceinline__ void load_weights(unsigned char* Bs, const bf16* W, int K, int tid) {
  for (int e = tid; e < K * kN / 8; e += kThreads) {
    const int k = e / (kN / 8), n8 = e - k * (kN / 8);
    const uint4 v = *reinterpret_cast<const uint4*>(W + (size_t)k * kN + n8 * 8);
    const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<bf16*>(Bs + core_off(n8 * 8 + q, k >> 3, kN) + (k & 7) * 2) = h[q];
  }
}

__device__ __forceinline__ void issue_mma(uint32_t tmem, uint32_t a_base, uint32_t b_base, int K, uint32_t bar) {
#pragma unroll 1
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = sdesc(a_base + kk * 2 * (16 * kRowsPerTile), 16 * kRowsPerTile, 128);
    const uint64_t bd = sdesc(b_base + kk * 2 * (16 * kN), 16 * kN, 128);
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(kk)
        : "memory");
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_umma_mlp(UmmaMlpArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* B1 = smem;                       // 256 x 64
  unsigned char* B2 = B1 + (size_t)kN * 64 * 2;   // 256 x 256
  unsigned char* Act = B2 + (size_t)kN * kN * 2;  // input tile (128 x 64), then hidden tile (128 x 256)
  float* half = reinterpret_cast<float*>(Act + (size_t)kRowsPerTile * kN * 2);
  uint64_t* bar = reinterpret_cast<uint64_t*>(half + kRowsPerTile);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_a = smem_u32(bar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(kN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
  load_weights(B1, a.W1, 64, tid);
  load_weights(B2, a.W2, kN, tid);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  const uint32_t act = smem_u32(Act), b1a = smem_u32(B1), b2a = smem_u32(B2);
  const int quarter = warp & 3, colh = warp >> 2;
  const int trow = quarter * 32 + lane;
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (a.rows + kRowsPerTile - 1) / kRowsPerTile;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long r0 = tile * kRowsPerTile;
    const long long row = r0 + trow;
    for (int c = tid; c < kRowsPerTile * 8; c += kThreads) {
      const int r = c >> 3, k8 = c & 7;
      const bool in = r0 + r < a.rows;
      const bf16* src = a.X + (in ? (r0 + r) * 64 + k8 * 8 : 0);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(act + core_off(r, k8, kRowsPerTile)),
                   "l"(src), "r"(in ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && !a.withhold_commit) issue_mma(tmem, act, b1a, 64, bar_a);
    bool arrived = mbar_wait(bar_a, phase);
    if (__syncthreads_or(arrived ? 0 : 1)) {
      if (tid == 0) atomicExch(a.err, 1);
      ok = false;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // hidden layer 1 -> BF16 operand of the second MMA, in shared memory
#pragma unroll 1
    for (int c0 = colh * (kN / 2); c0 < (colh + 1) * (kN / 2); c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + (uint32_t)c0, v);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + 8 * g + 2 * j;
          const bf16 lo = __float2bfloat16_rn(fmaxf(__uint_as_float(v[8 * g + 2 * j]) + a.b1[c], 0.0f));
          const bf16 hi = __float2bfloat16_rn(fmaxf(__uint_as_float(v[8 * g + 2 * j + 1]) + a.b1[c + 1], 0.0f));
          p[j] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        *reinterpret_cast<uint4*>(Act + core_off(trow, (c0 >> 3) + g, kRowsPerTile)) = make_uint4(p[0], p[1], p[2], p[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) issue_mma(tmem, act, b2a, kN, bar_a);
    arrived = mbar_wait(bar_a, phase);
    if (__syncthreads_or(arrived ? 0 : 1)) {
      if (tid == 0) atomicExch(a.err, 1);
      ok = false;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float acc_out = 0.0f;
#pragma unroll 1
    for (int c0 = colh * (kN / 2); c0 < (colh + 1) * (kN / 2); c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float h = fmaxf(__uint_as_float(v[j]) + a.b2[c0 + j], 0.0f);
        acc_out = fmaf(__bfloat162float(__float2bfloat16_rn(h)), a.w3[c0 + j], acc_out);
      }
    }
    if (colh == 1) half[trow] = acc_out;
    __syncthreads();
    if (colh == 0 && row < a.rows) a.out[row] = (acc_out + half[trow]) + *a.b3;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok && !a.withhold_commit) mbar_wait(bar_a, phase);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN) : "memory");
}

constexpr size_t kMlpSmem = (size_t)kN * 64 * 2 + (size_t)kN * kN * 2 + (size_t)kRowsPerTile * kN * 2 +
                            kRowsPerTile * 4 + 64;

}  // namespace

// out[r] = w3 . relu(W2^T relu(W1^T x_r + b1) + b2) + b3 for `rows` feature rows
// (X: [rows][64] BF16); err: device flag set on a timed-out wait.
cudaError_t umma_mlp_forward(const bf16* X, long long rows, const bf16* W1, const float* b1, const bf16* W2,
                             const float* b2, const float* w3, const float* b3, float* out, int* err,
                             cudaStream_t s, bool withhold_commit) {
  if (rows <= 0) return cudaSuccess;
  // launch configuration, once per device, from any host thread (not valid
  // across a cudaDeviceReset, like every per-device cache of the library)
  static std::mutex mu;
  constexpr int kDevs = 64;
  static int sms_of[kDevs];
  static bool attr_of[kDevs];
  cudaError_t e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!sms_of[dev] &&
        (e = cudaDeviceGetAttribute(&sms_of[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    if (!attr_of[dev]) {
      if ((e = cudaFuncSetAttribute(k_umma_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem)) !=
          cudaSuccess)
        return e;
      attr_of[dev] = true;
    }
    sms = sms_of[dev];
  }
  const long long tiles = (rows + kRowsPerTile - 1) / kRowsPerTile;
  const int grid = (int)(tiles < sms ? tiles : sms);
  UmmaMlpArgs a{rows, X, W1, b1, W2, b2, w3, b3, out, err, withhold_commit ? 1 : 0};
  k_umma_mlp<<<grid, kThreads, kMlpSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rlt2
