// Training GEMMs of the learned warm start on the 5th-generation tensor cores
// (tcgen05, sm_103a): C = A B with BF16 operands and FP32 accumulation in
// TMEM, for the forward layers and the backward products of the network
// (34 -> H -> H -> 1, H <= 256).
//
// One CTA of eight warps computes a 128-row block of C over a block of at most
// 128 columns (grid.x; one TMEM accumulator of FP32 columns) and a K range
// (grid.z splits K for the weight gradients, whose K is the batch).  K
// advances in chunks of 64 through a ring of three shared-memory slots: the
// copies of chunks k + 1 and k + 2 are in flight (cp.async) while chunk k is
// multiplied (tcgen05.mma by one thread, committed to the slot's mbarrier; a
// slot is refilled once the MMAs that read it are done).  The MMA reads both
// operands K-major (8 x 16-byte core matrices, as in umma.cu), whatever their
// layout in global memory:
//   K-contiguous operand (rows of K): 16-byte cp.async per core-matrix row;
//   MN-contiguous operand (rows of MN): copied as it lies (padded rows), then
//     transposed in shared memory, 8 x 8 blocks read by ldmatrix and written
//     back transposed by stmatrix.trans.
// Rows past M (or N) are zero-filled and their results not stored.  Every wait
// on an mbarrier is bounded; a timeout sets *err and the CTA stops after its
// in-flight MMAs, releasing its TMEM.
//
// Epilogues (per element, as the mma.sync GEMM of mlp.cu computes them):
// 0: FP32 store (atomic add when K is split);
// 1: bias + ReLU, rounded to BF16;  2: masked by mask > 0, rounded to BF16.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "rlt2_internal.h"
#include "rlt2_mlp_gemm.h"

namespace rlt2 {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kBM = 128;      // rows per CTA = TMEM lanes = MMA M
constexpr int kBK = 64;       // K per stage
constexpr int kMaxN = 256;    // columns of C
constexpr int kBN = 128;      // columns per CTA (MMA N, TMEM columns)
constexpr int kThreads = 256;
constexpr long long kWaitLimit = 1ll << 22;  // non-blocking mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row r, K group k8) in a K-major operand of R rows (R/8 row groups)
__device__ __forceinline__ uint32_t core_off(int r, int k8, int R) {
  return (uint32_t)((k8 * (R / 8) + (r >> 3)) * 128 + (r & 7) * 16);
}

// shared-memory matrix descriptor: start, LBO (K-adjacent core matrices), SBO
// (row-group-adjacent core matrices), version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3, M >> 4
__device__ __forceinline__ uint32_t idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
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

// Row stride (elements) of a raw MN-contiguous tile in shared memory: 8
// elements of padding put the eight 16-byte rows an ldmatrix reads in
// different banks.
constexpr int kRawPad = 8;

// Copies rows [r0, r0 + R) x K [k0, k0 + 64) of a K-contiguous operand (element
// (r, k) at g[r * ld + k]) into the K-major layout at `dst` by cp.async;
// rows >= rmax are zero-filled (R a multiple of 16).  A warp's lanes take 16
// consecutive rows at two adjacent K groups: each half-warp writes 16
// consecutive core-matrix rows (256 contiguous bytes, no bank conflict) and
// each row's two 16-byte pieces are one 32-byte sector of global memory.
__device__ __forceinline__ void load_kmajor(unsigned char* dst, int R, const bf16* g, int ld, int r0, int rmax,
                                            int k0, int tid) {
  const int rg = R / 16;
  for (int c = tid; c < R * 8; c += kThreads) {
    const int rest = c >> 5;
    const int r = (rest % rg) * 16 + (c & 15), k8 = 2 * (rest / rg) + ((c >> 4) & 1);
    const bool in = r0 + r < rmax;
    const bf16* src = g + (in ? (size_t)(r0 + r) * ld + k0 + k8 * 8 : 0);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst) + core_off(r, k8, R)),
                 "l"(src), "r"(in ? 16 : 0)
                 : "memory");
  }
}

// Copies the 64 x R tile of an MN-contiguous operand (element (r, k) at
// g[k * ld + r]; rows k0 .. k0 + 63, columns r0 .. r0 + R - 1) as it is laid
// out in memory into `raw` (row stride R + kRawPad) by cp.async; columns >= rmax
// are zero-filled (rmax - r0 a multiple of 8).
__device__ __forceinline__ void load_raw(unsigned char* raw, int R, const bf16* g, int ld, int r0, int rmax,
                                         int k0, int tid) {
  const int per = R / 8;
  for (int c = tid; c < 64 * per; c += kThreads) {
    const int k = c / per, r8 = c - k * per;
    const bool in = r0 + r8 * 8 < rmax;
    const bf16* src = g + (in ? (size_t)(k0 + k) * ld + r0 + r8 * 8 : 0);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(raw) +
                                                                      (uint32_t)((k * (R + kRawPad) + r8 * 8) * 2)),
                 "l"(src), "r"(in ? 16 : 0)
                 : "memory");
  }
}

// raw (64 k x R mn, row stride R + kRawPad) -> the K-major layout at dst: each
// 8 x 8 block is read by ldmatrix (rows = k) and written transposed by
// stmatrix.trans (rows = mn, the core-matrix rows); four blocks per warp step.
__device__ __forceinline__ void transpose_raw(unsigned char* dst, const unsigned char* raw, int R, int warp,
                                              int lane) {
  const int nblk = 8 * (R / 8);  // (k8, r8) blocks
  const int q = lane >> 3, j = lane & 7;
  for (int b0 = warp * 4; b0 < nblk; b0 += 8 * 4) {
    const int b = b0 + q;  // this lane addresses a row of block b
    const int k8 = b & 7, r8 = b >> 3;
    const uint32_t src = smem_u32(raw) + (uint32_t)(((k8 * 8 + j) * (R + kRawPad) + r8 * 8) * 2);
    const uint32_t dsta = smem_u32(dst) + core_off(r8 * 8 + j, k8, R);
    uint32_t x0, x1, x2, x3;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(x0), "=r"(x1), "=r"(x2), "=r"(x3)
                 : "r"(src)
                 : "memory");
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(dsta), "r"(x0),
                 "r"(x1), "r"(x2), "r"(x3)
                 : "memory");
  }
}

// Slots of the copy ring: per slot the K-major A (128 x 64) and B (NP x 64)
// tiles and, for an MN-contiguous operand, its raw tile (64 x R, padded rows).
// Three slots (two chunks in flight) where one CTA per SM fills the grid; two
// for the forward layers, whose 147 KB of three slots would leave one CTA per
// SM and two waves of CTAs.
constexpr int kMaxSlots = 3;
template <bool AK, bool BK, int EPI>
__host__ __device__ constexpr int slots_of() {
  return (AK && !BK && EPI == 1) ? 2 : 3;
}
struct SlotLayout {
  size_t a, b, ra, rb, slot;
};
__host__ __device__ inline SlotLayout slot_layout(int NP, bool ak, bool bk) {
  SlotLayout L{};
  L.a = 0;
  L.b = (size_t)kBM * kBK * 2;
  size_t off = L.b + (size_t)NP * kBK * 2;
  L.ra = off;
  if (!ak) off += (size_t)64 * (kBM + kRawPad) * 2;
  L.rb = off;
  if (!bk) off += (size_t)64 * (NP + kRawPad) * 2;
  L.slot = (off + 1023) & ~size_t(1023);
  return L;
}

template <bool AK, bool BK, int EPI>
__global__ void __launch_bounds__(kThreads, 2) k_umma_gemm(UmmaGemmArgs a) {
  constexpr int kSlots = slots_of<AK, BK, EPI>();
  extern __shared__ __align__(1024) unsigned char smem[];
  const int n0 = blockIdx.x * kBN;
  const int N = min(a.N - n0, kBN);  // this CTA's columns
  const int NP = (N + 15) & ~15;     // MMA N (staged B rows)
  const SlotLayout L = slot_layout(NP, AK, BK);
  auto slot = [&](int sl) { return smem + (size_t)sl * L.slot; };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)kSlots * L.slot);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + kSlots);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tcols = a.tmem_cols;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0)
    for (int sl = 0; sl < kSlots; ++sl)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + sl)) : "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int m0 = blockIdx.y * kBM;
  const int kbeg = blockIdx.z * a.kps;
  const int kend = min(a.K, kbeg + a.kps);
  const int nk = kend > kbeg ? (kend - kbeg) / kBK : 0;
  const uint32_t id = idesc(NP);
  uint32_t ph = 0u;  // bit sl: the phase of slot sl's barrier to wait for
  bool ok = true;
  int last = -1;  // slot of the last commit
  // the copies of chunk c into its slot (K-major operands directly, the
  // others as they lie in memory, transposed when the chunk is used)
  auto issue = [&](int c) {
    if (c < nk) {
      unsigned char* sp = slot(c % kSlots);
      const int k0 = kbeg + c * kBK;
      if constexpr (AK) load_kmajor(sp + L.a, kBM, a.A, a.lda, m0, a.M, k0, tid);
      else load_raw(sp + L.ra, kBM, a.A, a.lda, m0, a.M, k0, tid);
      if constexpr (BK) load_kmajor(sp + L.b, NP, a.B, a.ldb, n0, a.N, k0, tid);
      else load_raw(sp + L.rb, NP, a.B, a.ldb, n0, a.N, k0, tid);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int c = 0; c < kSlots - 1; ++c) issue(c);
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int sl = kt % kSlots;
    // chunk kt + kSlots - 1 goes into the slot the MMAs of chunk kt - 1 read
    if (kt >= 1 && kt + kSlots - 1 < nk) {
      const int ps = (kt - 1) % kSlots;
      const bool arrived = mbar_wait(smem_u32(bar + ps), (ph >> ps) & 1u);
      ph ^= 1u << ps;
      if (__syncthreads_or(arrived ? 0 : 1)) {
        ok = false;
        break;
      }
    }
    issue(kt + kSlots - 1);
    // chunk kt's copies (this thread's); the kSlots - 1 newer groups may be in flight
    if constexpr (kSlots == 3) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    unsigned char* sp = slot(sl);
    if constexpr (!AK) transpose_raw(sp + L.a, sp + L.ra, kBM, warp, lane);
    if constexpr (!BK) transpose_raw(sp + L.b, sp + L.rb, NP, warp, lane);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t aa = smem_u32(sp + L.a), bb = smem_u32(sp + L.b);
#pragma unroll 1
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t ad = sdesc(aa + kk * 2 * (16 * kBM), 16 * kBM, 128);
        const uint64_t bd = sdesc(bb + kk * 2 * (16 * NP), 16 * NP, 128);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(bar + sl))
                   : "memory");
    }
    last = sl;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy in flight past this point
  // the last commit covers every MMA issued before it (on a timeout: one more
  // bounded wait so that no MMA is in flight when the TMEM is released)
  if (last >= 0) {
    const bool arrived = mbar_wait(smem_u32(bar + last), (ph >> last) & 1u);
    if (__syncthreads_or(arrived ? 0 : 1)) ok = false;
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
  } else if (nk > 0) {
    // tcgen05.ld gives lane l the row l of a 32 x 32 block; each block is
    // turned around in a per-warp shared-memory scratch (the stages are free
    // now) so that lanes take consecutive columns of one row at a time and the
    // global stores, loads and atomic adds are coalesced
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* scr = reinterpret_cast<float*>(smem) + warp * (32 * 33);
    const int quarter = warp & 3, colh = warp >> 2;
    const int rbase = m0 + quarter * 32;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int half = NP / 2;  // a multiple of 8; chunks of 32 columns (the last may be partial)
    const int cend = min(N, (colh + 1) * half);
    const int cb = n0;  // column of C of the block's column 0
#pragma unroll 1
    for (int c0 = colh * half; c0 < (colh + 1) * half; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + lane_off + (uint32_t)c0, v);
      if constexpr (EPI == 2) {
        // the ReLU mask of this lane's row (row rbase + lane) over the chunk's
        // 32 columns, read as four 16-byte pieces and applied in registers;
        // pieces past the last column (N is a multiple of 8) or rows past M read
        // nothing
        const int row = rbase + lane;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint4 w = make_uint4(0u, 0u, 0u, 0u);
          if (row < a.M && c0 + 8 * q < cend)
            w = __ldg(reinterpret_cast<const uint4*>(a.mask + (size_t)row * a.ldc + n0 + c0 + 8 * q));
          const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const uint32_t bits = (ws[h >> 1] >> ((h & 1) * 16)) & 0xFFFFu;
            // a BF16 value is > 0 exactly when its bits lie in [0x0001, 0x7F80]
            // (positive subnormals up to +inf; zeros, negatives and NaNs not)
            const bool pos = bits - 1u < 0x7F80u;
            if (!pos) v[8 * q + h] = 0u;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) scr[lane * 33 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int cl = c0 + lane;
      const int c = cb + cl;
      if (cl < cend) {
        float bias_c = 0.0f;
        if constexpr (EPI == 1) bias_c = a.bias[c];
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
          const int row = rbase + rr;
          if (row >= a.M) break;
          const float x = scr[rr * 33 + lane];
          if constexpr (EPI == 0) {
            float* dst = a.C + (size_t)row * a.ldc + c;
            if (gridDim.z > 1) atomicAdd(dst, x);
            else *dst = x;
          } else if constexpr (EPI == 1) {
            a.Cb[(size_t)row * a.ldc + c] = __float2bfloat16_rn(fmaxf(x + bias_c, 0.0f));
          } else {
            a.Cb[(size_t)row * a.ldc + c] = __float2bfloat16_rn(x);  // masked above
          }
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

using GemmKernel = void (*)(UmmaGemmArgs);

// the slots (the first reused as the epilogue's per-warp 32 x 33 FP32 scratch,
// 33.8 KB, within one slot for every N >= 16), then the barriers and the TMEM
// address
size_t gemm_smem(int N, bool ak, bool bk, int epi) {
  const int NP = (std::min(N, kBN) + 15) & ~15;
  const int slots = (ak && !bk && epi == 1) ? slots_of<true, false, 1>() : kMaxSlots;
  return (size_t)slots * slot_layout(NP, ak, bk).slot + 64;
}

}  // namespace

bool umma_gemm_supported(int M, int N, int K) {
  return M >= 1 && N >= 16 && N <= kMaxN && N % 8 == 0 && K >= kBK && K % kBK == 0;
}

cudaError_t umma_gemm(UmmaGemmArgs a, int splits, cudaStream_t s) {
  if (!umma_gemm_supported(a.M, a.N, a.K) || !a.A || !a.B || !a.err || splits < 1) return cudaErrorInvalidValue;
  if (a.a_kmajor ? (a.lda < a.K || a.lda % 8) : (a.lda < a.M || a.lda % 8 || a.M % 8)) return cudaErrorInvalidValue;
  if (a.b_kmajor ? (a.ldb < a.K || a.ldb % 8) : (a.ldb < a.N || a.ldb % 8)) return cudaErrorInvalidValue;
  // the masked epilogue reads the mask in 16-byte pieces
  if (a.epi == 2 && (!a.mask || a.ldc % 8 || reinterpret_cast<uintptr_t>(a.mask) % 16)) return cudaErrorInvalidValue;
  GemmKernel kern = nullptr;
  if (a.a_kmajor && !a.b_kmajor && a.epi == 1) kern = k_umma_gemm<true, false, 1>;
  else if (!a.a_kmajor && !a.b_kmajor && a.epi == 0) kern = k_umma_gemm<false, false, 0>;
  else if (a.a_kmajor && a.b_kmajor && a.epi == 2) kern = k_umma_gemm<true, true, 2>;
  if (!kern) return cudaErrorInvalidValue;
  const int NP = (std::min(a.N, kBN) + 15) & ~15;
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < NP) a.tmem_cols <<= 1;
  const size_t smem = gemm_smem(a.N, a.a_kmajor, a.b_kmajor, a.epi);
  // shared-memory attribute once per (device, kernel), from any host thread
  static std::mutex mu;
  constexpr int kDevs = 64;
  static bool attr[kDevs][3];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
  const int ki = kern == k_umma_gemm<true, false, 1> ? 0 : (kern == k_umma_gemm<false, false, 0> ? 1 : 2);
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr[dev][ki]) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)gemm_smem(kBN, a.a_kmajor, a.b_kmajor, a.epi))) != cudaSuccess)
        return e;
      attr[dev][ki] = true;
    }
  }
  int kps = ((a.K / splits + kBK - 1) / kBK) * kBK;
  a.kps = kps;
  dim3 grid((a.N + kBN - 1) / kBN, (a.M + kBM - 1) / kBM, (a.K + kps - 1) / kps);
  kern<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rlt2
