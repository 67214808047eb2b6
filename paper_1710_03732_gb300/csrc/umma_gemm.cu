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
#include <cuda.h>  // CUtensorMap (the encoder is taken from the driver at run time)
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

// mbar_wait that also gives up as soon as another role of the CTA has set *abort
__device__ __forceinline__ bool mbar_wait_or(uint32_t bar, uint32_t phase, volatile int* abort) {
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
    if ((it & 63) == 63 && *abort) return false;
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

// The epilogue of one 128 x NP accumulator block at TMEM address tacc (rows
// m0 .., columns n0 .. of C): tcgen05.ld gives lane l the row l of a 32 x 32
// block; each block is turned around in the warp's 32 x 33 FP32 scratch `scr`
// so that lanes take consecutive columns of one row at a time and the global
// stores, loads and atomic adds are coalesced.  Warp w drains TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31 over the column half w / 4.
template <int EPI>
__device__ __forceinline__ void store_block(const UmmaGemmArgs& a, uint32_t tacc, int m0, int n0, int N, int NP,
                                            float* scr, int warp, int lane, bool atomic) {
  const int quarter = warp & 3, colh = warp >> 2;
  const int rbase = m0 + quarter * 32;
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  const int half = NP / 2;  // a multiple of 8; chunks of 32 columns (the last may be partial)
  const int cend = min(N, (colh + 1) * half);
  const int cb = n0;  // column of C of the block's column 0
#pragma unroll 1
  for (int c0 = colh * half; c0 < (colh + 1) * half; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tacc + lane_off + (uint32_t)c0, v);
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
          if (atomic) atomicAdd(dst, x);
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
    // the stages are free now: the first holds the warps' scratch
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* scr = reinterpret_cast<float*>(smem) + warp * (32 * 33);
    store_block<EPI>(a, tmem, m0, n0, N, NP, scr, warp, lane, gridDim.z > 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}


// ---- row GEMM: C = A B for tall A (M rows, K <= 256), persistent ------------
// The forward layers (B = W as stored, K x N) and dH1 = dH2 W2^T (B = W2, N x K)
// read a few hundred KB of B and stream A through once.  A CTA (one per SM)
// owns up to 128 columns of C (grid.x) and loops over 128-row tiles
// (blockIdx.y, += gridDim.y).  Its B block for all of K is staged once by
// cp.async (transposed in shared memory if B is N-contiguous), both operands
// in the 128-byte-swizzled K-major layout.  Three roles then run concurrently:
//   thread 0     TMA producer: 64-wide K chunks of A (cp.async.bulk.tensor, one
//                16 KB box each) into a ring of slots running across tiles;
//   thread 32    MMA issuer: tcgen05.mma per chunk into one of two TMEM
//                accumulators (tiles alternate), commits to the slot's and,
//                at a tile's end, the accumulator's mbarrier;
//   warps 4..7   epilogue: drain an accumulator (tcgen05.ld), bias + ReLU or
//                the ReLU mask (dH1: the mask tile comes by TMA into the
//                staging buffer), BF16 into a swizzled staging tile, stored by
//                TMA (cp.async.bulk.tensor, rows past M clipped).
// Every mbarrier wait is bounded and gives up when another role has: the CTA
// then sets *err, lets its copies land and its MMAs finish (bounded) and
// releases its TMEM.
// ring slots and output staging buffers (two, so that a tile's epilogue does
// not wait for the previous tile's stores; dH1's also receive the ReLU mask
// tile by TMA ahead of the epilogue)
template <int EPI>
__host__ __device__ constexpr int row_slots() { return EPI == 1 ? 6 : 5; }
template <int EPI>
__host__ __device__ constexpr int row_stages() { return 2; }
constexpr int kRowMaxK = 256;

// The row kernel's operands use the 128-byte-swizzled K-major layout: row r of
// a 64-wide K chunk is one 128-byte line at r * 128, its 16-byte piece k8 at
// ((k8 ^ (r % 8)) * 16), each 8-row group 1024 bytes (the chunk 1024-aligned).
__device__ __forceinline__ uint32_t sw128_off(int r, int k8) {
  return (uint32_t)(r * 128 + ((k8 ^ (r & 7)) << 4));
}

// matrix descriptor of a 128-byte-swizzled K-major operand: start (the chunk's
// base + 32 bytes per 16-element K step), LBO unused (1), SBO 1024 bytes
// between 8-row groups, version 1, layout type 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// load_kmajor into the swizzled layout: 8 consecutive lanes copy one row's 128
// bytes (one line of global memory), a warp four rows (four wavefronts).
__device__ __forceinline__ void load_kmajor_sw(unsigned char* dst, int R, const bf16* g, int ld, int r0, int rmax,
                                               int k0, int tid) {
  for (int c = tid; c < R * 8; c += kThreads) {
    const int r = c >> 3, k8 = c & 7;
    const bool in = r0 + r < rmax;
    const bf16* src = g + (in ? (size_t)(r0 + r) * ld + k0 + k8 * 8 : 0);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst) + sw128_off(r, k8)), "l"(src),
                 "r"(in ? 16 : 0)
                 : "memory");
  }
}

// transpose_raw into the swizzled layout
__device__ __forceinline__ void transpose_raw_sw(unsigned char* dst, const unsigned char* raw, int R, int warp,
                                                 int lane) {
  const int nblk = 8 * (R / 8);
  const int q = lane >> 3, j = lane & 7;
  for (int b0 = warp * 4; b0 < nblk; b0 += 8 * 4) {
    const int b = b0 + q;
    const int k8 = b & 7, r8 = b >> 3;
    const uint32_t src = smem_u32(raw) + (uint32_t)(((k8 * 8 + j) * (R + kRawPad) + r8 * 8) * 2);
    const uint32_t dsta = smem_u32(dst) + sw128_off(r8 * 8 + j, k8);
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

struct RowLayout {
  size_t b, ring, stage, stage_bytes, bar, total;
};
__host__ __device__ inline RowLayout row_layout(int NP, int K, int slots, int stages) {
  RowLayout L{};
  L.b = 0;                                               // NP x K, K-major, swizzled
  L.ring = ((size_t)NP * K * 2 + 1023) & ~size_t(1023);  // slots x (128 x 64)
  L.stage = L.ring + (size_t)slots * kBM * kBK * 2;      // stages x the output tile: boxes of 128 rows x 64 columns
  L.stage_bytes = (size_t)((NP + 63) / 64) * kBM * 64 * 2;
  L.bar = L.stage + (size_t)stages * L.stage_bytes;
  L.total = L.bar + (2 * slots + 6) * 8 + 16;  // barriers, the abort flags, the TMEM address
  return L;
}

// The row kernel's epilogue (EPI 1 or 2) of one 128 x NP accumulator block, by
// the warp that may read TMEM lanes 32 quarter .. 32 quarter + 31: lane l holds
// row 32 quarter + l of the tile and, from tcgen05.ld, 32 consecutive columns
// of it at a time; it applies bias + ReLU (EPI 1, the bias read as broadcast
// 16-byte loads) or the ReLU mask of its row (EPI 2, read from `stage`, where
// TMA put the mask tile), packs BF16 pairs and writes them into `stage`, the
// tile in the 128-byte-swizzled layout of the TMA store (boxes of 64 columns;
// a warp's 32 lines take four wavefronts).
template <int EPI>
__device__ __forceinline__ void store_rows(const UmmaGemmArgs& a, uint32_t tacc, unsigned char* stage, int m0,
                                           int n0, int N, int NP, int quarter, int lane) {
  (void)m0;
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  const int cend = N;
#pragma unroll 1
  for (int c0 = 0; c0 < NP; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tacc + lane_off + (uint32_t)c0, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cq = c0 + 8 * q;  // first of the piece's 8 columns (N is a multiple of 8)
      if (cq >= cend) break;
      float f[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) f[h] = __uint_as_float(v[8 * q + h]);
      if constexpr (EPI == 1) {
        const float4 b0 = __ldg(reinterpret_cast<const float4*>(a.bias + n0 + cq));
        const float4 b1 = __ldg(reinterpret_cast<const float4*>(a.bias + n0 + cq + 4));
        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) f[h] = fmaxf(f[h] + bb[h], 0.0f);
      } else {
        // the ReLU mask of this row, staged by TMA where the output piece goes:
        // a BF16 value is > 0 exactly when its bits lie in [0x0001, 0x7F80]
        // (positive subnormals up to +inf)
        const uint4 w = *reinterpret_cast<const uint4*>(stage + (size_t)(cq >> 6) * (kBM * 128) +
                                                        sw128_off(quarter * 32 + lane, (cq & 63) >> 3));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          const uint32_t bits = (ws[h >> 1] >> ((h & 1) * 16)) & 0xFFFFu;
          if (!(bits - 1u < 0x7F80u)) f[h] = 0.0f;
        }
      }
      uint4 out;
      uint32_t* o = reinterpret_cast<uint32_t*>(&out);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(f[2 * h], f[2 * h + 1]);
        o[h] = *reinterpret_cast<const uint32_t*>(&p2);
      }
      // 128-byte-swizzled staging: box cq / 64, line r, 16-byte piece (cq % 64) / 8
      const int r = quarter * 32 + lane;
      *reinterpret_cast<uint4*>(stage + (size_t)(cq >> 6) * (kBM * 128) + sw128_off(r, (cq & 63) >> 3)) = out;
    }
  }
}

template <bool BK, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_umma_rows(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmC,
                const __grid_constant__ CUtensorMap tmM, UmmaGemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * kBN;
  const int N = min(a.N - n0, kBN);
  const int NP = (N + 15) & ~15;
  const int K = a.K, cpt = K / kBK;
  constexpr int kS = row_slots<EPI>(), kNS = row_stages<EPI>();
  const RowLayout L = row_layout(NP, K, kS, kNS);
  unsigned char* bs = smem + L.b;
  unsigned char* ring = smem + L.ring;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar);  // kS: the slot's A chunk has landed
  uint64_t* empty = full + kS;                          // kS: the MMAs reading the slot are done
  uint64_t* accf = empty + kS;                          // 2: an accumulator's tile is complete
  uint64_t* acce = accf + 2;                                   // 2: an accumulator has been drained
  uint64_t* mfull = acce + 2;                                  // 2: a staging buffer holds its tile's mask (EPI 2)
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mfull + 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mfull + 2) + 1;
  volatile int* epi_fail = reinterpret_cast<volatile int*>(mfull + 2) + 2;  // written by epilogue warps only
  const uint32_t tcols = 2 * kBN;  // two accumulators
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 2 * kS + 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + b)) : "memory");
    for (int b = 0; b < 2; ++b) {  // one arrival per epilogue warp
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(acce + b)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mfull + b)) : "memory");
    }
    *abort_flag = 0;
    *epi_fail = 0;
  }
  // B for all of K, K-major and swizzled: chunk kc (NP lines of 128 bytes) at bs + kc * NP * 128
  for (int kc = 0; kc < cpt; ++kc) {
    if constexpr (BK) {
      load_kmajor_sw(bs + (size_t)kc * NP * 128, NP, a.B, a.ldb, n0, a.N, kc * kBK, tid);
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
      load_raw(ring, NP, a.B, a.ldb, n0, a.N, kc * kBK, tid);  // the ring is free until the A copies start
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      transpose_raw_sw(bs + (size_t)kc * NP * 128, ring, NP, warp, lane);
      __syncthreads();
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int nmt = (a.M + kBM - 1) / kBM;
  const int ntile = blockIdx.y < nmt ? (nmt - 1 - (int)blockIdx.y) / (int)gridDim.y + 1 : 0;
  const int G = ntile * cpt;  // A chunks of this CTA
  if (tid == 0 && G > 0) {
    // TMA producer: the A chunk g of tile g / cpt lands in slot g % kS (one 16 KB box,
    // 128-byte swizzled, rows past M zero-filled); a slot is refilled once the MMAs of
    // the chunk it held are done
    int issued = 0;
    for (; issued < G; ++issued) {
      const int i = issued / cpt, kc = issued - i * cpt, sl = issued % kS;
      if (issued >= kS &&
          !mbar_wait_or(smem_u32(empty + sl), (uint32_t)(((issued - kS) / kS) & 1), abort_flag)) {
        *abort_flag = 1;
        atomicExch(a.err, 1);
        break;
      }
      const uint32_t bar = smem_u32(full + sl);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBM * kBK * 2) : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              smem_u32(ring + (size_t)sl * kBM * kBK * 2)),
          "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kc * kBK), "r"((blockIdx.y + i * gridDim.y) * kBM), "r"(bar)
          : "memory");
    }
    // every started copy lands before the shared memory is released (the last kS
    // chunks; an earlier one was consumed before its slot was refilled)
    for (int c = issued - 1; c >= 0 && c >= issued - kS; --c)
      (void)mbar_wait(smem_u32(full + c % kS), (uint32_t)((c / kS) & 1));
  } else if (tid == 32 && G > 0) {
    // MMA issuer: chunk g into the accumulator (g / cpt) % 2, committed to the slot's
    // barrier (the producer refills it) and, at a tile's last chunk, to the accumulator's
    const uint32_t id = idesc(NP);
    const uint32_t bb = smem_u32(bs);
    int g = 0;
    for (; g < G; ++g) {
      const int i = g / cpt, kc = g - i * cpt, sl = g % kS;
      bool ok = mbar_wait_or(smem_u32(full + sl), (uint32_t)((g / kS) & 1), abort_flag);
      // the first chunk of tile i writes the accumulator tile i - 2 used: wait until it is drained
      if (ok && kc == 0 && i >= 2) ok = mbar_wait_or(smem_u32(acce + (i & 1)), (uint32_t)(((i - 2) >> 1) & 1), abort_flag);
      if (!ok) {
        *abort_flag = 1;
        atomicExch(a.err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (a.withhold) continue;  // diagnostics: nothing issued, nothing committed
      const uint32_t aa = smem_u32(ring + (size_t)sl * kBM * kBK * 2);
      const uint32_t acc = tmem + (uint32_t)((i & 1) * kBN);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t ad = sdesc_sw128(aa + kk * 32);
        const uint64_t bd = sdesc_sw128(bb + (uint32_t)(kc * NP * 128 + kk * 32));
        const uint32_t accum = (kc > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
            "l"(ad), "l"(bd), "r"(id), "r"(accum)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(empty + sl))
                   : "memory");
      if (kc == cpt - 1)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accf + (i & 1)))
                     : "memory");
    }
    // no MMA in flight when the TMEM is released (the last commit covers all)
    if (g > 0 && !a.withhold) (void)mbar_wait(smem_u32(empty + (g - 1) % kS), (uint32_t)(((g - 1) / kS) & 1));
  } else if (warp >= 4) {
    // epilogue warps: warp 4 + q drains TMEM lanes 32 q .. 32 q + 31 (rows of the tile) over all
    // columns into the staging tile j % 2, which thread 128 then stores by TMA (boxes of 64
    // columns, rows past M clipped); the named barrier 1 orders the four warps around it
    const int q = warp - 4;
    const bool leader = tid == 128;
    const int nbox = (NP + 63) / 64;
    // EPI 2: the mask tile of tile j comes by TMA into staging buffer j % 2 (zeros past M)
    auto load_mask = [&](int j) {
      const uint32_t bar = smem_u32(mfull + (j & 1));
      unsigned char* st = smem + L.stage + (size_t)(j & 1) * L.stage_bytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(nbox * kBM * 128)
                   : "memory");
      for (int h = 0; h < nbox; ++h)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(smem_u32(st + (size_t)h * kBM * 128)),
            "l"(reinterpret_cast<uint64_t>(&tmM)), "r"(n0 + 64 * h), "r"((blockIdx.y + j * gridDim.y) * kBM),
            "r"(bar)
            : "memory");
    };
    if constexpr (EPI == 2) {
      if (leader && ntile > 0) load_mask(0);
    }
    for (int j = 0; j < ntile; ++j) {
      // warp-uniform: the TMEM loads below are warp-collective
      bool arrived = mbar_wait_or(smem_u32(accf + (j & 1)), (uint32_t)((j >> 1) & 1), abort_flag);
      if constexpr (EPI == 2)
        arrived = arrived && mbar_wait_or(smem_u32(mfull + (j & 1)), (uint32_t)((j >> 1) & 1), abort_flag);
      if (!__all_sync(0xffffffffu, arrived) && lane == 0) *epi_fail = 1;
      // one staging buffer (EPI 1): free once the TMA stores of tile j - 1 have read it
      if (kNS == 1 && leader) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      // one decision for the four warps: the flag is written only before this barrier
      if (*epi_fail) {
        if (leader) {
          atomicExch(a.err, 1);
          // the mask copy of this tile (the only one started) lands before the CTA ends
          if constexpr (EPI == 2) (void)mbar_wait(smem_u32(mfull + (j & 1)), (uint32_t)((j >> 1) & 1));
        }
        *abort_flag = 1;
        break;
      }
      unsigned char* stage = smem + L.stage + (size_t)(kNS == 1 ? 0 : (j & 1)) * L.stage_bytes;
      const int m0 = (blockIdx.y + j * gridDim.y) * kBM;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      store_rows<EPI>(a, tmem + (uint32_t)((j & 1) * kBN), stage, m0, n0, N, NP, q, lane);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acce + (j & 1))) : "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (leader) {
        for (int h = 0; h < nbox; ++h)
          asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                           reinterpret_cast<uint64_t>(&tmC)),
                       "r"(n0 + 64 * h), "r"(m0), "r"(smem_u32(stage + (size_t)h * kBM * 128))
                       : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        if constexpr (EPI == 2) {
          // buffer (j + 1) % 2 is free once the stores of tile j - 1 have read it: its mask next
          if (j + 1 < ntile) {
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            load_mask(j + 1);
          }
        }
      }
    }
    // the stores complete before the CTA ends
    if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
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

using RowKernel = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, UmmaGemmArgs);

// cuTensorMapEncodeTiled, taken from the driver once (no link to libcuda)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled tensor_map_encoder() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// The TMA map of the row kernel's A (M rows of K BF16, row stride lda): boxes of
// 64 K x 128 rows, 128-byte swizzle (the MMA's K-major layout), rows past M read
// as zeros.  False (and the tile kernel runs) where TMA cannot address A.
bool encode_rows_map(CUtensorMap* m, const UmmaGemmArgs& a) {
  const EncodeTiled enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(a.A) & 15) || (a.lda * 2) % 16) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)a.M};
  const cuuint64_t strides[1] = {(cuuint64_t)a.lda * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(a.A), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The TMA map of the row kernel's output Cb (M rows of N BF16, row stride ldc):
// boxes of 64 columns x 128 rows from the 128-byte-swizzled staging tile; the
// parts of a box past N or M are not written.
// (also the map of the ReLU mask of dH1, an M x N BF16 array with the same
// leading dimension: read into the staging tile, zeros past M)
bool encode_out_map(CUtensorMap* m, const UmmaGemmArgs& a, const bf16* p) {
  const EncodeTiled enc = tensor_map_encoder();
  if (!enc || !p || (reinterpret_cast<uintptr_t>(p) & 15) || (a.ldc * 2) % 16) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)a.N, (cuuint64_t)a.M};
  const cuuint64_t strides[1] = {(cuuint64_t)a.ldc * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  constexpr int kDevs = 64;
  if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
  static std::mutex mu;
  // tall products (the forward layers, dH1): the persistent row kernel, whose
  // epilogue writes and reads 16-byte pieces of C, the bias and the mask
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  CUtensorMap tmA, tmC, tmM;
  if (a.a_kmajor && splits == 1 && a.K <= kRowMaxK &&
      ((!a.b_kmajor && a.epi == 1) || (a.b_kmajor && a.epi == 2)) && a.Cb && al16(a.Cb) && a.ldc % 8 == 0 &&
      (a.epi != 1 || (a.bias && al16(a.bias))) && encode_rows_map(&tmA, a) && encode_out_map(&tmC, a, a.Cb) &&
      (a.epi != 2 || encode_out_map(&tmM, a, a.mask))) {
    if (a.epi != 2) tmM = tmC;  // unused
    static bool rattr[kDevs][2];
    static int sms[kDevs];
    const RowKernel rk = a.b_kmajor ? k_umma_rows<true, 2> : k_umma_rows<false, 1>;
    const int ri = a.b_kmajor ? 1 : 0;
    const int slots = a.b_kmajor ? row_slots<2>() : row_slots<1>();
    const int stages = a.b_kmajor ? row_stages<2>() : row_stages<1>();
    {
      std::lock_guard<std::mutex> lock(mu);
      if (!sms[dev] && (e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
      if (!rattr[dev][ri]) {
        if ((e = cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)row_layout(kBN, kRowMaxK, slots, stages).total)) != cudaSuccess)
          return e;
        rattr[dev][ri] = true;
      }
    }
    const int NP = (std::min(a.N, kBN) + 15) & ~15;
    const int gx = (a.N + kBN - 1) / kBN, nmt = (a.M + kBM - 1) / kBM;
    const int gy = std::max(1, std::min(nmt, sms[dev] / gx));  // one CTA per SM
    rk<<<dim3(gx, gy), kThreads, row_layout(NP, a.K, slots, stages).total, s>>>(tmA, tmC, tmM, a);
    return cudaGetLastError();
  }
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
  static bool attr[kDevs][3];
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
