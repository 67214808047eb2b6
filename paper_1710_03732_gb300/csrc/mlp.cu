// Learned warm start for the Z-LAPs (not in the paper; the paper's only warm
// start is parent -> child multipliers in branch and bound, Section 4).
//
// A per-row network predicts how much each row dual of a Z-LAP changed since
// the previous iteration, from that row's sorted, column-min-reduced,
// max-scaled costs, the row's previous dual and m/32 (34 features, so one set
// of weights serves every LAP size m <= 32): u0 = u_prev + scale * net.  The prediction only seeds the exact Hungarian: the column-min
// repair makes it feasible and the searches finish the solve, so bounds are
// exactly those of a cold start; what the network saves is augmenting searches.
//
// Network: 34 -> H -> H -> 1, ReLU, BF16 weights and activations, FP32
// accumulation.  Inference of the H = 256 network runs on the 5th-generation
// tensor cores in one fused kernel (tcgen05.mma with TMEM accumulators,
// umma.cu); the training GEMMs (forward layers, and the backward products
// with transposed operands) of widths up to 256 run on a tcgen05 GEMM
// (umma_gemm.cu); wider networks use a hand-written mma.sync (m16n8k16,
// BF16 -> FP32) GEMM with ldmatrix fragment loads and a cp.async
// double-buffered shared-memory pipeline.
// Features are built without FP64 arithmetic (FP64 -> FP32 by truncating the
// significand on the integer pipe) because FP64 is GB300's scarce resource.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "rlt2_internal.h"
#include "rlt2_mlp_gemm.h"

namespace rlt2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kIn = 34;      // features per row
constexpr int kInPad = 64;   // padded input width (GEMM K)
constexpr int kChunk = 1 << 18;  // rows per inference/training chunk
using bf16 = __nv_bfloat16;

__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  unsigned out;
  if (e == 0) {
    out = sign;
  } else {
    const int ef = e - 1023 + 127;
    if (ef <= 0) out = sign;
    else if (ef >= 255) out = sign | 0x7f7fffffu;
    else out = sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffff);
  }
  return __uint_as_float(out);
}

// ------------------------------------------------------------- features ----
// One warp per tile; lane j holds column j.  Writes 64 BF16 inputs per row
// (34 features + zero padding), optional FP32 targets and the tile scale.
// The tile (at most 8 KB) is read three times -- column minima, the scale, then
// row by row for the sorts -- so only the first pass reaches DRAM and the
// kernel keeps few registers (occupancy hides the load latency).
__global__ void __launch_bounds__(256, 4) k_features(long long ntiles, int m, const double* __restrict__ tiles,
                                                     const double* __restrict__ prev_u,
                                                     const double* __restrict__ target_u, bf16* __restrict__ X,
                                                     float* __restrict__ target, float* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const bool col = lane < m;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles; t += nw) {
    const double* c = tiles + t * m * m;
    float cmin = INFINITY;
    for (int i = 0; i < m; ++i)
      if (col) cmin = fminf(cmin, f32_trunc(c[i * m + lane]));
    float rmax = 0.0f;
    for (int i = 0; i < m; ++i)
      if (col) rmax = fmaxf(rmax, __fsub_rn(f32_trunc(c[i * m + lane]), cmin));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(kFull, rmax, off));
    const float s = rmax > 0.0f ? rmax : 1.0f;
    const float inv = __fdiv_rn(1.0f, s);
    if (lane == 0 && scale) scale[t] = s;
    for (int i = 0; i < m; ++i) {
      float v = col ? __fmul_rn(__fsub_rn(f32_trunc(c[i * m + lane]), cmin), inv) : INFINITY;
      // bitonic sort across the warp, ascending
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
          const float o = __shfl_xor_sync(kFull, v, j);
          const bool up = (lane & k) == 0;
          const bool low = (lane & j) == 0;
          v = (low == up) ? fminf(v, o) : fmaxf(v, o);
        }
      }
      const long long row = t * m + i;
      bf16* xr = X + row * kInPad;
      xr[lane] = __float2bfloat16_rn(col ? v : 0.0f);
      float hi = 0.0f;
      if (lane == 0) hi = prev_u ? __fmul_rn(f32_trunc(prev_u[row]), inv) : 0.0f;
      if (lane == 1) hi = (float)m / 32.0f;
      xr[32 + lane] = __float2bfloat16_rn(hi);
    }
    if (target && target_u && col) {
      // the network predicts the change of the row dual since the previous iteration
      const long long r = t * m + lane;
      const double d = prev_u ? __dsub_rn(target_u[r], prev_u[r]) : target_u[r];
      target[r] = __fmul_rn(f32_trunc(d), inv);
    }
  }
}

// ----------------------------------------------------------------- GEMM ----
// C[M x N] = A[M x K] * B[K x N] with BF16 inputs and FP32 accumulation on the
// tensor cores (mma.sync m16n8k16).  TA: A is stored transposed ([K x M] row-
// major); TB: B is stored transposed ([N x K] row-major).  M, N multiples of
// 64, K a multiple of 32 (buffers are padded).  Epilogues: EPI 0 FP32 store
// (atomic add when split over K), EPI 1 bias + ReLU -> BF16, EPI 2 ReLU-mask
// by `mask` (> 0) -> BF16.
constexpr int BM = 64, BN = 64, BK = 32;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g));
}
__device__ __forceinline__ void ldm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16* __restrict__ A, int lda,
                                              const bf16* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              bf16* __restrict__ Cb, const float* __restrict__ bias,
                                              const bf16* __restrict__ mask, int kps) {
  constexpr int A_R = TA ? BK : BM, A_C = (TA ? BM : BK) + 8;
  constexpr int B_R = TB ? BN : BK, B_C = (TB ? BK : BN) + 8;
  __shared__ __align__(16) bf16 sA[2][A_R][A_C];
  __shared__ __align__(16) bf16 sB[2][B_R][B_C];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kps;
  const int kend = min(K, kbeg + kps);
  const int nk = (kend - kbeg) / BK;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;

  auto load = [&](int buf, int k0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int ch = tid + i * 128;
      if (!TA) {
        const int r = ch >> 2, c8 = (ch & 3) * 8;
        cp16(&sA[buf][r][c8], A + (size_t)(m0 + r) * lda + k0 + c8);
      } else {
        const int r = ch >> 3, c8 = (ch & 7) * 8;
        cp16(&sA[buf][r][c8], A + (size_t)(k0 + r) * lda + m0 + c8);
      }
      if (!TB) {
        const int r = ch >> 3, c8 = (ch & 7) * 8;
        cp16(&sB[buf][r][c8], B + (size_t)(k0 + r) * ldb + n0 + c8);
      } else {
        const int r = ch >> 2, c8 = (ch & 3) * 8;
        cp16(&sB[buf][r][c8], B + (size_t)(n0 + r) * ldb + k0 + c8);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  if (nk > 0) load(0, kbeg);
  const int mat = lane >> 3, rr = lane & 7;
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) {
      load((kt + 1) & 1, kbeg + (kt + 1) * BK);
      asm volatile("cp.async.wait_group 1;\n" ::);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncthreads();
    const int buf = kt & 1;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int mrow = wm * 32 + mi * 16;
        if (!TA)
          ldm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], &sA[buf][mrow + (mat & 1) * 8 + rr][kk + (mat >> 1) * 8]);
        else
          ldm_x4_t(af[mi][0], af[mi][1], af[mi][2], af[mi][3],
                   &sA[buf][kk + (mat >> 1) * 8 + rr][mrow + (mat & 1) * 8]);
      }
      unsigned bfr[4][2];
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        const int ncol = wn * 32 + nj * 16;
        unsigned r0, r1, r2, r3;
        if (!TB)
          ldm_x4_t(r0, r1, r2, r3, &sB[buf][kk + (mat & 1) * 8 + rr][ncol + (mat >> 1) * 8]);
        else
          ldm_x4(r0, r1, r2, r3, &sB[buf][ncol + (mat >> 1) * 8 + rr][kk + (mat & 1) * 8]);
        bfr[nj * 2][0] = r0;
        bfr[nj * 2][1] = r1;
        bfr[nj * 2 + 1][0] = r2;
        bfr[nj * 2 + 1][1] = r3;
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma16816(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
    }
    __syncthreads();
  }
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wm * 32 + mi * 16 + g + h * 8;
        const int c = n0 + wn * 32 + ni * 8 + tq * 2;
        float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
        if (EPI == 0) {
          if (gridDim.z > 1) {
            atomicAdd(C + (size_t)r * ldc + c, v0);
            atomicAdd(C + (size_t)r * ldc + c + 1, v1);
          } else {
            C[(size_t)r * ldc + c] = v0;
            C[(size_t)r * ldc + c + 1] = v1;
          }
        } else if (EPI == 1) {
          v0 = fmaxf(v0 + bias[c], 0.0f);
          v1 = fmaxf(v1 + bias[c + 1], 0.0f);
          Cb[(size_t)r * ldc + c] = __float2bfloat16_rn(v0);
          Cb[(size_t)r * ldc + c + 1] = __float2bfloat16_rn(v1);
        } else {
          const float m0v = __bfloat162float(mask[(size_t)r * ldc + c]);
          const float m1v = __bfloat162float(mask[(size_t)r * ldc + c + 1]);
          Cb[(size_t)r * ldc + c] = __float2bfloat16_rn(m0v > 0.0f ? v0 : 0.0f);
          Cb[(size_t)r * ldc + c + 1] = __float2bfloat16_rn(m1v > 0.0f ? v1 : 0.0f);
        }
      }
}

// ------------------------------------------------------- small kernels ----
// out[r] = b3 + sum_j H2[r][j] * w3[j] (one warp per row, fixed order)
__global__ void k_out(long long rows, int H, const bf16* __restrict__ H2, const float* __restrict__ w3,
                      const float* __restrict__ b3, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += nw) {
    float s = 0.0f;
    for (int j = lane; j < H; j += 32) s += __bfloat162float(H2[r * H + j]) * w3[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if (lane == 0) out[r] = s + *b3;
  }
}

// u0 = prev + out * scale of the row's tile (FP32 product, widened exactly);
// predicted changes below `gate` (in scaled units) are dropped so that the row
// keeps its previous dual exactly
__global__ void k_u0(long long rows, int m, const float* __restrict__ out, const float* __restrict__ scale,
                     const double* __restrict__ prev_u, float gate, double* __restrict__ u0) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
    const float o = fabsf(out[r]) < gate ? 0.0f : out[r];
    const double d = (double)__fmul_rn(o, scale[r / m]);
    u0[r] = prev_u ? __dadd_rn(prev_u[r], d) : d;
  }
}

// dout = (out - t)/nvalid on valid rows; loss += 0.5 e^2 / nvalid
__global__ void k_loss(long long rows, long long nvalid, const float* out, const float* t, float* dout, double* loss) {
  __shared__ double red[256];
  double part = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
    if (r < nvalid) {
      const float e = out[r] - t[r];
      dout[r] = e / (float)nvalid;
      part += 0.5 * (double)e * (double)e / (double)nvalid;
    } else {
      dout[r] = 0.0f;
    }
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// dH2 = relu'(H2) * dout x w3 (BF16)
// one thread per 8 consecutive elements of a row (16-byte loads and stores; H
// a multiple of 8, rows * H / 8 < 2^31: 32-bit index arithmetic)
__global__ void k_dh2(long long rows, int H, const bf16* H2, const float* dout, const float* w3, bf16* dH2) {
  const unsigned per = (unsigned)(H / 8), tot = (unsigned)(rows * per);
  for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < tot; p += gridDim.x * blockDim.x) {
    const unsigned r = p / per, j0 = (p - r * per) * 8;
    const uint4 hv = *reinterpret_cast<const uint4*>(H2 + (size_t)p * 8);
    const bf16* h = reinterpret_cast<const bf16*>(&hv);
    const float d = dout[r];
    uint4 ov;
    bf16* o = reinterpret_cast<bf16*>(&ov);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16_rn(__bfloat162float(h[k]) > 0.0f ? d * w3[j0 + k] : 0.0f);
    *reinterpret_cast<uint4*>(dH2 + (size_t)p * 8) = ov;
  }
}

// out[j] += sum_r M[r][j] * (rs ? rs[r] : 1) over a slice of rows per block
__global__ void k_colsum(long long rows, int cols, const bf16* Mx, const float* rs, float* out) {
  const int j = threadIdx.x;  // blockDim.x == cols (<= 1024)
  const long long per = (rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  float s = 0.0f;
  for (long long r = r0; r < r1; ++r) s += __bfloat162float(Mx[r * cols + j]) * (rs ? rs[r] : 1.0f);
  atomicAdd(out + j, s);
}

__global__ void k_sum(long long rows, const float* x, float* out) {
  __shared__ float red[256];
  float s = 0.0f;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
    s += x[r];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// AdamW on FP32 master weights; refreshes the BF16 copy when given.
__global__ void k_adamw(int n, float* w, float* mo, float* ve, const float* g, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2, bf16* wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    mo[i] = b1 * mo[i] + (1.0f - b1) * gi;
    ve[i] = b2 * ve[i] + (1.0f - b2) * gi * gi;
    const float mh = mo[i] / c1, vh = ve[i] / c2;
    float x = w[i] * (1.0f - lr * wd) - lr * mh / (sqrtf(vh) + eps);
    w[i] = x;
    if (wb) wb[i] = __float2bfloat16_rn(x);
  }
}

// deterministic init: normal(0, std) from a counter-based hash (SplitMix64 + Box-Muller)
__device__ __forceinline__ unsigned long long smix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_init_normal(int n, int valid_rows, int cols, float stdv, unsigned long long seed, float* w,
                              bf16* wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long a = smix(seed ^ (2ull * i)), b = smix(seed ^ (2ull * i + 1));
    const float u1 = ((a >> 40) + 1) * (1.0f / 16777217.0f), u2 = (b >> 40) * (1.0f / 16777216.0f);
    float x = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2) * stdv;
    if (i / cols >= valid_rows) x = 0.0f;
    w[i] = x;
    if (wb) wb[i] = __float2bfloat16_rn(x);
  }
}

// gather a minibatch: rows idx = hash(seed, r) % nrows
// one thread per 16-byte piece of a sampled row (8 pieces per row, the row's
// hash computed once per piece instead of once per element)
__global__ void k_gather(long long brows, long long nrows, unsigned long long seed, const bf16* X, const float* T,
                         bf16* Xb, float* Tb) {
  constexpr int kPieces = kInPad / 8;
  const long long tot = brows * kPieces;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / kPieces;
    const int k = (int)(e - r * kPieces);
    const long long src = (long long)(smix(seed ^ (unsigned long long)r) % (unsigned long long)nrows);
    *reinterpret_cast<uint4*>(Xb + r * kInPad + k * 8) = *reinterpret_cast<const uint4*>(X + src * kInPad + k * 8);
    if (k == 0) Tb[r] = T[src];
  }
}

}  // namespace
}  // namespace rlt2

using namespace rlt2;

struct rlt2_mlp {
  int H = 256;
  cudaStream_t stream = nullptr;
  // parameters: FP32 masters, BF16 copies of the two GEMM weights, Adam moments
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr;
  bf16 *W1b = nullptr, *W2b = nullptr;
  float* mom = nullptr;  // 2 * nparams
  float* grad = nullptr; // nparams, same packing as the parameters
  long long nparams = 0;
  int adam_t = 0;
  float gate = 0.0f;
  // dataset (feature rows + targets)
  bf16* Xd = nullptr;
  float* Td = nullptr;
  long long rows = 0, cap = 0;
  // scratch for one chunk
  bf16 *Xc = nullptr, *H1 = nullptr, *H2 = nullptr, *dH2 = nullptr, *dH1 = nullptr;
  float *out = nullptr, *tgt = nullptr, *dout = nullptr, *scale = nullptr;
  double* loss = nullptr;
  int* err = nullptr;  // set by the tensor-core inference kernel on a timed-out wait
};

namespace {
// parameter packing: W1 [64 x H] | b1 [H] | W2 [H x H] | b2 [H] | w3 [H] | b3 [1]
void param_ptrs(rlt2_mlp* m) {
  const int H = m->H;
  float* base = m->W1;
  m->b1 = base + kInPad * H;
  m->W2 = m->b1 + H;
  m->b2 = m->W2 + (size_t)H * H;
  m->w3 = m->b2 + H;
  m->b3 = m->w3 + H;
}

// ta: A stored [K x M]; tb: B stored [N x K].  Widths up to 256 run on the
// tcgen05 GEMM (umma_gemm.cu; err: its timeout flag), others on the mma.sync one.
cudaError_t gemm(bool ta, bool tb, int epi, int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
                 float* C, int ldc, bf16* Cb, const float* bias, const bf16* mask, int splits, int* err,
                 cudaStream_t s) {
  const bool tc_case = (!ta && !tb && epi == 1) || (ta && !tb && epi == 0) || (!ta && tb && epi == 2);
  if (err && tc_case && umma_gemm_supported(M, N, K)) {
    UmmaGemmArgs u{};
    u.M = M;
    u.N = N;
    u.K = K;
    u.A = A;
    u.lda = lda;
    u.a_kmajor = !ta;
    u.B = B;
    u.ldb = ldb;
    u.b_kmajor = tb;
    u.epi = epi;
    u.C = C;
    u.ldc = ldc;
    u.Cb = Cb;
    u.bias = bias;
    u.mask = mask;
    u.err = err;
    // a K split over the batch (weight gradients): chunks of 512 rows per CTA,
    // so that the few 128-row blocks of the output still fill the GPU
    const int tsplits = splits > 1 ? std::max(splits, std::min(64, K / 512)) : 1;
    return umma_gemm(u, tsplits, s);
  }
  const int kps = ((K / splits + BK - 1) / BK) * BK;
  dim3 grid(N / BN, M / BM, (K + kps - 1) / kps);
#define RLT2_GEMM_CASE(TA_, TB_, EPI_)                                                                       \
  if (ta == TA_ && tb == TB_ && epi == EPI_) {                                                             \
    k_gemm<TA_, TB_, EPI_><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, Cb, bias, mask, kps);     \
    return cudaGetLastError();                                                                             \
  }
  RLT2_GEMM_CASE(false, false, 1)
  RLT2_GEMM_CASE(false, true, 2)
  RLT2_GEMM_CASE(true, false, 0)
  RLT2_GEMM_CASE(false, false, 0)
#undef RLT2_GEMM_CASE
  return cudaErrorInvalidValue;
}

// forward on `rows` (multiple of 64) rows of X -> out (FP32)
cudaError_t forward(rlt2_mlp* m, const bf16* X, long long rows, float* out, cudaStream_t s) {
  const int H = m->H;
  cudaError_t e;
  if ((e = gemm(false, false, 1, (int)rows, H, kInPad, X, kInPad, m->W1b, H, nullptr, H, m->H1, m->b1, nullptr, 1,
                m->err, s)) != cudaSuccess)
    return e;
  if ((e = gemm(false, false, 1, (int)rows, H, H, m->H1, H, m->W2b, H, nullptr, H, m->H2, m->b2, nullptr, 1, m->err, s)) !=
      cudaSuccess)
    return e;
  k_out<<<(int)std::min<long long>(4096, (rows + 7) / 8), 256, 0, s>>>(rows, H, m->H2, m->w3, m->b3, out);
  return cudaGetLastError();
}

// loss and gradients (accumulated into m->grad) for `rows` rows of which
// `nvalid` carry targets T
cudaError_t backward(rlt2_mlp* m, const bf16* X, const float* T, long long rows, long long nvalid, cudaStream_t s) {
  const int H = m->H;
  cudaError_t e;
  float* gW1 = m->grad;
  float* gb1 = gW1 + kInPad * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (size_t)H * H;
  float* gw3 = gb2 + H;
  float* gb3 = gw3 + H;
  if ((e = forward(m, X, rows, m->out, s)) != cudaSuccess) return e;
  k_loss<<<256, 256, 0, s>>>(rows, nvalid, m->out, T, m->dout, m->loss);
  k_dh2<<<4096, 256, 0, s>>>(rows, H, m->H2, m->dout, m->w3, m->dH2);
  const int gsplit = (int)std::max<long long>(1, std::min<long long>(256, rows / 1024));
  // column sums: 32 rows per block (latency-bound with fewer blocks), atomic adds
  const int csplit = (int)std::max<long long>(1, std::min<long long>(4096, rows / 32));
  k_colsum<<<csplit, H, 0, s>>>(rows, H, m->H2, m->dout, gw3);
  k_sum<<<64, 256, 0, s>>>(rows, m->dout, gb3);
  if ((e = gemm(true, false, 0, H, H, (int)rows, m->H1, H, m->dH2, H, gW2, H, nullptr, nullptr, nullptr, gsplit, m->err, s)) !=
      cudaSuccess)
    return e;
  k_colsum<<<csplit, H, 0, s>>>(rows, H, m->dH2, nullptr, gb2);
  if ((e = gemm(false, true, 2, (int)rows, H, H, m->dH2, H, m->W2b, H, nullptr, H, m->dH1, nullptr, m->H1, 1, m->err, s)) !=
      cudaSuccess)
    return e;
  if ((e = gemm(true, false, 0, kInPad, H, (int)rows, X, kInPad, m->dH1, H, gW1, H, nullptr, nullptr, nullptr, gsplit,
                m->err, s)) != cudaSuccess)
    return e;
  k_colsum<<<csplit, H, 0, s>>>(rows, H, m->dH1, nullptr, gb1);
  return cudaGetLastError();
}

cudaError_t ensure_dataset(rlt2_mlp* m, long long need) {
  if (need <= m->cap) return cudaSuccess;
  long long cap = std::max<long long>(need, 2 * m->cap);
  cap = (cap + 63) / 64 * 64;
  bf16* X = nullptr;
  float* T = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&X, sizeof(bf16) * cap * kInPad)) != cudaSuccess) return e;
  if ((e = cudaMalloc((void**)&T, sizeof(float) * cap)) != cudaSuccess) {
    cudaFree(X);
    return e;
  }
  if (m->rows) {
    cudaMemcpyAsync(X, m->Xd, sizeof(bf16) * m->rows * kInPad, cudaMemcpyDeviceToDevice, m->stream);
    cudaMemcpyAsync(T, m->Td, sizeof(float) * m->rows, cudaMemcpyDeviceToDevice, m->stream);
    cudaStreamSynchronize(m->stream);
  }
  cudaFree(m->Xd);
  cudaFree(m->Td);
  m->Xd = X;
  m->Td = T;
  m->cap = cap;
  return cudaSuccess;
}
}  // namespace

namespace rlt2 {
// tcgen05 inference of the H = 256 network (umma.cu)
cudaError_t umma_mlp_forward(const bf16* X, long long rows, const bf16* W1, const float* b1, const bf16* W2,
                             const float* b2, const float* w3, const float* b3, float* out, int* err,
                             cudaStream_t s, bool withhold_commit = false);

// Predict Z-LAP row duals u0 (FP64) for ntiles tiles of size m; prev_u nullable.
cudaError_t mlp_predict_enqueue(rlt2_mlp* m, long long ntiles, int mz, const double* tiles, const double* prev_u,
                                double* u0, cudaStream_t s, int* launched) {
  cudaError_t e;
  const long long tiles_per_chunk = std::max<long long>(1, kChunk / mz);
  for (long long t0 = 0; t0 < ntiles; t0 += tiles_per_chunk) {
    const long long nt = std::min(tiles_per_chunk, ntiles - t0);
    const long long rows = nt * mz, prows = (rows + 63) / 64 * 64;
    k_features<<<(int)std::min<long long>(8192, (nt + 7) / 8), 256, 0, s>>>(
        nt, mz, tiles + t0 * mz * mz, prev_u ? prev_u + t0 * mz : nullptr, nullptr, m->Xc, nullptr, m->scale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (prows > rows && (e = cudaMemsetAsync(m->Xc + rows * kInPad, 0, sizeof(bf16) * (prows - rows) * kInPad, s)) !=
                            cudaSuccess)
      return e;
    if (m->H == 256) {
      // tcgen05 path: the whole network in one persistent kernel
      if ((e = umma_mlp_forward(m->Xc, rows, m->W1b, m->b1, m->W2b, m->b2, m->w3, m->b3, m->out, m->err, s)) !=
          cudaSuccess)
        return e;
    } else if ((e = forward(m, m->Xc, prows, m->out, s)) != cudaSuccess) {
      return e;
    }
    k_u0<<<(int)std::min<long long>(4096, (rows + 255) / 256), 256, 0, s>>>(
        rows, mz, m->out, m->scale, prev_u ? prev_u + t0 * mz : nullptr, m->gate, u0 + t0 * mz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (launched) *launched += m->H == 256 ? 3 : 5;  // features, the network, starts
  }
  return cudaSuccess;
}
}  // namespace rlt2

#define CKM(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

extern "C" rlt2_status rlt2_mlp_create(int hidden, unsigned long long seed, void* stream, rlt2_mlp** out) {
  if (!out || hidden < 64 || hidden > 1024 || hidden % 64 != 0) {
    set_error("rlt2_mlp_create: hidden must be a multiple of 64 in [64, 1024]");
    return RLT2_EINVAL;
  }
  *out = nullptr;
  rlt2_mlp* m = new rlt2_mlp();
  m->H = hidden;
  m->stream = (cudaStream_t)stream;
  const int H = hidden;
  m->nparams = (long long)kInPad * H + H + (long long)H * H + H + H + 1;
  cudaError_t e;
  auto fail = [&](cudaError_t err) {
    rlt2_mlp_destroy(m);
    return cuda_fail(err, "rlt2_mlp_create");
  };
  if ((e = cudaMalloc((void**)&m->W1, sizeof(float) * m->nparams)) != cudaSuccess) return fail(e);
  param_ptrs(m);
  if ((e = cudaMalloc((void**)&m->mom, sizeof(float) * 2 * m->nparams)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->grad, sizeof(float) * m->nparams)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->W1b, sizeof(bf16) * kInPad * H)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->W2b, sizeof(bf16) * H * H)) != cudaSuccess) return fail(e);
  const size_t cr = kChunk + 64;
  if ((e = cudaMalloc((void**)&m->Xc, sizeof(bf16) * cr * kInPad)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->H1, sizeof(bf16) * cr * H)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->H2, sizeof(bf16) * cr * H)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->dH1, sizeof(bf16) * cr * H)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->dH2, sizeof(bf16) * cr * H)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->out, sizeof(float) * cr)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->tgt, sizeof(float) * cr)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->dout, sizeof(float) * cr)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->scale, sizeof(float) * cr)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->loss, sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&m->err, sizeof(int))) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(m->err, 0, sizeof(int), m->stream)) != cudaSuccess) return fail(e);
  cudaStream_t s = m->stream;
  // He initialisation of W1 (34 valid input rows) and W2, small w3, zero biases
  if ((e = cudaMemsetAsync(m->W1, 0, sizeof(float) * m->nparams, s)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(m->mom, 0, sizeof(float) * 2 * m->nparams, s)) != cudaSuccess) return fail(e);
  k_init_normal<<<256, 256, 0, s>>>(kInPad * H, kIn, H, sqrtf(2.0f / kIn), seed * 3 + 1, m->W1, m->W1b);
  k_init_normal<<<256, 256, 0, s>>>(H * H, H, H, sqrtf(2.0f / H), seed * 3 + 2, m->W2, m->W2b);
  k_init_normal<<<4, 256, 0, s>>>(H, 1, H, sqrtf(1.0f / H), seed * 3 + 3, m->w3, nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
  *out = m;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_destroy(rlt2_mlp* m) {
  if (!m) return RLT2_OK;
  if (m->stream) cudaStreamSynchronize(m->stream);
  void* ptrs[] = {m->W1, m->mom, m->grad, m->W1b, m->W2b, m->Xd, m->Td, m->Xc, m->H1, m->H2, m->dH1, m->dH2,
                  m->out, m->tgt, m->dout, m->scale, m->loss, m->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_get_weights(rlt2_mlp* m, float* W1, float* b1, float* W2, float* b2, float* w3,
                                            float* b3) {
  if (!m) return RLT2_EINVAL;
  const int H = m->H;
  std::vector<float> all(m->nparams);
  CKM(cudaMemcpyAsync(all.data(), m->W1, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->stream));
  CKM(cudaStreamSynchronize(m->stream));
  if (W1) memcpy(W1, all.data(), sizeof(float) * kIn * H);
  const float* p = all.data() + kInPad * H;
  if (b1) memcpy(b1, p, sizeof(float) * H);
  p += H;
  if (W2) memcpy(W2, p, sizeof(float) * H * H);
  p += (size_t)H * H;
  if (b2) memcpy(b2, p, sizeof(float) * H);
  p += H;
  if (w3) memcpy(w3, p, sizeof(float) * H);
  p += H;
  if (b3) *b3 = *p;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_set_weights(rlt2_mlp* m, const float* W1, const float* b1, const float* W2,
                                            const float* b2, const float* w3, const float* b3) {
  if (!m || !W1 || !b1 || !W2 || !b2 || !w3 || !b3) return RLT2_EINVAL;
  const int H = m->H;
  std::vector<float> all(m->nparams, 0.0f);
  memcpy(all.data(), W1, sizeof(float) * kIn * H);
  float* p = all.data() + kInPad * H;
  memcpy(p, b1, sizeof(float) * H);
  p += H;
  memcpy(p, W2, sizeof(float) * H * H);
  p += (size_t)H * H;
  memcpy(p, b2, sizeof(float) * H);
  p += H;
  memcpy(p, w3, sizeof(float) * H);
  p += H;
  *p = *b3;
  std::vector<bf16> w1b(kInPad * H), w2b((size_t)H * H);
  for (size_t i = 0; i < w1b.size(); ++i) w1b[i] = __float2bfloat16_rn(all[i]);
  for (size_t i = 0; i < w2b.size(); ++i) w2b[i] = __float2bfloat16_rn(W2[i]);
  CKM(cudaMemcpyAsync(m->W1, all.data(), sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->stream));
  CKM(cudaMemcpyAsync(m->W1b, w1b.data(), sizeof(bf16) * w1b.size(), cudaMemcpyHostToDevice, m->stream));
  CKM(cudaMemcpyAsync(m->W2b, w2b.data(), sizeof(bf16) * w2b.size(), cudaMemcpyHostToDevice, m->stream));
  CKM(cudaMemsetAsync(m->mom, 0, sizeof(float) * 2 * m->nparams, m->stream));
  m->adam_t = 0;
  CKM(cudaStreamSynchronize(m->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_add_samples(rlt2_mlp* m, long long ntiles, int mz, const double* tiles,
                                            const double* prev_u, const double* target_u) {
  if (!m || ntiles < 0 || mz < 1 || mz > 32 || (ntiles > 0 && (!tiles || !target_u))) {
    set_error("rlt2_mlp_add_samples: invalid argument");
    return RLT2_EINVAL;
  }
  if (ntiles == 0) return RLT2_OK;
  CKM(ensure_dataset(m, m->rows + ntiles * mz));
  float* scale = nullptr;
  CKM(cudaMalloc((void**)&scale, sizeof(float) * ntiles));
  k_features<<<(int)std::min<long long>(8192, (ntiles + 7) / 8), 256, 0, m->stream>>>(
      ntiles, mz, tiles, prev_u, target_u, m->Xd + m->rows * kInPad, m->Td + m->rows, scale);
  cudaError_t e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(m->stream);
  cudaFree(scale);
  if (e != cudaSuccess) return cuda_fail(e, "k_features");
  if (e2 != cudaSuccess) return cuda_fail(e2, "k_features sync");
  m->rows += ntiles * mz;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_samples(rlt2_mlp* m, long long* rows, void* X_bf16, float* targets) {
  if (!m) return RLT2_EINVAL;
  if (rows) *rows = m->rows;
  if (X_bf16 && m->rows)
    CKM(cudaMemcpyAsync(X_bf16, m->Xd, sizeof(bf16) * m->rows * kInPad, cudaMemcpyDeviceToHost, m->stream));
  if (targets && m->rows)
    CKM(cudaMemcpyAsync(targets, m->Td, sizeof(float) * m->rows, cudaMemcpyDeviceToHost, m->stream));
  CKM(cudaStreamSynchronize(m->stream));
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_clear_samples(rlt2_mlp* m) {
  if (!m) return RLT2_EINVAL;
  m->rows = 0;
  return RLT2_OK;
}

// ETIMEOUT (and the flag cleared) if a tensor-core wait of the network's kernels
// timed out since the flag was last cleared; the stream is synchronised.
static rlt2_status tc_wait_status(rlt2_mlp* m, const char* where) {
  int err = 0;
  CKM(cudaStreamSynchronize(m->stream));
  CKM(cudaMemcpy(&err, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!err) return RLT2_OK;
  CKM(cudaMemset(m->err, 0, sizeof(int)));
  set_error(std::string(where) + ": a tensor-core wait timed out");
  return RLT2_ETIMEOUT;
}

// loss and gradients on the first `rows` samples (<= one chunk), no update
extern "C" rlt2_status rlt2_mlp_grad(rlt2_mlp* m, long long rows, double* loss, float* gW1, float* gb1, float* gW2,
                                     float* gb2, float* gw3, float* gb3) {
  if (!m || rows < 1 || rows > m->rows || rows > kChunk) {
    set_error("rlt2_mlp_grad: rows must be in [1, min(samples, 262144)]");
    return RLT2_EINVAL;
  }
  const int H = m->H;
  cudaStream_t s = m->stream;
  const long long prows = (rows + 63) / 64 * 64;
  CKM(cudaMemcpyAsync(m->Xc, m->Xd, sizeof(bf16) * rows * kInPad, cudaMemcpyDeviceToDevice, s));
  if (prows > rows) CKM(cudaMemsetAsync(m->Xc + rows * kInPad, 0, sizeof(bf16) * (prows - rows) * kInPad, s));
  CKM(cudaMemcpyAsync(m->tgt, m->Td, sizeof(float) * rows, cudaMemcpyDeviceToDevice, s));
  CKM(cudaMemsetAsync(m->grad, 0, sizeof(float) * m->nparams, s));
  CKM(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
  CKM(backward(m, m->Xc, m->tgt, prows, rows, s));
  std::vector<float> g(m->nparams);
  double l = 0.0;
  CKM(cudaMemcpyAsync(g.data(), m->grad, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, s));
  CKM(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKM(cudaStreamSynchronize(s));
  if (rlt2_status ts = tc_wait_status(m, "rlt2_mlp_grad"); ts != RLT2_OK) return ts;
  if (loss) *loss = l;
  const float* p = g.data();
  if (gW1) memcpy(gW1, p, sizeof(float) * kIn * H);
  p += kInPad * H;
  if (gb1) memcpy(gb1, p, sizeof(float) * H);
  p += H;
  if (gW2) memcpy(gW2, p, sizeof(float) * H * H);
  p += (size_t)H * H;
  if (gb2) memcpy(gb2, p, sizeof(float) * H);
  p += H;
  if (gw3) memcpy(gw3, p, sizeof(float) * H);
  p += H;
  if (gb3) *gb3 = *p;
  return RLT2_OK;
}

// AdamW on minibatches drawn (counter-based hash) from the samples
extern "C" rlt2_status rlt2_mlp_fit(rlt2_mlp* m, int steps, int batch_rows, double lr, double weight_decay,
                                    unsigned long long seed, double* loss_hist) {
  if (!m || steps < 0 || batch_rows < 64 || batch_rows > kChunk || batch_rows % 64 != 0 || m->rows < 1) {
    set_error("rlt2_mlp_fit: need samples and batch_rows a multiple of 64 in [64, 262144]");
    return RLT2_EINVAL;
  }
  const int H = m->H;
  cudaStream_t s = m->stream;
  const float b1 = 0.9f, b2 = 0.999f;
  std::vector<double> losses(steps, 0.0);
  for (int st = 0; st < steps; ++st) {
    k_gather<<<4096, 256, 0, s>>>(batch_rows, m->rows, seed * 1000003ull + (unsigned long long)st * 7919ull, m->Xd,
                                  m->Td, m->Xc, m->tgt);
    CKM(cudaGetLastError());
    CKM(cudaMemsetAsync(m->grad, 0, sizeof(float) * m->nparams, s));
    CKM(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
    CKM(backward(m, m->Xc, m->tgt, batch_rows, batch_rows, s));
    ++m->adam_t;
    const float c1 = 1.0f - powf(b1, (float)m->adam_t), c2 = 1.0f - powf(b2, (float)m->adam_t);
    // W1 and W2 are refreshed in BF16; the padded rows of W1 keep zero gradient
    k_adamw<<<256, 256, 0, s>>>(kInPad * H, m->W1, m->mom, m->mom + m->nparams, m->grad, (float)lr, b1, b2, 1e-8f,
                                (float)weight_decay, c1, c2, m->W1b);
    const long long o2 = (long long)kInPad * H + H;
    k_adamw<<<256, 256, 0, s>>>(H, m->b1, m->mom + kInPad * H, m->mom + m->nparams + kInPad * H,
                                m->grad + kInPad * H, (float)lr, b1, b2, 1e-8f, 0.0f, c1, c2, nullptr);
    k_adamw<<<256, 256, 0, s>>>(H * H, m->W2, m->mom + o2, m->mom + m->nparams + o2, m->grad + o2, (float)lr, b1, b2,
                                1e-8f, (float)weight_decay, c1, c2, m->W2b);
    const long long o3 = o2 + (long long)H * H;
    k_adamw<<<8, 256, 0, s>>>(2 * H + 1, m->b2, m->mom + o3, m->mom + m->nparams + o3, m->grad + o3, (float)lr, b1,
                              b2, 1e-8f, 0.0f, c1, c2, nullptr);
    CKM(cudaGetLastError());
    if (loss_hist) CKM(cudaMemcpyAsync(&losses[st], m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CKM(cudaStreamSynchronize(s));
  if (rlt2_status ts = tc_wait_status(m, "rlt2_mlp_fit"); ts != RLT2_OK) return ts;
  if (loss_hist)
    for (int st = 0; st < steps; ++st) loss_hist[st] = losses[st];
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_set_gate(rlt2_mlp* m, double gate) {
  if (!m || !(gate >= 0.0)) return RLT2_EINVAL;
  m->gate = (float)gate;
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_check_wait_timeout(rlt2_mlp* m) {
  if (!m || m->H != 256) {
    set_error("rlt2_mlp_check_wait_timeout: needs a network with H = 256");
    return RLT2_EINVAL;
  }
  CKM(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
  CKM(cudaMemsetAsync(m->Xc, 0, sizeof(bf16) * 128 * kInPad, m->stream));
  CKM(umma_mlp_forward(m->Xc, 128, m->W1b, m->b1, m->W2b, m->b2, m->w3, m->b3, m->out, m->err, m->stream, true));
  CKM(cudaStreamSynchronize(m->stream));
  int err = 0;
  CKM(cudaMemcpy(&err, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  CKM(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
  CKM(cudaStreamSynchronize(m->stream));
  if (err) {
    set_error("rlt2_mlp_check_wait_timeout: the inference kernel's wait ran out (expected)");
    return RLT2_ETIMEOUT;
  }
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_check_gemm_wait_timeout(rlt2_mlp* m) {
  if (!m || m->H != 256) {
    set_error("rlt2_mlp_check_gemm_wait_timeout: needs a network with H = 256");
    return RLT2_EINVAL;
  }
  // the second forward layer's product on 1,024 zero rows (eight 128-row tiles,
  // four K chunks each) with the MMAs withheld
  constexpr int kRows = 1024;
  const int H = m->H;
  CKM(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
  CKM(cudaMemsetAsync(m->H1, 0, sizeof(bf16) * kRows * H, m->stream));
  UmmaGemmArgs u{};
  u.M = kRows;
  u.N = H;
  u.K = H;
  u.A = m->H1;
  u.lda = H;
  u.a_kmajor = true;
  u.B = m->W2b;
  u.ldb = H;
  u.b_kmajor = false;
  u.epi = 1;
  u.Cb = m->H2;
  u.ldc = H;
  u.bias = m->b2;
  u.err = m->err;
  u.withhold = 1;
  CKM(umma_gemm(u, 1, m->stream));
  CKM(cudaStreamSynchronize(m->stream));
  int err = 0;
  CKM(cudaMemcpy(&err, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  CKM(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
  CKM(cudaStreamSynchronize(m->stream));
  if (err) {
    set_error("rlt2_mlp_check_gemm_wait_timeout: the training GEMM's waits ran out (expected)");
    return RLT2_ETIMEOUT;
  }
  return RLT2_OK;
}

extern "C" rlt2_status rlt2_mlp_predict(rlt2_mlp* m, long long ntiles, int mz, const double* tiles,
                                        const double* prev_u, double* u0) {
  if (!m || ntiles < 0 || mz < 1 || mz > 32 || (ntiles > 0 && (!tiles || !u0))) {
    set_error("rlt2_mlp_predict: invalid argument");
    return RLT2_EINVAL;
  }
  CKM(mlp_predict_enqueue(m, ntiles, mz, tiles, prev_u, u0, m->stream));
  CKM(cudaStreamSynchronize(m->stream));
  int err = 0;
  CKM(cudaMemcpy(&err, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    set_error("rlt2_mlp_predict: a tensor-core wait timed out");
    return RLT2_ETIMEOUT;
  }
  return RLT2_OK;
}
