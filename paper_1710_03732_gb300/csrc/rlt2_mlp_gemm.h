// The tcgen05 GEMM of the learned start's training (umma_gemm.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rlt2 {

// C[M x N] = A[M x K] B[K x N], BF16 operands, FP32 accumulation on tcgen05.
struct UmmaGemmArgs {
  int M, N, K;               // N <= 256 and a multiple of 8; K a multiple of 64
  const __nv_bfloat16* A;    // a_kmajor: A(m, k) at A[m * lda + k]; else at A[k * lda + m]
  int lda;
  bool a_kmajor;
  const __nv_bfloat16* B;    // b_kmajor: B(k, n) at B[n * ldb + k]; else at B[k * ldb + n]
  int ldb;
  bool b_kmajor;
  int epi;                   // 0: FP32 C (atomic add when K is split), 1: bias + ReLU -> BF16 Cb,
                             // 2: masked by mask > 0 -> BF16 Cb (C, Cb, mask: leading dimension ldc)
  float* C;
  int ldc;
  __nv_bfloat16* Cb;
  const float* bias;
  const __nv_bfloat16* mask;
  int* err;                  // set on a timed-out wait
  int kps;                   // K per split (set by umma_gemm)
  unsigned tmem_cols;        // TMEM columns allocated (set by umma_gemm)
  int withhold;              // diagnostics (tall products): issue no MMA and no commit, so that
                             // the bounded waits run out (failure detection without a fault)
};

// Shapes the kernel takes (the caller falls back to the mma.sync GEMM otherwise).
bool umma_gemm_supported(int M, int N, int K);
// Launches the GEMM with K split `splits` ways (grid.z); EPI 0 adds atomically when split.
cudaError_t umma_gemm(UmmaGemmArgs a, int splits, cudaStream_t s);

}  // namespace rlt2
