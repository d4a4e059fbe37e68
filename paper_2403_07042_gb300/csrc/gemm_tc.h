// tcgen05 GEMM for the split-precision increment products.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace qed {

// Operands are FP16, K-major, stored as [2 planes (hi, lo)][rows][K].  The kernel computes
//   C[M x N] = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// as one K loop over three segments (the lo*lo product is dropped), accumulating in FP32
// in tensor memory, and writes split-K partial sums out[split][M][N] (FP32).
struct TcGemm {
    CUtensorMap a;      // dims (K, M, 2), box (64, 128, 1), 128-byte swizzle
    CUtensorMap b;      // dims (K, N, 2), box (64, BN, 1)
    int M = 0, N = 0, K = 0;
    int splits = 1;
    int kb_per_split = 0;
};

constexpr int kTcBM = 128;
constexpr int kTcBN = 128;
constexpr int kTcBK = 64;
constexpr int kTcStages = 6;

// Encodes the two tensor maps and picks the split-K factor for `num_sms`.
// Returns false (with an error message set) if the driver entry point is unavailable.
bool tc_gemm_plan(TcGemm &g, const void *a_planes, const void *b_planes, int M, int N, int K, int num_sms,
                  int force_splits = 0);

// Launch on `s`; `err` receives kErrTimeout if a bounded wait ran out.
void tc_gemm_launch(const TcGemm &g, float *out, uint32_t *err, cudaStream_t s);

size_t tc_gemm_smem_bytes();

}  // namespace qed
