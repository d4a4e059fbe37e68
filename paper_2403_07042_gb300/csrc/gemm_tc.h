// tcgen05 GEMM for the split-precision increment products.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace qed {

// Operands are FP16, K-major, stored as [planes][rows][K] (the pieces of an FP64 value:
// hi, then lo, or hi, mid, lo).  The kernel computes
//   C[M x N] = sum over segments s of A_{pa(s)} B_{pb(s)}^T
// as one K loop over the segments (e.g. hi*hi + hi*lo + lo*hi), accumulating in FP32 in
// tensor memory, and writes split-K partial sums out[split][M][N] (FP32).
constexpr int kTcMaxSeg = 6;

struct TcGemm {
    CUtensorMap a;      // dims (K, M, planes_a), box (64, 128, 1), 128-byte swizzle
    CUtensorMap b;      // dims (K, N, planes_b), box (64, BN, 1)
    int M = 0, N = 0, K = 0;
    int nseg = 0;
    int seg_a[kTcMaxSeg] = {}, seg_b[kTcMaxSeg] = {};
    int splits = 1;
    int kb_per_split = 0;
};

constexpr int kTcBM = 128;
constexpr int kTcBN = 128;
constexpr int kTcBK = 64;
constexpr int kTcStages = 6;

// Encodes the two tensor maps and picks the split-K factor for `num_sms`.
// Returns false (with an error message set) if the driver entry point is unavailable.
bool tc_gemm_plan(TcGemm &g, const void *a_planes, int planes_a, const void *b_planes, int planes_b, int M, int N,
                  int K, int nseg, const int *seg_pairs, int num_sms, int force_splits = 0);

// Launch on `s`; `err` receives kErrTimeout if a bounded wait ran out.
void tc_gemm_launch(const TcGemm &g, float *out, uint32_t *err, cudaStream_t s);

// Grouped form: many independent products (instances of a batch) in one launch.  Each
// work item is one 128 x 128 tile of one split-K slice of one job; all jobs of a launch
// share the plane-segment list.
struct GemmJob {
    const CUtensorMap *map_a;  // device address of the job's A tensor map (64-byte aligned)
    const CUtensorMap *map_b;
    float *out;                // [splits][M][N]
    int M, N, kb_per_seg, kb_per_split;
};

struct GemmItem {
    int job, tile_m, tile_n, split;
};

struct TcSegs {
    int nseg;
    int a[kTcMaxSeg], b[kTcMaxSeg];
};

bool tc_gemm_prepare_grouped();
void tc_gemm_grouped_launch(const GemmItem *items, int n_items, const GemmJob *jobs, const TcSegs &segs,
                            uint32_t *err, cudaStream_t s);

size_t tc_gemm_smem_bytes();

}  // namespace qed
