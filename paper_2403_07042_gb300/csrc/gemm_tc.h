// tcgen05 GEMM for the split-precision increment products.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
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
    CUtensorMap b;      // dims (K, N, planes_b), box (64, BN, 1); rows past N read as zeros
    int M = 0, N = 0, K = 0;
    int nseg = 0;
    int seg_a[kTcMaxSeg] = {}, seg_b[kTcMaxSeg] = {};
    int splits = 1;
    int kb_per_split = 0;
    int bn = 256;        // tile width: 128 or 256
    int b_box_rows = 0;  // min(bn, N): rows of B one stage loads
};

constexpr int kTcBM = 128;
// The planner splits K into at most this many slices (the element-wise kernels that sum
// the slices of the step's products hold that many loads in flight).
constexpr int kTcMaxAutoSplits = 4;
// Tile widths: 128 x 256 x 16 instructions run near the SM's tensor peak, 128 x 128 x 16 at
// about half, but small products need the narrower tiles to spread over the SMs.
constexpr int kTcBNMax = 256;
constexpr int kTcBK = 64;
__host__ __device__ constexpr int tc_stages(int bn) { return bn == 128 ? 6 : 4; }

// Encodes the two tensor maps and picks the split-K factor for `num_sms`.
// Returns false (with an error message set) if the driver entry point is unavailable.
bool tc_gemm_plan(TcGemm &g, const void *a_planes, int planes_a, const void *b_planes, int planes_b, int M, int N,
                  int K, int nseg, const int *seg_pairs, int num_sms, int force_splits = 0, int force_bn = 0);

// Launch on `s`; `err` receives kErrTimeout if a bounded wait ran out.  Returns the
// status of the launch itself (a launch-configuration error is reported here, not later).
cudaError_t tc_gemm_launch(const TcGemm &g, float *out, uint32_t *err, cudaStream_t s);

// Epilogues: kEpiPlain stores the FP32 tile into its split-K slice; kEpiW (for unsplit
// products) treats the output as GEMM1's [W_re; W_im]
// (2Dp x Dp) and writes W, W^T (FP32 [2][Dp][Dp], scaled by inv_w) and the FP16 hi/lo
// planes of GEMM2's A operand (rows k = [W_re | W_im], scaled by s_w).
enum { kEpiPlain = 0, kEpiW = 1 };

struct TcEpilogueW {
    int64_t Dp = 0;
    float inv_w = 1.f, s_w = 1.f;
    float *w32 = nullptr, *wt32 = nullptr;
    __half *w_pl = nullptr;
};

// Grouped form: many independent products (instances of a batch) in one launch.  Each
// work item is one 128 x 128 tile of one split-K slice of one job; all jobs of a launch
// share the plane-segment list.
struct GemmJob {
    const CUtensorMap *map_a;  // device address of the job's A tensor map (64-byte aligned)
    const CUtensorMap *map_b;
    float *out;                // [splits][M][N]: kEpiPlain writes slice `split` of its item
    int M, N, kb_per_seg, kb_per_split;
    int tx_bytes;              // bytes one stage receives (A tile + B box)
    int mode;                  // kEpiPlain or kEpiW
    TcEpilogueW w;
};

struct GemmItem {
    int job, tile_m, tile_n, split;
};

struct TcSegs {
    int nseg;
    int a[kTcMaxSeg], b[kTcMaxSeg];
};

bool tc_gemm_prepare_grouped();
// All jobs of one launch share the tile width bn (128 or 256).
void tc_gemm_grouped_launch(const GemmItem *items, int n_items, const GemmJob *jobs, const TcSegs &segs, int bn,
                            uint32_t *err, cudaStream_t s);

size_t tc_gemm_smem_bytes(int bn);

}  // namespace qed
