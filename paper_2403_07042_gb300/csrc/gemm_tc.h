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
// accumulating in FP32 in tensor memory: either as one K loop over the segments (e.g.
// hi*hi + hi*lo + lo*hi), writing split-K partial sums out[split][M][N] (kEpiPlain), or, for
// the step's products, with every plane of a 64-wide k-block loaded once and all segment
// products issued on it, the split-K slices summed inside a cluster (kEpiW / kEpiV).
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
// The planner splits K into at most this many slices (a cluster of that many CTAs sums
// them on chip); qed_autotune may also try 8 for the first product.
constexpr int kTcMaxAutoSplits = 4;
// Tile widths: 128 x 256 x 16 instructions run near the SM's tensor peak, 128 x 128 x 16 at
// about half, but small products need the narrower tiles to spread over the SMs.
constexpr int kTcBNMax = 256;
constexpr int kTcBK = 64;
__host__ __device__ constexpr int tc_stages(int bn) { return bn == 128 ? 6 : 4; }

// Encodes the two tensor maps and picks the split-K factor for `num_sms`.
// Returns false (with an error message set) if the driver entry point is unavailable.
bool tc_gemm_plan(TcGemm &g, const void *a_planes, int planes_a, const void *b_planes, int planes_b, int M, int N,
                  int K, int nseg, const int *seg_pairs, int num_sms, int force_splits = 0, int force_bn = 0,
                  bool merged = false);

// Launch on `s`; `err` receives kErrTimeout if a bounded wait ran out.  Returns the
// status of the launch itself (a launch-configuration error is reported here, not later).
cudaError_t tc_gemm_launch(const TcGemm &g, float *out, uint32_t *err, cudaStream_t s);

// Epilogues.
//   kEpiPlain: the FP32 tile goes into its split-K slice of `out` (the caller sums slices).
//   kEpiW (GEMM1 of the step, output [W_re; W_im], 2Dp x Dp): the split-K slices of a tile
//     are one thread-block cluster; their partial tiles are summed through distributed
//     shared memory (fixed order) and each CTA of the cluster writes its share of rows: W
//     (FP32 [2][Dp][Dp], scaled by inv) and the FP16 hi/lo planes of GEMM2's A operand
//     (rows k = [W_re | W_im], scaled by s_w).
//   kEpiV (GEMM2): B's rows are ordered so that every 128 rows hold [X_re | X_im] of 64
//     complex columns (64g..64g+63 for the g-th 128 rows); a tile covers one such group
//     (128-wide) or two (256-wide).  Only tiles on or above the diagonal are launched (X and
//     V are Hermitian).  After the same cluster reduction each
//     CTA forms, for its rows m and the tile's columns n >= m,
//       V_mn = P_m conj(P_n) (rho_mn + W_mn + conj(W_nm) + inv X_mn)
//     in double-float (U rho U^+ in the increment form) and writes V_mn and V_nm = conj(V_mn).
enum { kEpiPlain = 0, kEpiW = 1, kEpiV = 2 };

// Cluster sizes (split-K slices reduced on chip) the epilogues accept: kEpiW 1, 2, 4 or 8;
// kEpiV 1, 2 or 4.
constexpr int kTcMaxCluster = 8;
constexpr int kTcMaxClusterV = 4;

struct TcEpilogue {
    int64_t D = 0, Dp = 0;
    float inv = 1.f;              // kEpiW: 1 / (s_Delta s_rho) -> W;  kEpiV: 1 / (s_W s_Delta) -> X
    float s_w = 1.f;              // kEpiW: scale of the W planes
    float *w32 = nullptr;         // W, FP32 [2][Dp][Dp] (written by kEpiW, read by kEpiV)
    __half *w_pl = nullptr;       // kEpiW: W planes [2][Dp][2Dp]
    const float4 *rho = nullptr;  // kEpiV: double-float state, D x D
    const float4 *phase = nullptr;  // kEpiV: P_k as double-float complex
    float4 *V = nullptr;          // kEpiV: output, D x D double-float complex
};

// Grouped form: many independent products (instances of a batch) in one launch.  Each
// work item is one output tile of one split-K slice of one job; all jobs of a launch share
// the plane-segment list, the tile width and the cluster size.
struct GemmJob {
    const CUtensorMap *map_a;  // device address of the job's A tensor map (64-byte aligned)
    const CUtensorMap *map_b;
    float *out;                // [splits][M][N]: kEpiPlain writes slice `split` of its item
    int M, N, kb_per_seg, kb_per_split;
    int tx_bytes;              // bytes one stage receives (A tile + B box)
    int mode;                  // kEpiPlain, kEpiW or kEpiV
    const uint32_t *gate;      // test hook (qed_set_wait_gate): wait for *gate == 0, or null
    long long gate_budget;     // cycles that wait may take before the CTA gives up
    TcEpilogue epi;
};

// One work item; the items of one tile are consecutive with split = 0..cluster-1 (for the
// cluster epilogues, split is the CTA's rank in its cluster).
struct GemmItem {
    int job, tile_m, tile_n, split;
};

struct TcSegs {
    int nseg;
    int a[kTcMaxSeg], b[kTcMaxSeg];
};

bool tc_gemm_prepare_grouped();
// All jobs of one launch share the epilogue mode (kEpiW or kEpiV), the tile width bn (128
// or 256) and the cluster size (equal to the jobs' splits).  Returns the
// launch status.
cudaError_t tc_gemm_grouped_launch(const GemmItem *items, int n_items, const GemmJob *jobs, const TcSegs &segs,
                                   int bn, int mode, int cluster, uint32_t *err, cudaStream_t s);

// One model's product (kEpiW or kEpiV) with its tensor maps and job passed as kernel
// parameters (nothing read from tables before the first TMA load).  The work items are the
// same as the grouped form's for that model: kEpiW skips the tiles that lie wholly in the
// zero padding (rows of a plane or columns >= D), kEpiV runs the tiles on or above the
// diagonal (128 rows x 64 or 128 complex columns), each as g.splits consecutive CTAs (a
// cluster).
cudaError_t tc_gemm_single_launch(const TcGemm &g, const GemmJob &job, const TcSegs &segs, int64_t D,
                                  uint32_t *err, cudaStream_t s);
// Bytes one pipeline stage of a product in `mode` receives (kEpiW / kEpiV stages hold every
// plane of both operands for one 64-wide k-block).
int tc_stage_tx_bytes(const TcGemm &g, int mode);
// Number of CTAs tc_gemm_single_launch starts for that product.
int tc_gemm_single_ctas(const TcGemm &g, int mode, int64_t D);

size_t tc_gemm_smem_bytes(int bn);

}  // namespace qed
