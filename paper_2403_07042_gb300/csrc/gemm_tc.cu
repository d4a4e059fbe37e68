// tcgen05 / TMA / mbarrier GEMM for sm_103a (Blackwell): the dense products of the
// "unitary evolution" stage (Sec. 4.2, Table 3) in split precision.
//
// One CTA computes one 128 x 256 FP32 tile of one split-K slice:
//   warp 0, one lane : TMA producer, 4-stage ring of (A 128x64, B 256x64) FP16 tiles of the
//                      current segment's planes (a last tile of 128 columns reads zeros),
//                      128-byte swizzled, completion tracked by mbarrier transaction bytes
//   warp 1, one lane : MMA issuer, tcgen05.mma.cta_group::1.kind::f16 (M=128, N=256, K=16)
//                      into a TMEM accumulator; tcgen05.commit frees each smem stage
//   warps 0-3        : epilogue, tcgen05.ld 32x32b (thread = accumulator row), transposed
//                      through shared memory so that each store writes 128 contiguous bytes
// Every wait is bounded by a clock budget; on expiry the kernel records kErrTimeout,
// stops issuing work, waits (bounded) for what it issued, frees TMEM and returns.
#include <cstdio>
#include <cstring>
#include <string>

#include <cuda_fp16.h>

#include "gemm_tc.h"
#include "pdl.h"
#include "kernels.h"
#include "model.h"

namespace qed {

namespace {

constexpr uint32_t kStageA = kTcBM * kTcBK * 2;  // bytes
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored with the 128-byte swizzle:
// rows of 128 bytes, 8-row core groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4)                      // D format F32
           | (0u << 7) | (0u << 10)       // A, B format F16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct Params {
    int M, N;
    int kb_per_seg;
    int kb_total;
    int kb_per_split;
    uint32_t seg_a, seg_b;  // plane of segment q in bits 3q..3q+2 (kept in registers)
    int tx_bytes;
    int mode;   // epilogue: kEpiPlain (slice split of out) or kEpiW (unsplit products only)
    float *out;
    uint32_t *err;
    TcEpilogueW w;
};

// One 128 x 128 output tile of one split-K slice (the body shared by the single and the
// grouped kernel).  tmA / tmB are generic addresses of tensor maps in parameter or global
// memory.
template <int BN>
__device__ __forceinline__ void gemm_tile(const CUtensorMap *tmA, const CUtensorMap *tmB, const Params &p,
                                          int tile_m, int tile_n, int split) {
    constexpr int kTcBN = BN;
    constexpr int kTcStages = tc_stages(BN);
    constexpr uint32_t kStageB = BN * kTcBK * 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + kTcStages * kStageA;
    uint64_t *bars = (uint64_t *)(sB + kTcStages * kStageB);  // full[S], empty[S], accum
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * kTcStages + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;    // TMA stage loads issued by the producer
    volatile int *consumed = abort_flag + 2;  // stage loads the MMA issuer has waited for

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb0 = split * p.kb_per_split;
    const int nkb = min(p.kb_per_split, p.kb_total - kb0);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kTcStages),
                   accum = smem_u32(bars + 2 * kTcStages);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        *issued = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tmB) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // operands and outputs are shared with the neighbouring kernels of the step
    pdl_wait();
    pdl_trigger();

    if (warp == 0 && lane == 0) {
        // producer
        for (int i = 0; i < nkb; ++i) {
            const int s = i % kTcStages;
            const uint32_t par = ((i / kTcStages) & 1) ^ 1;
            if (!mbar_wait(empty0 + 8 * s, par, kWaitCycles)) {
                *abort_flag = 1;
                atomicOr(p.err, kErrTimeout);
                break;
            }
            if (*abort_flag) break;
            const int kb = kb0 + i;
            const int seg = kb / p.kb_per_seg, kk = kb % p.kb_per_seg;
            const uint32_t bar = full0 + 8 * s;
            mbar_expect_tx(bar, (uint32_t)p.tx_bytes);
            tma_load_3d(smem_u32(sA + s * kStageA), tmA, kk * kTcBK, tile_m * kTcBM, (p.seg_a >> (3 * seg)) & 7, bar);
            tma_load_3d(smem_u32(sB + s * kStageB), tmB, kk * kTcBK, tile_n * kTcBN, (p.seg_b >> (3 * seg)) & 7, bar);
            *issued = i + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_f16(kTcBM, kTcBN);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % kTcStages;
            const uint32_t par = (i / kTcStages) & 1;
            const long long budget = *abort_flag ? 2000000LL : kWaitCycles;
            if (!mbar_wait(full0 + 8 * s, par, budget)) {
                *abort_flag = 1;
                atomicOr(p.err, kErrTimeout);
                break;
            }
            *consumed = i + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!*abort_flag) {
                const uint64_t ad = smem_desc_sw128(smem_u32(sA + s * kStageA));
                const uint64_t bd = smem_desc_sw128(smem_u32(sB + s * kStageB));
#pragma unroll
                for (int k = 0; k < kTcBK / 16; ++k)  // 16 FP16 = 32 bytes per step along K
                    mma_f16(tmem, ad + 2 * k, bd + 2 * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(accum);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // epilogue
    const bool ready = mbar_wait(accum, 0, kWaitCycles);
    if (!ready && lane == 0) atomicOr(p.err, kErrTimeout);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, ready && !*abort_flag);
    // register copies: the epilogue's global stores must not force reloads of p
    const int mode = p.mode, pN = p.N;
    float *const out = p.out + (int64_t)split * p.M * pN;  // this split-K slice
    const int64_t Dp = p.w.Dp;
    const float inv_w = p.w.inv_w, s_w = p.w.s_w;
    float *const w32 = p.w.w32;
    float *const wt32 = p.w.wt32;
    __half *const w_pl = p.w.w_pl;
    const int col0 = tile_n * BN;
    const int ncols = min(BN, pN - col0);
    const uint32_t tm_row = tmem + ((uint32_t)(warp * 32) << 16);
    const int64_t R0 = (int64_t)tile_m * kTcBM + warp * 32;  // output row of lane 0
    // the stage buffers are free once every MMA of the CTA has completed
    float *tbuf = (float *)sA + warp * (32 * 36);  // per-warp [32][36] transpose tile
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < ncols; c += 32) {
            float v[32];
            tmem_ld32(tm_row + (uint32_t)c, v);
            if (mode == kEpiW) {
                // W^T straight from the rows: lanes hold consecutive k of one column
                const int64_t R = R0 + lane;
                const int64_t plane = R / Dp, k = R % Dp;
                float *dst = wt32 + plane * Dp * Dp + (int64_t)(col0 + c) * Dp + k;
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[(int64_t)j * Dp] = v[j] * inv_w;
            }
            // transpose through shared memory: row-major 16-byte pieces, 4 rows per store
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *(float4 *)(tbuf + lane * 36 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            __syncwarp();
            const int sub = lane >> 3, col4 = 4 * (lane & 7);
            if (mode == kEpiW) {
                const int64_t plane = R0 / Dp;  // every row of a tile lies in one plane
                const int64_t k0 = R0 % Dp, L = col0 + c + col4;
                const int64_t lo_off = Dp * 2 * Dp;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int r = 4 * it + sub;
                    float4 x = *(const float4 *)(tbuf + r * 36 + col4);
                    x.x *= inv_w;
                    x.y *= inv_w;
                    x.z *= inv_w;
                    x.w *= inv_w;
                    *(float4 *)(w32 + plane * Dp * Dp + (k0 + r) * Dp + L) = x;
                    const float a0 = x.x * s_w, a1 = x.y * s_w, a2 = x.z * s_w, a3 = x.w * s_w;
                    const __half h0 = __float2half_rn(a0), h1 = __float2half_rn(a1), h2 = __float2half_rn(a2),
                                 h3 = __float2half_rn(a3);
                    __half2 hi[2] = {__halves2half2(h0, h1), __halves2half2(h2, h3)};
                    __half2 lo[2] = {
                        __halves2half2(__float2half_rn(a0 - __half2float(h0)), __float2half_rn(a1 - __half2float(h1))),
                        __halves2half2(__float2half_rn(a2 - __half2float(h2)), __float2half_rn(a3 - __half2float(h3)))};
                    __half *hp = w_pl + (k0 + r) * 2 * Dp + plane * Dp + L;
                    *(uint2 *)hp = *(const uint2 *)hi;
                    *(uint2 *)(hp + lo_off) = *(const uint2 *)lo;
                }
            } else {
                float *op = out + (R0 * pN) + col0 + c + col4;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int r = 4 * it + sub;
                    *(float4 *)(op + (int64_t)r * pN) = *(const float4 *)(tbuf + r * 36 + col4);
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        // drain: wait (bounded) for stage loads that were issued but never consumed
        for (int j = *consumed; j < *issued; ++j)
            mbar_wait(full0 + 8 * (j % kTcStages), (j / kTcStages) & 1, 20000000LL);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcBN) : "memory");
    }
}

template <int BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, Params p) {
    gemm_tile<BN>(&tmA, &tmB, p, blockIdx.y, blockIdx.x, blockIdx.z);
}

// Grouped launch: CTA b computes work item items[b] of job items[b].job (one instance of
// a batch), with that job's tensor maps read from global memory.
template <int BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_grouped_kernel(const GemmItem *__restrict__ items,
                                                                 const GemmJob *__restrict__ jobs, TcSegs segs,
                                                                 uint32_t *err) {
    const GemmItem it = items[blockIdx.x];
    const GemmJob jb = jobs[it.job];
    Params p;
    p.M = jb.M;
    p.N = jb.N;
    p.kb_per_seg = jb.kb_per_seg;
    p.kb_total = segs.nseg * jb.kb_per_seg;
    p.kb_per_split = jb.kb_per_split;
    p.tx_bytes = jb.tx_bytes;
    p.mode = jb.mode;
    p.w = jb.w;
    p.seg_a = 0;
    p.seg_b = 0;
#pragma unroll
    for (int q = 0; q < kTcMaxSeg; ++q) {
        p.seg_a |= (uint32_t)segs.a[q] << (3 * q);
        p.seg_b |= (uint32_t)segs.b[q] << (3 * q);
    }
    p.out = jb.out;
    p.err = err;
    gemm_tile<BN>(jb.map_a, jb.map_b, p, it.tile_m, it.tile_n, it.split);
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
        cudaGetLastError();
    }
    return fn;
}

bool encode(CUtensorMap *map, const void *base, int K, int rows, int planes, int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)K * 2 * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return false;
    }
    return true;
}

}  // namespace

constexpr size_t stage_bytes(int bn) { return (size_t)tc_stages(bn) * (kStageA + (size_t)bn * kTcBK * 2); }
static_assert((size_t)4 * 32 * 36 * 4 <= stage_bytes(128), "epilogue tiles must fit in the stage buffers");

size_t tc_gemm_smem_bytes(int bn) { return 1024 + stage_bytes(bn) + (2 * tc_stages(bn) + 1) * 8 + 32; }

template <class F>
bool set_smem(F kernel, int bn) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_gemm_smem_bytes(bn)) !=
        cudaSuccess) {
        cudaGetLastError();
        set_error("cudaFuncSetAttribute(max dynamic smem) failed for the tcgen05 GEMM");
        return false;
    }
    return true;
}

bool tc_gemm_plan(TcGemm &g, const void *a_planes, int planes_a, const void *b_planes, int planes_b, int M, int N,
                  int K, int nseg, const int *seg_pairs, int num_sms, int force_splits, int force_bn) {
    if (M % kTcBM || N % 128 || K % kTcBK || ((uintptr_t)a_planes & 15) || ((uintptr_t)b_planes & 15)) {
        set_error("tc_gemm: M and N must be multiples of 128, K of 64, planes 16-byte aligned");
        return false;
    }
    if (nseg < 1 || nseg > kTcMaxSeg || planes_a < 1 || planes_b < 1) {
        set_error("tc_gemm: 1..6 segments and at least one plane per operand");
        return false;
    }
    for (int q = 0; q < nseg; ++q) {
        if (seg_pairs[2 * q] < 0 || seg_pairs[2 * q] >= planes_a || seg_pairs[2 * q + 1] < 0 ||
            seg_pairs[2 * q + 1] >= planes_b) {
            set_error("tc_gemm: segment plane index out of range");
            return false;
        }
        g.seg_a[q] = seg_pairs[2 * q];
        g.seg_b[q] = seg_pairs[2 * q + 1];
    }
    g.nseg = nseg;
    g.M = M;
    g.N = N;
    g.K = K;
    // wide tiles once they alone fill half the SMs, narrow ones below that
    g.bn = force_bn ? force_bn : ((M / kTcBM) * ((N + 255) / 256) * 2 >= num_sms ? 256 : 128);
    g.b_box_rows = N < g.bn ? N : g.bn;
    if (!encode(&g.a, a_planes, K, M, planes_a, kTcBM) || !encode(&g.b, b_planes, K, N, planes_b, g.b_box_rows))
        return false;
    const int tiles = (M / kTcBM) * ((N + g.bn - 1) / g.bn);
    const int kb_total = nseg * (K / kTcBK);
    // split-K slices (a power of two <= 4) while the tiles fill fewer
    // than half the SMs and each slice keeps at least 4 k-blocks
    int splits = 1;
    while (splits < kTcMaxAutoSplits && tiles * splits * 2 <= num_sms && kb_total / (splits * 2) >= 4) splits *= 2;
    if (force_splits > 0) splits = force_splits > kb_total ? kb_total : force_splits;
    g.kb_per_split = (kb_total + splits - 1) / splits;
    g.splits = (kb_total + g.kb_per_split - 1) / g.kb_per_split;
    static bool attr_set = false;
    if (!attr_set) {
        if (!set_smem(tc_gemm_kernel<128>, 128) || !set_smem(tc_gemm_kernel<256>, 256)) return false;
        attr_set = true;
    }
    return true;
}

template <int BN>
void grouped_launch(const GemmItem *items, int n_items, const GemmJob *jobs, const TcSegs &segs, uint32_t *err,
                    cudaStream_t s) {
    launch_pdl(tc_gemm_grouped_kernel<BN>, dim3(n_items), dim3(128), tc_gemm_smem_bytes(BN), s, items, jobs, segs,
               err);
}

void tc_gemm_grouped_launch(const GemmItem *items, int n_items, const GemmJob *jobs, const TcSegs &segs, int bn,
                            uint32_t *err, cudaStream_t s) {
    if (n_items <= 0) return;
    count_launches(1);
    if (bn == 128)
        grouped_launch<128>(items, n_items, jobs, segs, err, s);
    else
        grouped_launch<256>(items, n_items, jobs, segs, err, s);
}

bool tc_gemm_prepare_grouped() {
    static bool done = false;
    if (done) return true;
    if (!set_smem(tc_gemm_grouped_kernel<128>, 128) || !set_smem(tc_gemm_grouped_kernel<256>, 256)) return false;
    done = true;
    return true;
}

cudaError_t tc_gemm_launch(const TcGemm &g, float *out, uint32_t *err, cudaStream_t s) {
    Params p;
    p.M = g.M;
    p.N = g.N;
    p.kb_per_seg = g.K / kTcBK;
    p.kb_total = g.nseg * p.kb_per_seg;
    p.seg_a = 0;
    p.seg_b = 0;
    for (int q = 0; q < g.nseg; ++q) {
        p.seg_a |= (uint32_t)g.seg_a[q] << (3 * q);
        p.seg_b |= (uint32_t)g.seg_b[q] << (3 * q);
    }
    p.kb_per_split = g.kb_per_split;
    p.tx_bytes = (int)kStageA + g.b_box_rows * kTcBK * 2;
    p.mode = kEpiPlain;
    p.w = TcEpilogueW();
    p.out = out;
    p.err = err;
    dim3 grid((g.N + g.bn - 1) / g.bn, g.M / kTcBM, g.splits);
    count_launches(1);
    if (g.bn == 128) return launch_pdl(tc_gemm_kernel<128>, grid, dim3(128), tc_gemm_smem_bytes(128), s, g.a, g.b, p);
    return launch_pdl(tc_gemm_kernel<256>, grid, dim3(128), tc_gemm_smem_bytes(256), s, g.a, g.b, p);
}

}  // namespace qed

extern "C" qed_status qed_tc_gemm(const void *a_planes, int32_t planes_a, const void *b_planes, int32_t planes_b,
                                  int32_t M, int32_t N, int32_t K, int32_t n_seg, const int32_t *seg_pairs,
                                  int32_t splits, float *out, qed_stream stream) {
    using namespace qed;
    if (!a_planes || !b_planes || !out || !seg_pairs || M <= 0 || N <= 0 || K <= 0 || splits <= 0) {
        set_error("qed_tc_gemm: bad argument");
        return QED_EINVAL;
    }
    TcGemm g;
    int pairs[2 * kTcMaxSeg];
    for (int q = 0; q < 2 * n_seg && q < 2 * kTcMaxSeg; ++q) pairs[q] = seg_pairs[q];
    if (!tc_gemm_plan(g, a_planes, planes_a, b_planes, planes_b, M, N, K, n_seg, pairs, 1, splits)) return QED_EINVAL;
    if (g.splits != splits) {
        set_error("qed_tc_gemm: splits must divide the n_seg*K/64 k-blocks into that many non-empty slices");
        return QED_EINVAL;
    }
    uint32_t *err = nullptr;
    if (cudaMalloc((void **)&err, 4) != cudaSuccess) {
        cudaGetLastError();
        set_error("qed_tc_gemm: cudaMalloc failed");
        return QED_ENOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t le = cudaMemsetAsync(err, 0, 4, s);
    if (le == cudaSuccess) le = tc_gemm_launch(g, out, err, s);
    if (le != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaFree(err);
        set_error(std::string("qed_tc_gemm: launch failed: ") + cudaGetErrorString(le));
        return QED_ECUDA;
    }
    uint32_t h = 0;
    cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) {
        set_error(std::string("qed_tc_gemm: ") + cudaGetErrorString(e));
        return QED_ECUDA;
    }
    if (h & kErrTimeout) {
        set_error("qed_tc_gemm: a bounded wait ran out");
        return QED_ETIMEOUT;
    }
    return QED_OK;
}
