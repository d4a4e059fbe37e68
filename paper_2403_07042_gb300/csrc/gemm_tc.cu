// tcgen05 / TMA / mbarrier GEMM for sm_103a (Blackwell): the dense products of the
// "unitary evolution" stage (Sec. 4.2, Table 3) in split precision.
//
// One CTA computes one output tile (128 x BN, BN = 128 or 256) of one split-K slice:
//   warp 0, one lane : TMA producer, ring of FP16 tiles (A 128x64, B BNx64), 128-byte
//                      swizzled, completion tracked by mbarrier transaction bytes.  The
//                      plain product walks the segments' K blocks one plane pair per stage;
//                      the step's products (kEpiW, kEpiV) load every plane of both operands
//                      for one 64-wide K block into one stage (2 stages)
//   warp 1, one lane : MMA issuer, tcgen05.mma.cta_group::1.kind::f16 (M=128, N=BN, K=16);
//                      the step's products issue every plane product of the stage, the
//                      leading one (hi x hi) into one TMEM accumulator and the corrections
//                      into a second; tcgen05.commit frees each smem stage
//   epilogue         : kEpiPlain (4 warps) stores the slice; kEpiW / kEpiV (8 warps) add the
//                      two accumulators into shared memory, sum the cluster's split-K slices
//                      through distributed shared memory and write W (and its FP16 planes)
//                      or V = U rho U^+ (gemm_tc.h)
// All set-up (barriers, TMEM allocation, tensor-map prefetch) comes before the wait on the
// previous kernel of the step (programmatic dependent launch); every load comes after it.
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel records
// kErrTimeout, stops issuing work, waits (bounded) for what it issued, frees TMEM and
// returns.  Every CTA of a cluster reaches each cluster barrier exactly once on every path.
#include <cstdio>
#include <cstring>
#include <string>

#include <cuda_fp16.h>

#include "df.h"
#include "checks.h"
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

// Asynchronous 16-byte global -> shared copies (the epilogue's inputs, staged while the
// mainloop runs).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Accumulator columns into registers without waiting; tmem_wait() completes every load
// issued before it.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
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
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct Params {
    int M, N;
    int kb_per_seg;
    int kb_total;
    int kb_per_split;
    uint32_t seg_a, seg_b;  // plane of segment q in bits 3q..3q+2 (kept in registers)
    int tx_bytes;   // bytes one stage receives
    int nseg;       // plane products
    const uint32_t *gate;   // test hook: bounded wait for *gate == 0 before any load, or null
    long long gate_budget;
    float *out;
    uint32_t *err;
    TcEpilogue epi;
};

// ------------------------------------------------------------------ cluster helpers
// Cluster barrier (every thread of every CTA of the cluster arrives; like __syncthreads it
// completes once all of them have reached it, and every path of the kernel reaches each
// one exactly once).  Release / acquire order the shared-memory writes before it with the
// distributed-shared-memory reads after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address, in the cluster's shared window, of the same offset in the CTA of rank `rank`.
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// Loads from a peer's shared memory.  Volatile keeps them after the cluster barrier and in
// program order; without a memory clobber they do not serialise the surrounding loads, so a
// thread can have many of them in flight.
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// ------------------------------------------------------------------ shared-memory layout
// [stage ring: A and B tiles][kEpiV: staged epilogue inputs][barriers, TMEM slot, flags]
// After the mainloop the stage ring holds the CTA's FP32 partial tile (row stride BN + 4)
// and, for kEpiV, the staging arrays of the V epilogue.
template <int BN, int MODE>
__host__ __device__ constexpr int stages_of() { return MODE == kEpiPlain ? tc_stages(BN) : 2; }

// Plane tiles per stage: kEpiPlain one A and one B tile (the segments' k-blocks follow one
// another); kEpiW every plane of Delta (hi, mid, lo) and of rho (hi, lo); kEpiV every plane
// of W (hi, lo) and the two planes of Delta its products use (hi, mid).
template <int MODE>
__host__ __device__ constexpr int planes_a_of() { return MODE == kEpiW ? 3 : (MODE == kEpiV ? 2 : 1); }
template <int MODE>
__host__ __device__ constexpr int planes_b_of() { return MODE == kEpiPlain ? 1 : 2; }

template <int BN, int MODE>
__host__ __device__ constexpr uint32_t stage_bytes_of() {
    return planes_a_of<MODE>() * kStageA + planes_b_of<MODE>() * (uint32_t)BN * kTcBK * 2;
}

template <int BN>
__host__ __device__ constexpr int tile_stride() { return BN + 4; }

template <int BN, int MODE>
__host__ __device__ constexpr size_t ring_bytes() {
    return (size_t)stages_of<BN, MODE>() * stage_bytes_of<BN, MODE>();
}

// kEpiV inputs of one 32-row chunk: rho [32][64] float4, W(m, n) [2][32][64], W(n, m)
// [2][64][32] (re, im planes), P_m [32] and P_n [64] float4.
constexpr size_t kPrefRho = 0, kPrefW = 32 * 64 * 16, kPrefWT = kPrefW + 2 * 32 * 64 * 4,
                 kPrefPm = kPrefWT + 2 * 64 * 32 * 4, kPrefPn = kPrefPm + 32 * 16, kPrefBytes = kPrefPn + 64 * 16;

// The staged first chunk is kept for 128-wide kEpiV tiles only: a 256-wide one (large
// products, long main loops) has no room for it beside its two 96 KB stages.
template <int BN, int MODE>
__host__ __device__ constexpr size_t pref_bytes_of() { return MODE == kEpiV && BN == 128 ? kPrefBytes : 0; }

template <int BN, int MODE>
__host__ __device__ constexpr size_t smem_bytes_of() {
    return 1024 + ring_bytes<BN, MODE>() + pref_bytes_of<BN, MODE>() + (2 * stages_of<BN, MODE>() + 1) * 8 + 32;
}

static_assert((size_t)4 * 32 * 36 * 4 <= ring_bytes<128, kEpiPlain>(), "plain epilogue tiles fit the ring");
static_assert((size_t)kTcBM * tile_stride<128>() * 4 + 32 * 65 * (8 + 16) <= ring_bytes<128, kEpiV>(),
              "kEpiV buffers fit the ring");
static_assert((size_t)kTcBM * tile_stride<256>() * 4 + 32 * 65 * (8 + 16) <= ring_bytes<256, kEpiV>(),
              "kEpiV buffers fit the ring (256-wide)");
static_assert((size_t)kTcBM * tile_stride<256>() * 4 <= ring_bytes<256, kEpiW>(), "kEpiW tile fits the ring");
static_assert(smem_bytes_of<128, kEpiV>() <= 232448 && smem_bytes_of<128, kEpiW>() <= 232448 &&
                  smem_bytes_of<256, kEpiW>() <= 232448 && smem_bytes_of<256, kEpiV>() <= 232448,
              "shared memory per CTA");

// Threads of the cluster kernels: warps 0-3 run the pipeline roles and read the accumulator
// lanes they own; warps 4-7 join them for the accumulator copy and the epilogues; warps 2-7
// stage the kEpiV inputs while the mainloop runs.
constexpr int kClusterThreads = 256;

// ------------------------------------------------------------------ kEpiW
// After the cluster reduction: rows [r0, r0 + rows) of the tile (global rows
// R = 128 tile_m + row of [W_re; W_im]), summed over the cluster's partial tiles in rank
// order, scaled, written as W (FP32) and as the FP16 hi/lo planes of GEMM2's A operand.
template <int BN, int NT, int S>
__device__ __forceinline__ void epilogue_w(const Params &p, const uint32_t *peer, int r0, int tile_m, int tile_n) {
    constexpr int TS = tile_stride<BN>();
    constexpr int rows = kTcBM / S;
    constexpr int per_row = BN / 4;            // float4 per tile row
    constexpr int rows_per_it = NT / per_row;  // rows one pass of the block covers
    constexpr int kU = S >= 8 ? 2 : 4;         // rows per thread whose loads are in flight together
    static_assert(rows % (rows_per_it * kU) == 0 || rows < rows_per_it * kU, "row chunk");
    const int64_t Dp = p.epi.Dp;
    const float inv = p.epi.inv, s_w = p.epi.s_w;
    float *const w32 = p.epi.w32;
    __half *const w_pl = p.epi.w_pl;
    const int64_t lo_off = Dp * 2 * Dp;
    const int c4 = 4 * ((int)threadIdx.x % per_row), rsub = (int)threadIdx.x / per_row;
    const int64_t L = (int64_t)tile_n * BN + c4;
#pragma unroll 1
    for (int base = 0; base < rows; base += rows_per_it * kU) {
        float4 part[S][kU];
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int row = r0 + base + u * rows_per_it + rsub;
                if (base + u * rows_per_it + rsub < rows)
                    part[q][u] = ld_cluster_f4(peer[q] + (uint32_t)(row * TS + c4) * 4u);
            }
        if (L >= p.N) continue;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (base + u * rows_per_it + rsub >= rows) continue;
            float4 x = part[0][u];
#pragma unroll
            for (int q = 1; q < S; ++q) {
                x.x += part[q][u].x;
                x.y += part[q][u].y;
                x.z += part[q][u].z;
                x.w += part[q][u].w;
            }
            x.x *= inv;
            x.y *= inv;
            x.z *= inv;
            x.w *= inv;
            const int64_t R = (int64_t)tile_m * kTcBM + r0 + base + u * rows_per_it + rsub;
            if (!qed_check(p.err, R < 2 * Dp)) continue;
            const int64_t plane = R / Dp, k = R % Dp;
            *(float4 *)(w32 + plane * Dp * Dp + k * Dp + L) = x;
            const float a0 = x.x * s_w, a1 = x.y * s_w, a2 = x.z * s_w, a3 = x.w * s_w;
            const __half h0 = __float2half_rn(a0), h1 = __float2half_rn(a1), h2 = __float2half_rn(a2),
                         h3 = __float2half_rn(a3);
            __half2 hi[2] = {__halves2half2(h0, h1), __halves2half2(h2, h3)};
            __half2 lo[2] = {
                __halves2half2(__float2half_rn(a0 - __half2float(h0)), __float2half_rn(a1 - __half2float(h1))),
                __halves2half2(__float2half_rn(a2 - __half2float(h2)), __float2half_rn(a3 - __half2float(h3)))};
            __half *hp = w_pl + k * 2 * Dp + plane * Dp + L;
            *(uint2 *)hp = *(const uint2 *)hi;
            *(uint2 *)(hp + lo_off) = *(const uint2 *)lo;
        }
    }
}

// ------------------------------------------------------------------ kEpiV
// Stages the inputs of the CTA's first 32-row chunk (rows m0 .. m0 + 31, columns n0 .. n0 + 63)
// into `pref` with cp.async; run by threads [first, NT) while the mainloop runs.
template <int NT>
__device__ __forceinline__ void prefetch_v(const Params &p, uint32_t pref, int64_t m0, int64_t n0, int first) {
    const int pt = (int)threadIdx.x - first, np = NT - first;
    const int64_t D = p.epi.D, Dp = p.epi.Dp;
    const float4 *rho = p.epi.rho;
    const float *w32 = p.epi.w32;
    for (int c = pt; c < 32 * 64; c += np) {  // rho: one element per 16 bytes
        const int64_t m = m0 + (c >> 6), n = n0 + (c & 63);
        if (m < D && n < D) cp_async16(pref + kPrefRho + (uint32_t)c * 16u, rho + m * D + n);
    }
    for (int c = pt; c < 2 * 32 * 16; c += np) {  // W(m, n): 16 chunks of 4 floats per row
        const int pl = c >> 9, r = (c >> 4) & 31, q = c & 15;
        cp_async16(pref + kPrefW + (uint32_t)(pl * 2048 + r * 64 + q * 4) * 4u,
                   w32 + pl * Dp * Dp + (m0 + r) * Dp + n0 + q * 4);
    }
    for (int c = pt; c < 2 * 64 * 8; c += np) {  // W(n, m): 8 chunks of 4 floats per row n
        const int pl = c >> 9, r = (c >> 3) & 63, q = c & 7;
        cp_async16(pref + kPrefWT + (uint32_t)(pl * 2048 + r * 32 + q * 4) * 4u,
                   w32 + pl * Dp * Dp + (n0 + r) * Dp + m0 + q * 4);
    }
    for (int c = pt; c < 96; c += np) {  // phases P_m, P_n
        if (c < 32) {
            if (m0 + c < D) cp_async16(pref + kPrefPm + (uint32_t)c * 16u, p.epi.phase + m0 + c);
        } else if (n0 + c - 32 < D) {
            cp_async16(pref + kPrefPn + (uint32_t)(c - 32) * 16u, p.epi.phase + n0 + c - 32);
        }
    }
    cp_async_commit();
}

// One 32-row chunk of one 64-column group of the tile (rows s0 .. s0 + 31; m = 128 tile_m +
// row, n = 64 tj + c, the group's [X_re | X_im] at columns coff .. coff + 127 of the tile):
//   1. W(n, m) of the chunk transposed into shared memory,
//   2. V_mn = P_m conj(P_n) (rho_mn + W_mn + conj(W_nm) + inv X_mn) for n >= m (lanes along
//      n), written and kept in shared memory,
//   3. V_nm = conj(V_mn) for n > m (lanes along m).
// STAGED: rho, W and the phases come from the staged copy `pref`; otherwise from global
// memory (with all of a thread's loads of a group in flight together).  `scratch` holds
// [32][65] float2 and [32][65] float4.
template <int NT, int S, bool STAGED, int BN>
__device__ __forceinline__ void v_chunk(const Params &p, const uint32_t *peer, int s0, int tile_m, int tj, int coff,
                                        uint8_t *scratch, const uint8_t *pref) {
    static_assert(NT == 256, "the kEpiV thread mapping assumes 8 warps");
    constexpr int TS = tile_stride<BN>();
    typedef float2 WRow[65];
    typedef float4 VRow[65];
    WRow *WTs = (WRow *)scratch;
    VRow *Vs = (VRow *)(scratch + 32 * 65 * sizeof(float2));
    const int64_t D = p.epi.D, Dp = p.epi.Dp;
    const float inv = p.epi.inv;
    const float *const w_re = p.epi.w32;
    const float *const w_im = p.epi.w32 + Dp * Dp;
    const float4 *const rho = p.epi.rho;
    const float4 *const phase = p.epi.phase;
    float4 *const V = p.epi.V;
    const float4 *pr_rho = (const float4 *)(pref + kPrefRho);
    const float *pr_w = (const float *)(pref + kPrefW);
    const float *pr_wt = (const float *)(pref + kPrefWT);
    const float4 *pr_pm = (const float4 *)(pref + kPrefPm);
    const float4 *pr_pn = (const float4 *)(pref + kPrefPn);
    const int64_t m0 = (int64_t)tile_m * kTcBM, n0 = (int64_t)tj * 64;
    const int t = threadIdx.x;
    {  // 1. W(n, m): lanes along m, 8 columns n per thread
        const int ml = t & 31, nb = t >> 5;
        const int64_t m = m0 + s0 + ml;
        float wr[8], wi[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int nl = nb + 8 * it;
            if (STAGED) {
                wr[it] = pr_wt[nl * 32 + ml];
                wi[it] = pr_wt[2048 + nl * 32 + ml];
            } else {
                const int64_t n = n0 + nl;
                const int64_t o = (m < D && n < D) ? n * Dp + m : 0;
                wr[it] = w_re[o];
                wi[it] = w_im[o];
            }
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) WTs[ml][nb + 8 * it] = make_float2(wr[it], wi[it]);
    }
    __syncthreads();
    {  // 2. V_mn, n >= m: 16 threads per row, 4 consecutive columns n each, 16 rows per pass
        const int nq = (t & 15) * 4, mr = t >> 4;
        cdf pn[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t n = n0 + nq + c;
            pn[c] = load_cdf(STAGED ? pr_pn[nq + c] : phase[n < D ? n : 0]);
        }
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const int ml = mr + 16 * pass;
            const int row = s0 + ml;
            const int64_t m = m0 + row;
            const uint32_t off = (uint32_t)(row * TS + coff + nq) * 4u;
            float4 xr[S], xi[S];
#pragma unroll
            for (int q = 0; q < S; ++q) {
                xr[q] = ld_cluster_f4(peer[q] + off);
                xi[q] = ld_cluster_f4(peer[q] + off + 64u * 4u);
            }
            float4 wr, wi, pm4;
            float4 rv[4];
            if (STAGED) {
                wr = *(const float4 *)(pr_w + ml * 64 + nq);
                wi = *(const float4 *)(pr_w + 2048 + ml * 64 + nq);
#pragma unroll
                for (int c = 0; c < 4; ++c) rv[c] = pr_rho[ml * 64 + nq + c];
                pm4 = pr_pm[ml];
            } else {
                const int64_t mc = m < D ? m : 0;
                wr = *(const float4 *)(w_re + mc * Dp + n0 + nq);
                wi = *(const float4 *)(w_im + mc * Dp + n0 + nq);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int64_t n = n0 + nq + c;
                    rv[c] = rho[mc * D + (n < D ? n : 0)];
                }
                pm4 = phase[mc];
            }
#pragma unroll
            for (int q = 1; q < S; ++q) {
                xr[0].x += xr[q].x;
                xr[0].y += xr[q].y;
                xr[0].z += xr[q].z;
                xr[0].w += xr[q].w;
                xi[0].x += xi[q].x;
                xi[0].y += xi[q].y;
                xi[0].z += xi[q].z;
                xi[0].w += xi[q].w;
            }
            const float xrc[4] = {xr[0].x, xr[0].y, xr[0].z, xr[0].w};
            const float xic[4] = {xi[0].x, xi[0].y, xi[0].z, xi[0].w};
            const float wrc[4] = {wr.x, wr.y, wr.z, wr.w};
            const float wic[4] = {wi.x, wi.y, wi.z, wi.w};
            const cdf pm = load_cdf(pm4);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t n = n0 + nq + c;
                if (!(m < D && n < D && n >= m)) continue;
                const float2 wt = WTs[ml][nq + c];
                const float ir = wrc[c] + wt.x + xrc[c] * inv;
                const float ii = wic[c] - wt.y + xic[c] * inv;
                cdf r = load_cdf(rv[c]);
                r.re = df_add_f(r.re, ir);
                r.im = df_add_f(r.im, ii);
                const float4 v = store_cdf(cdf_mul(cdf_mul_conj(pm, pn[c]), r));
                V[m * D + n] = v;
                Vs[ml][nq + c] = v;
            }
        }
    }
    __syncthreads();
    {  // 3. the mirror V_nm = conj(V_mn), n > m: lanes along m
        const int ml = t & 31, nb = t >> 5;
        const int64_t m = m0 + s0 + ml;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int nl = nb + 8 * it;
            const int64_t n = n0 + nl;
            if (m < D && n < D && n > m) {
                const float4 v = Vs[ml][nl];
                V[n * D + m] = make_float4(v.x, v.y, -v.z, -v.w);
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ the tile
// One output tile of one split-K slice.  tmA / tmB are generic addresses of tensor maps in
// parameter or global memory.  MODE and the cluster size S are compile-time: kEpiPlain
// (NT = 128, S = 1) writes the slice; kEpiW / kEpiV (NT = 256) reduce the S slices of the
// tile inside the cluster (the CTA of rank `split` owns rows [split 128/S, (split+1) 128/S)).
template <int BN, int NT, int MODE, int S>
__device__ __forceinline__ void gemm_tile(const CUtensorMap *tmA, const CUtensorMap *tmB, const Params &p,
                                          int tile_m, int tile_n, int split) {
    constexpr int kTcBN = BN;
    constexpr int kTcStages = stages_of<BN, MODE>();
    constexpr int NA = planes_a_of<MODE>(), NB = planes_b_of<MODE>();
    constexpr uint32_t kTileB = BN * kTcBK * 2;
    constexpr uint32_t kStage = stage_bytes_of<BN, MODE>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = smem;
    uint8_t *pref = smem + ring_bytes<BN, MODE>();
    uint64_t *bars = (uint64_t *)(pref + pref_bytes_of<BN, MODE>());  // full[S], empty[S], accum
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * kTcStages + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;    // TMA stage loads issued by the producer
    volatile int *consumed = abort_flag + 2;  // stage loads the MMA issuer has waited for

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a 256-wide tile with 128 columns of the product left (the last tile when N is an odd
    // multiple of 128) computes only those
    // (kEpiV: the tile's second 64-column group lies wholly past D)
    const bool narrow = BN == 256 && (MODE == kEpiV ? (int64_t)(2 * tile_n + 1) * 64 >= p.epi.D
                                                    : p.N - tile_n * BN <= BN / 2);
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
    // the step's products keep two accumulators: columns [0, BN) for the leading plane
    // product (hi x hi) and [BN, 2 BN) for the correction products, which are 2^-11 of it and
    // would otherwise lose bits when added into the large partial sums
    constexpr uint32_t kTmemCols = MODE == kEpiPlain ? BN : 2 * BN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
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
    if (p.gate) {
        // wait-gate test hook: a bounded wait on a flag, taken before this CTA issues any
        // load or product; when it runs out the CTA records the timeout and does no work
        if (threadIdx.x == 0) {
            const long long t0 = clock64();
            while (*(volatile const uint32_t *)p.gate != 0u) {
                if (clock64() - t0 > p.gate_budget) {
                    *abort_flag = 1;
                    atomicOr(p.err, kErrTimeout);
                    break;
                }
            }
        }
        __syncthreads();
    }

    constexpr int rows = kTcBM / S;
    const int r0 = split * rows;
    if constexpr (MODE == kEpiV && BN == 128) {
        if (warp >= 2) prefetch_v<NT>(p, smem_u32(pref), (int64_t)tile_m * kTcBM + r0, (int64_t)tile_n * 64, 64);
    }

    // Stage i of this slice: kEpiPlain walks the segments' k-blocks one after another (one A
    // and one B tile per stage); the step's products (kEpiW / kEpiV) load every plane of both
    // operands for one k-block once (NA A tiles, NB B tiles) and issue all plane products
    // of that k-block on them.
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
            const uint32_t bar = full0 + 8 * s;
            uint8_t *st = ring + s * kStage;
            mbar_expect_tx(bar, (uint32_t)p.tx_bytes);
            const int kb = kb0 + i;
            if constexpr (MODE == kEpiPlain) {
                const int seg = kb / p.kb_per_seg, kk = kb % p.kb_per_seg;
                tma_load_3d(smem_u32(st), tmA, kk * kTcBK, tile_m * kTcBM, (p.seg_a >> (3 * seg)) & 7, bar);
                tma_load_3d(smem_u32(st + kStageA), tmB, kk * kTcBK, tile_n * kTcBN, (p.seg_b >> (3 * seg)) & 7,
                            bar);
            } else {
#pragma unroll
                for (int a = 0; a < NA; ++a)
                    tma_load_3d(smem_u32(st + a * kStageA), tmA, kb * kTcBK, tile_m * kTcBM, a, bar);
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    tma_load_3d(smem_u32(st + NA * kStageA + b * kTileB), tmB, kb * kTcBK, tile_n * kTcBN, b, bar);
            }
            *issued = i + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer; a 256-wide tile with only 128 columns left before N (N is a multiple of
        // 128) issues 128-wide MMAs: the other half of its B box is the TMA's zero fill
        const uint32_t idesc =
            narrow ? idesc_f16(kTcBM, kTcBN / 2) : idesc_f16(kTcBM, kTcBN);
        for (int i = 0; i < nkb; ++i) {
            if (*abort_flag) break;  // the stages already issued are drained at the end
            const int s = i % kTcStages;
            const uint32_t par = (i / kTcStages) & 1;
            const long long budget = kWaitCycles;
            if (!mbar_wait(full0 + 8 * s, par, budget)) {
                *abort_flag = 1;
                atomicOr(p.err, kErrTimeout);
                break;
            }
            *consumed = i + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!*abort_flag) {
                const uint8_t *st = ring + s * kStage;
                if constexpr (MODE == kEpiPlain) {
                    const uint64_t ad = smem_desc_sw128(smem_u32(st));
                    const uint64_t bd = smem_desc_sw128(smem_u32(st + kStageA));
#pragma unroll
                    for (int k = 0; k < kTcBK / 16; ++k)  // 16 FP16 = 32 bytes per step along K
                        mma_f16(tmem, ad + 2 * k, bd + 2 * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
                } else {
                    for (int q = 0; q < p.nseg; ++q) {
                        const int pa = (p.seg_a >> (3 * q)) & 7, pb = (p.seg_b >> (3 * q)) & 7;
                        const uint64_t ad = smem_desc_sw128(smem_u32(st + pa * kStageA));
                        const uint64_t bd = smem_desc_sw128(smem_u32(st + NA * kStageA + pb * kTileB));
                        const uint32_t acc = q == 0 ? tmem : tmem + (uint32_t)BN;
                        const bool first = i == 0 && q <= 1;  // first product into its accumulator
#pragma unroll
                        for (int k = 0; k < kTcBK / 16; ++k)
                            mma_f16(acc, ad + 2 * k, bd + 2 * k, idesc, (first && k == 0) ? 0u : 1u);
                    }
                }
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
    // warp w may read the accumulator lanes 32 (w % 4) .. 32 (w % 4) + 31
    const uint32_t tm_row = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    if constexpr (MODE == kEpiPlain) {
        // register copies: the epilogue's global stores must not force reloads of p
        const int pN = p.N;
        float *const out = p.out + (int64_t)split * p.M * pN;  // this split-K slice
        const int col0 = tile_n * BN;
        const int ncols = min(BN, pN - col0);
        const int64_t R0 = (int64_t)tile_m * kTcBM + warp * 32;  // output row of lane 0
        // the stage buffers are free once every MMA of the CTA has completed
        float *tbuf = (float *)ring + warp * (32 * 36);  // per-warp [32][36] transpose tile
        if (ok && warp < 4) {
#pragma unroll 1
            for (int c = 0; c < ncols; c += 32) {
                uint32_t r[32];
                tmem_ld32_async(tm_row + (uint32_t)c, r);
                tmem_wait();
                // transpose through shared memory: row-major 16-byte pieces, 4 rows per store
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *(float4 *)(tbuf + lane * 36 + 4 * q) =
                        make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                    __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                __syncwarp();
                const int sub = lane >> 3, col4 = 4 * (lane & 7);
                float *op = out + (R0 * pN) + col0 + c + col4;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int rr = 4 * it + sub;
                    *(float4 *)(op + (int64_t)rr * pN) = *(const float4 *)(tbuf + rr * 36 + col4);
                }
                __syncwarp();
            }
        }
    } else {
        static_assert(NT == kClusterThreads, "cluster epilogues run with 8 warps");
        // the CTA's partial tile into its shared memory (the stage buffers, free once every
        // MMA has completed), row-major with a padded stride; each warp group copies its half
        // of the columns, two 32-column loads in flight at a time
        constexpr int TS = tile_stride<BN>();
        constexpr int cols = BN / (NT / 128);
        float *tile = (float *)ring;
        if (ok) {
            const int c0 = (warp >> 2) * cols;
            const bool corr = p.nseg > 1;
            const int c_end = narrow ? min(c0 + cols, BN / 2) : c0 + cols;  // columns the MMAs wrote
#pragma unroll 1
            for (int c = c0; c < c_end; c += 32) {
                uint32_t mv[32], cv[32];
                tmem_ld32_async(tm_row + (uint32_t)c, mv);
                tmem_ld32_async(tm_row + (uint32_t)(BN + c), cv);
                tmem_wait();
                float *dst = tile + ((warp & 3) * 32 + lane) * TS + c;
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    dst[q] = __uint_as_float(mv[q]) + (corr ? __uint_as_float(cv[q]) : 0.f);
            }
        }
        if constexpr (MODE == kEpiV && BN == 128) {
            if (warp >= 2) cp_async_wait_all();  // the staged inputs of the first chunk
        }
        __syncwarp();
        cluster_sync();  // every partial tile (and the staged inputs) in place
        uint32_t peer[S];
#pragma unroll
        for (int q = 0; q < S; ++q) peer[q] = map_rank(smem_u32(tile), (uint32_t)q);
        if constexpr (MODE == kEpiW) {
            epilogue_w<BN, NT, S>(p, peer, r0, tile_m, tile_n);
        } else {
            uint8_t *scratch = (uint8_t *)(tile + kTcBM * TS);
            if constexpr (BN == 128) {
                v_chunk<NT, S, true, BN>(p, peer, r0, tile_m, tile_n, 0, scratch, pref);
#pragma unroll 1
                for (int s0 = r0 + 32; s0 < r0 + rows; s0 += 32)
                    v_chunk<NT, S, false, BN>(p, peer, s0, tile_m, tile_n, 0, scratch, pref);
            } else {
                // the tile's 64-column groups one after another (B's rows hold [re | im] of 64
                // columns per 128 rows); groups wholly past D are padding
#pragma unroll 1
                for (int g = 0; g < BN / 128; ++g) {
                    const int tj = (BN / 128) * tile_n + g;
                    if ((int64_t)tj * 64 >= p.epi.D) break;
#pragma unroll 1
                    for (int s0 = r0; s0 < r0 + rows; s0 += 32)
                        v_chunk<NT, S, false, BN>(p, peer, s0, tile_m, tj, 128 * g, scratch, pref);
                }
            }
        }
        __syncwarp();
        cluster_sync();  // no CTA leaves while a peer may still read its tile
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

template <int BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, Params p) {
    gemm_tile<BN, 128, kEpiPlain, 1>(&tmA, &tmB, p, blockIdx.y, blockIdx.x, blockIdx.z);
}

Params params_of(const GemmJob &jb, const TcSegs &segs, uint32_t *err) {
    Params p;
    p.M = jb.M;
    p.N = jb.N;
    p.kb_per_seg = jb.kb_per_seg;
    p.kb_total = jb.kb_per_seg;  // the step's products split the k-blocks, each carrying every plane product
    p.kb_per_split = jb.kb_per_split;
    p.tx_bytes = jb.tx_bytes;
    p.nseg = segs.nseg;
    p.gate = jb.gate;
    p.gate_budget = jb.gate_budget;
    p.epi = jb.epi;
    p.seg_a = 0;
    p.seg_b = 0;
    for (int q = 0; q < segs.nseg; ++q) {
        p.seg_a |= (uint32_t)segs.a[q] << (3 * q);
        p.seg_b |= (uint32_t)segs.b[q] << (3 * q);
    }
    p.out = jb.out;
    p.err = err;
    return p;
}

// Grouped launch (batches, one CTA per item, clusters of one): CTA b computes work item
// items[b] of job items[b].job, with that job's tensor maps read from global memory.
template <int BN, int MODE>
__global__ void __launch_bounds__(kClusterThreads, 1) tc_gemm_grouped_kernel(const GemmItem *__restrict__ items,
                                                                           const GemmJob *__restrict__ jobs,
                                                                           TcSegs segs, uint32_t *err) {
    const GemmItem it = items[blockIdx.x];
    const GemmJob &jb = jobs[it.job];
    Params p;
    p.M = jb.M;
    p.N = jb.N;
    p.kb_per_seg = jb.kb_per_seg;
    p.kb_total = jb.kb_per_seg;  // the step's products split the k-blocks, each carrying every plane product
    p.kb_per_split = jb.kb_per_split;
    p.tx_bytes = jb.tx_bytes;
    p.nseg = segs.nseg;
    p.gate = jb.gate;
    p.gate_budget = jb.gate_budget;
    p.epi = jb.epi;
    p.seg_a = 0;
    p.seg_b = 0;
#pragma unroll
    for (int q = 0; q < kTcMaxSeg; ++q) {
        p.seg_a |= (uint32_t)segs.a[q] << (3 * q);
        p.seg_b |= (uint32_t)segs.b[q] << (3 * q);
    }
    p.out = jb.out;
    p.err = err;
    gemm_tile<BN, kClusterThreads, MODE, 1>(jb.map_a, jb.map_b, p, it.tile_m, it.tile_n, 0);
}

// Tile decoding of one model's product (tc_gemm_single_launch).
struct SingleTiles {
    int nmp;  // kEpiW: row tiles of one plane holding rows < D
    int dpt;  // kEpiW: row tiles per plane (Dp / 128)
    int ntn;  // kEpiW: column tiles holding columns < D
    int ntj;  // kEpiV: 64-column groups holding columns < D
};

template <int BN, int MODE, int S>
__global__ void __launch_bounds__(kClusterThreads, 1) tc_gemm_single_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                          const __grid_constant__ CUtensorMap tmB,
                                                                          const __grid_constant__ Params p,
                                                                          SingleTiles tl) {
    const int split = blockIdx.x % S;
    int t = blockIdx.x / S, tm, tn;
    if (MODE == kEpiW) {
        tn = t % tl.ntn;
        const int tmv = t / tl.ntn;
        tm = (tmv / tl.nmp) * tl.dpt + tmv % tl.nmp;
    } else {
        // rows of tiles on or above the diagonal: row tm holds the tiles from column tile
        // 2 tm / c (c = 64-column groups per tile) to the last holding columns < D
        constexpr int c = BN / 128;
        const int ntt = (tl.ntj + c - 1) / c;
        tm = 0;
        while (t >= ntt - 2 * tm / c) {
            t -= ntt - 2 * tm / c;
            ++tm;
        }
        tn = 2 * tm / c + t;
    }
    gemm_tile<BN, kClusterThreads, MODE, S>(&tmA, &tmB, p, tm, tn, split);
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

size_t tc_gemm_smem_bytes(int bn) { return bn == 128 ? smem_bytes_of<128, kEpiW>() : smem_bytes_of<256, kEpiW>(); }

template <class F>
bool set_smem(F kernel, size_t bytes) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaFuncSetAttribute(max dynamic smem) failed for the tcgen05 GEMM");
        return false;
    }
    return true;
}

bool tc_gemm_plan(TcGemm &g, const void *a_planes, int planes_a, const void *b_planes, int planes_b, int M, int N,
                  int K, int nseg, const int *seg_pairs, int num_sms, int force_splits, int force_bn, bool merged) {
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
    // k-blocks to split: one per segment and 64 columns of K, or (merged) one per 64 columns
    // of K carrying every segment's product
    const int kb_total = (merged ? 1 : nseg) * (K / kTcBK);
    // split-K slices (a power of two <= 4) while the tiles fill fewer than half the SMs and
    // each slice keeps at least 4 segment k-blocks of work
    int splits = 1;
    while (splits < kTcMaxAutoSplits && tiles * splits * 2 <= num_sms && kb_total / (splits * 2) >= (merged ? 1 : 4))
        splits *= 2;
    if (force_splits > 0) splits = force_splits > kb_total ? kb_total : force_splits;
    g.kb_per_split = (kb_total + splits - 1) / splits;
    g.splits = (kb_total + g.kb_per_split - 1) / g.kb_per_split;
    static bool attr_set = false;
    if (!attr_set) {
        if (!set_smem(tc_gemm_kernel<128>, smem_bytes_of<128, kEpiPlain>()) ||
            !set_smem(tc_gemm_kernel<256>, smem_bytes_of<256, kEpiPlain>()))
            return false;
        attr_set = true;
    }
    return true;
}

bool tc_gemm_prepare_grouped() {
    static bool done = false;
    if (done) return true;
    if (!set_smem(tc_gemm_grouped_kernel<128, kEpiW>, smem_bytes_of<128, kEpiW>()) ||
        !set_smem(tc_gemm_grouped_kernel<256, kEpiW>, smem_bytes_of<256, kEpiW>()) ||
        !set_smem(tc_gemm_grouped_kernel<128, kEpiV>, smem_bytes_of<128, kEpiV>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiW, 1>, smem_bytes_of<128, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiW, 2>, smem_bytes_of<128, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiW, 4>, smem_bytes_of<128, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiW, 8>, smem_bytes_of<128, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiW, 1>, smem_bytes_of<256, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiW, 2>, smem_bytes_of<256, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiW, 4>, smem_bytes_of<256, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiW, 8>, smem_bytes_of<256, kEpiW>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiV, 1>, smem_bytes_of<128, kEpiV>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiV, 2>, smem_bytes_of<128, kEpiV>()) ||
        !set_smem(tc_gemm_single_kernel<128, kEpiV, 4>, smem_bytes_of<128, kEpiV>()) ||
        !set_smem(tc_gemm_grouped_kernel<256, kEpiV>, smem_bytes_of<256, kEpiV>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiV, 1>, smem_bytes_of<256, kEpiV>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiV, 2>, smem_bytes_of<256, kEpiV>()) ||
        !set_smem(tc_gemm_single_kernel<256, kEpiV, 4>, smem_bytes_of<256, kEpiV>()))
        return false;
    done = true;
    return true;
}

cudaError_t tc_gemm_grouped_launch(const GemmItem *items, int n_items, const GemmJob *jobs, const TcSegs &segs,
                                   int bn, int mode, int cluster, uint32_t *err, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    // the grouped form runs every product unsplit (each instance of a batch is one job)
    if (cluster != 1 || (mode != kEpiW && mode != kEpiV) || (bn != 128 && bn != 256)) return cudaErrorInvalidValue;
    count_launches(1);
    const dim3 grid(n_items), block(kClusterThreads);
    if (mode == kEpiV && bn == 128)
        return launch_pdl(tc_gemm_grouped_kernel<128, kEpiV>, grid, block, smem_bytes_of<128, kEpiV>(), s, items, jobs,
                          segs, err);
    if (mode == kEpiV)
        return launch_pdl(tc_gemm_grouped_kernel<256, kEpiV>, grid, block, smem_bytes_of<256, kEpiV>(), s, items, jobs,
                          segs, err);
    if (bn == 128)
        return launch_pdl(tc_gemm_grouped_kernel<128, kEpiW>, grid, block, smem_bytes_of<128, kEpiW>(), s, items, jobs,
                          segs, err);
    return launch_pdl(tc_gemm_grouped_kernel<256, kEpiW>, grid, block, smem_bytes_of<256, kEpiW>(), s, items, jobs,
                      segs, err);
}

SingleTiles single_tiles(const TcGemm &g, int mode, int64_t D) {
    SingleTiles t;
    const int64_t Dp = mode == kEpiV ? g.M : g.N;  // GEMM2: Dp x 2Dp; GEMM1: 2Dp x Dp
    t.dpt = (int)(Dp / kTcBM);
    t.nmp = (int)((D + kTcBM - 1) / kTcBM);
    t.ntn = (int)((D + g.bn - 1) / g.bn);
    t.ntj = (int)((D + 63) / 64);
    return t;
}

int tc_stage_tx_bytes(const TcGemm &g, int mode) {
    const int b_tile = g.b_box_rows * kTcBK * 2;
    if (mode == kEpiW) return planes_a_of<kEpiW>() * (int)kStageA + planes_b_of<kEpiW>() * b_tile;
    if (mode == kEpiV) return planes_a_of<kEpiV>() * (int)kStageA + planes_b_of<kEpiV>() * b_tile;
    return (int)kStageA + b_tile;
}

int tc_gemm_single_ctas(const TcGemm &g, int mode, int64_t D) {
    const SingleTiles t = single_tiles(g, mode, D);
    int tiles = 0;
    if (mode == kEpiW) {
        tiles = 2 * t.nmp * t.ntn;
    } else {
        const int c = g.bn / 128, ntt = (t.ntj + c - 1) / c;
        for (int tm = 0; tm < t.nmp; ++tm) tiles += ntt - 2 * tm / c;
    }
    return tiles * g.splits;
}

template <int BN, int MODE, int S>
cudaError_t single_launch(const TcGemm &g, const Params &p, const SingleTiles &t, int ctas, cudaStream_t s) {
    return launch_pdl_cluster(tc_gemm_single_kernel<BN, MODE, S>, dim3(ctas), dim3(kClusterThreads),
                              smem_bytes_of<BN, MODE>(), s, S, g.a, g.b, p, t);
}

cudaError_t tc_gemm_single_launch(const TcGemm &g, const GemmJob &job, const TcSegs &segs, int64_t D, uint32_t *err,
                                  cudaStream_t s) {
    const int mode = job.mode;
    const int ctas = tc_gemm_single_ctas(g, mode, D);
    if (ctas <= 0) return cudaSuccess;
    const Params p = params_of(job, segs, err);
    const SingleTiles t = single_tiles(g, mode, D);
    count_launches(1);
    if (mode == kEpiV) {
        if (g.bn == 128) {
            switch (g.splits) {
                case 1: return single_launch<128, kEpiV, 1>(g, p, t, ctas, s);
                case 2: return single_launch<128, kEpiV, 2>(g, p, t, ctas, s);
                case 4: return single_launch<128, kEpiV, 4>(g, p, t, ctas, s);
                default: return cudaErrorInvalidValue;
            }
        }
        switch (g.splits) {
            case 1: return single_launch<256, kEpiV, 1>(g, p, t, ctas, s);
            case 2: return single_launch<256, kEpiV, 2>(g, p, t, ctas, s);
            case 4: return single_launch<256, kEpiV, 4>(g, p, t, ctas, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (mode != kEpiW) return cudaErrorInvalidValue;
    if (g.bn == 128) {
        switch (g.splits) {
            case 1: return single_launch<128, kEpiW, 1>(g, p, t, ctas, s);
            case 2: return single_launch<128, kEpiW, 2>(g, p, t, ctas, s);
            case 4: return single_launch<128, kEpiW, 4>(g, p, t, ctas, s);
            case 8: return single_launch<128, kEpiW, 8>(g, p, t, ctas, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (g.splits) {
        case 1: return single_launch<256, kEpiW, 1>(g, p, t, ctas, s);
        case 2: return single_launch<256, kEpiW, 2>(g, p, t, ctas, s);
        case 4: return single_launch<256, kEpiW, 4>(g, p, t, ctas, s);
        case 8: return single_launch<256, kEpiW, 8>(g, p, t, ctas, s);
        default: return cudaErrorInvalidValue;
    }
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
    p.nseg = g.nseg;
    p.gate = nullptr;
    p.gate_budget = 0;
    p.epi = TcEpilogue();
    p.out = out;
    p.err = err;
    dim3 grid((g.N + g.bn - 1) / g.bn, g.M / kTcBM, g.splits);
    count_launches(1);
    if (g.bn == 128)
        return launch_pdl(tc_gemm_kernel<128>, grid, dim3(128), smem_bytes_of<128, kEpiPlain>(), s, g.a, g.b, p);
    return launch_pdl(tc_gemm_kernel<256>, grid, dim3(128), smem_bytes_of<256, kEpiPlain>(), s, g.a, g.b, p);
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
    if (device_malloc((void **)&err, 4) != cudaSuccess) {
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
