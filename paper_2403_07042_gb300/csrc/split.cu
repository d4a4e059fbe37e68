// Split-precision step in increment form.
//
// With E_k = H_kk and P = diag(exp(-i E_k dt)), the propagator factors exactly as
// U = P (I + Delta), Delta = P^-1 U - I, so the "unitary evolution" of Sec. 4.2 is
//     V = U rho U^+ = P (rho + W + W^+ + X) P^+,   W = Delta rho,  X = W Delta^+.
// Only the small increments W and X go through the tensor cores: every operand is split
// into power-of-two scaled FP16 pieces (rho and W: hi + lo; the constant Delta: hi + mid +
// lo, because its representation error would otherwise add up coherently step after
// step) and the products that matter at 2^-22 are accumulated in FP32 (GEMM1: four,
// GEMM2: three).  Complex products use the real embedding with the signs folded into the
// constant operands:
//   GEMM1  [W_re; W_im] (2Dp x Dp)  = [[D_re, D_im], [D_im, -D_re]] . [rho_re | rho_im]^T
//   GEMM2  [X_re | X_im] (Dp x 2Dp) = [W_re | W_im] . [[D_re, D_im], [-D_im, D_re]]^T
// (rho^T = conj(rho) for the Hermitian rho, so the row-major rho planes are the K-major
// operand directly.)
//
// The master rho is held as a double-float (an unevaluated sum of two FP32 words, about
// 48 significant bits): GB300 executes FP64 at a small fraction of its FP32 rate, so the
// per-step element work (forming V, the phase, the Lindblad update of Eq. 3, the next
// FP16 planes) runs entirely in FP32 arithmetic with error-free transformations.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "checks.h"
#include "gemm_tc.h"
#include "kernels.h"
#include "pdl.h"
#include "split.h"
#include "df.h"

namespace qed {

// Device-side description of one instance (one model) for the grouped kernels.
struct InstDesc {
    int64_t D, Dp;
    float s_rho;            // scale of the rho planes
    float4 *rho, *V, *Y;    // state, V = U rho U^+, stage buffer of the Strang step
    const float4 *phase;
    const float2 *damp;
    const int32_t *in_ptr, *in_jump, *in_src;
    const float2 *coef;
    const int4 *in_tab;     // [D][kInMax] {jump, src, coef hi, coef lo} or null (use the lists)
    const int4 *jtab;       // [D][kInMax] per jump j < nj: {src or -1, coef hi, coef lo, 0}, or null
    int nj;
    __half *rho_pl;
    uint32_t *err;          // the instance's error word (bounds checks of the QED_CHECKS build)
};

// Rows with at most kInMax incoming jump entries use a padded table (one vector load per
// entry, all gathers in flight together) instead of the two-pointer merge of the lists.
constexpr int kInMax = 4;
constexpr int kNoJump = 0x7fffffff;
// Pairs of incoming lists longer than this in total are merged by the whole warp.
constexpr int kLongMerge = 32;

// 32 x (8 kRows) element blocks (the Lindblad kernels) of one instance
struct TileItem {
    int inst, bx, by, pad;
};

// The grouped work of one or many instances: descriptors, GEMM jobs and work lists.
struct Batch {
    int n = 0;
    InstDesc *desc = nullptr;
    GemmJob *jobs1 = nullptr, *jobs2 = nullptr;
    CUtensorMap *maps = nullptr;  // [4 n]: A1, B1, A2, B2 of each instance
    GemmItem *items1 = nullptr, *items2 = nullptr;
    int n_items1 = 0, n_items2 = 0;
    TileItem *etiles = nullptr;
    int n_etiles = 0;
    bool jt = false;  // every instance has per-jump incoming tables (dissipate_jt_kernel)
    int cs1 = 1, cs2 = 1;  // split-K slices of GEMM1 / GEMM2 = CTAs per cluster
    int scheme = QED_SCHEME_LIE;
    int bn1 = 256, bn2 = 128;  // tile widths (one per grouped launch)
    // one model on its own: its products launch with their tensor maps and jobs as kernel
    // parameters (tc_gemm_single_launch) instead of through the tables above
    bool single = false;
    int64_t D = 0;
    TcGemm g1, g2;
    GemmJob j1, j2;
    void release() {
        void *ptrs[] = {desc, jobs1, jobs2, maps, items1, items2, etiles};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        *this = Batch();
    }
};

struct SplitState {
    Batch self;               // this model as a batch of one
    int64_t Dp = 0;           // padded dimension (multiple of 128)
    int num_sms = 148;
    TcGemm g1, g2;
    // constant operands, FP16 [3 (hi, mid, lo)][2Dp][2Dp]
    __half *a1 = nullptr;     // [[Dre, Dim], [Dim, -Dre]]   (GEMM1 A)
    __half *b2 = nullptr;     // [[Dre, Dim], [-Dim, Dre]]   (GEMM2 B), rows in [re | im] groups of 64
    // dynamic operands, FP16 [2 (hi, lo)][Dp][2Dp]
    __half *rho_pl = nullptr; // rows l: [rho_re | rho_im]
    __half *w_pl = nullptr;   // rows k: [W_re | W_im]
    float *w32 = nullptr;     // [2][Dp][Dp]  W (re plane, im plane)
    float4 *rho_df[2] = {nullptr, nullptr};  // D x D {re_hi, re_lo, im_hi, im_lo}: rho, then V
    float4 *y_df = nullptr;                  // D x D stage buffer of the Strang step
    float4 *phase_df = nullptr;              // D: P_k as {re_hi, re_lo, im_hi, im_lo}
    float2 *damp_df = nullptr;               // D: dt/2 * d_k as {hi, lo}
    float2 *coef_df = nullptr;               // incoming jump entries: sqrt(dt) * coefficient
    int4 *in_tab = nullptr;                  // padded incoming table (rows with <= kInMax entries)
    int4 *jtab = nullptr;                    // per-jump incoming table (at most kInMax jumps)
    int nj = 0;
    double scale_delta = 1.0, scale_rho = 1.0, scale_w = 1.0;
    int batch_bn1 = kTcBNMax, batch_bn2 = kTcBNMax;  // tile widths of the grouped launches (qed_autotune_batched)
};

namespace {

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------ set-up kernels
__device__ __forceinline__ void split_half3(double x, __half &hi, __half &mid, __half &lo) {
    hi = __double2half(x);
    double r = x - (double)__half2float(hi);
    mid = __double2half(r);
    lo = __double2half(r - (double)__half2float(mid));
}

// Delta = P_k^-1 U_kl - delta_kl: conj(P_k) U_kl for the unit phases of U = exp(-i H dt)
// (unit != 0), conj(P_k) U_kl / |P_k|^2 for the damped phases of the effective step
__global__ void make_delta_kernel(int64_t D, const double2 *U, const double2 *P, double2 *Dl, int unit) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    int64_t k = idx / D, l = idx % D;
    double2 u = U[idx], p = P[k];
    double2 d = make_double2(p.x * u.x + p.y * u.y, p.x * u.y - p.y * u.x);
    if (!unit) {
        const double inv = 1.0 / (p.x * p.x + p.y * p.y);
        d.x *= inv;
        d.y *= inv;
    }
    if (k == l) d.x -= 1.0;
    Dl[idx] = d;
}

// a1 = [[Dre, Dim], [Dim, -Dre]] and b2 = [[Dre, Dim], [-Dim, Dre]] (2Dp x 2Dp) as three
// FP16 planes (hi, mid, lo), about 33 significant bits.  b2's rows are GEMM2's output
// columns; they are stored in groups of 128 = [the re rows of 64 consecutive n | the im rows
// of the same n], so that one 128-wide output tile holds X_re and X_im of 64 columns.
__global__ void static_planes_kernel(int64_t D, int64_t Dp, const double2 *Dl, double s, __half *a1, __half *b2) {
    const int64_t W2 = 2 * Dp;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= W2 * W2) return;
    int64_t r = idx / W2, c = idx % W2;
    int64_t cm = c % Dp;
    bool clo = c >= Dp;
    int64_t rk = r % Dp;                             // a1: row r = plane (r >= Dp), index r % Dp
    bool rlo = r >= Dp;
    int64_t rkb = 64 * (r / 128) + (r % 64);         // b2: column group r / 128, part (r % 128) / 64
    bool rlob = (r % 128) >= 64;
    double va = 0.0, vb = 0.0;
    if (rk < D && cm < D) {
        double2 d = Dl[rk * D + cm];
        if (!rlo && !clo) va = d.x;
        else if (!rlo && clo) va = d.y;
        else if (rlo && !clo) va = d.y;
        else va = -d.x;
    }
    if (rkb < D && cm < D) {
        double2 d = Dl[rkb * D + cm];
        if (!rlob && !clo) vb = d.x;
        else if (!rlob && clo) vb = d.y;
        else if (rlob && !clo) vb = -d.y;
        else vb = d.x;
    }
    __half h, md, l;
    split_half3(va * s, h, md, l);
    a1[idx] = h;
    a1[W2 * W2 + idx] = md;
    a1[2 * W2 * W2 + idx] = l;
    split_half3(vb * s, h, md, l);
    b2[idx] = h;
    b2[W2 * W2 + idx] = md;
    b2[2 * W2 * W2 + idx] = l;
}

// ------------------------------------------------------------------ per-evolve kernels
// caller rho (FP64) -> double-float state and the FP16 planes of GEMM1's B operand
__global__ void import_kernel(int64_t D, int64_t Dp, const double2 *rho, float s, float4 *st, __half *pl) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.y;
    if (n >= D) return;
    const double2 v = rho[m * D + n];
    const float rh = (float)v.x, ih = (float)v.y;
    const df re = {rh, (float)(v.x - (double)rh)}, im = {ih, (float)(v.y - (double)ih)};
    st[m * D + n] = make_float4(re.hi, re.lo, im.hi, im.lo);
    const int64_t plane = Dp * 2 * Dp;
    __half h, l;
    df_to_half2(re, s, h, l);
    pl[m * 2 * Dp + n] = h;
    pl[plane + m * 2 * Dp + n] = l;
    df_to_half2(im, s, h, l);
    pl[m * 2 * Dp + Dp + n] = h;
    pl[plane + m * 2 * Dp + Dp + n] = l;
}

// FP16 planes of GEMM1's B operand from the double-float state
__global__ void planes_from_state_kernel(int64_t D, int64_t Dp, const float4 *st, float s, __half *pl) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.y;
    if (n >= D) return;
    const float4 v = st[m * D + n];
    const int64_t plane = Dp * 2 * Dp;
    __half h, l;
    df_to_half2({v.x, v.y}, s, h, l);
    pl[m * 2 * Dp + n] = h;
    pl[plane + m * 2 * Dp + n] = l;
    df_to_half2({v.z, v.w}, s, h, l);
    pl[m * 2 * Dp + Dp + n] = h;
    pl[plane + m * 2 * Dp + Dp + n] = l;
}

// The split path's precondition on the caller's rho: Hermitian (its GEMM1 operand is the
// row-major rho read as rho^T = conj(rho), and X = W Delta^+ is formed as a Hermitian
// matrix) and of unit trace (the FP16 scale assumes |rho_mn| <= 1 and the renormalisation
// divides by the trace).  One thread per pair m <= n; block 0 also sums the diagonal.
__global__ void __launch_bounds__(256) check_density_kernel(int64_t D, const double2 *rho, uint32_t *err,
                                                             int unit_trace) {
    __shared__ double part[256];
    const int t = threadIdx.y * 32 + threadIdx.x;
    const int64_t n = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t m = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (m < D && n < D && n >= m) {
        const double2 a = rho[m * D + n], b = rho[n * D + m];
        const double dr = fabs(a.x - b.x), di = fabs(a.y + b.y);
        if (!(dr <= kDensityHermTol) || !(di <= kDensityHermTol)) atomicOr(err, kErrNotDensity);
    }
    if (blockIdx.x != 0 || blockIdx.y != 0) return;
    double s = 0.0;
    for (int64_t k = t; k < D; k += 256) s += rho[k * D + k].x;
    part[t] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) part[t] += part[t + h];
        __syncthreads();
    }
    const bool trace_ok = unit_trace ? fabs(part[0] - 1.0) <= kDensityTraceTol
                                     : (part[0] > 0.0 && part[0] <= 1.0 + kDensityTraceTol);
    if (t == 0 && !trace_ok) atomicOr(err, kErrNotDensity);
}

__global__ void export_kernel(int64_t D, const float4 *st, double2 *rho) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    const float4 v = st[idx];
    rho[idx] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// The Lindblad term of Eq. (3) as an update of the double-float buffers:
//   out_mn = B_mn + f [ -(dt/2)(d_m + d_n) X_mn + dt sum_j c_j(m) c_j(n) X[src_j(m), src_j(n)] ],
// f a power of two (exact).  The correction (relative size dt gamma) is formed to FP32
// accuracy and added to the double-float B.  With X = B = V, f = 1 and out = rho this is
// the Euler step of the Lie splitting; with f = 1/4 and 1/2 it gives the two stages of the
// explicit midpoint rule of the Strang splitting.  Optionally writes the FP16 planes of out
// (the next GEMM1's operand).  Buffers are chosen by index: 0 rho, 1 V, 2 the stage buffer.
__device__ __forceinline__ float4 *state_buf(const InstDesc &a, int sel) {
    return sel == 0 ? a.rho : (sel == 1 ? a.V : a.Y);
}

// A pair of long incoming lists (many jumps into one state, e.g. every leak into the
// vacuum): the whole warp (blockDim.x == 32, every lane present) shares the merge of each
// such pair.  Lanes take every 32nd entry of the shorter list and find its jump in the
// longer one by bisection; the owner lane gets the sum of c_p c_q X[src_p, src_q] (dt
// included in the coefficients) added to (gr, gi).  Returns whether this lane's own pair
// was handled.  Kept out of line so that the common path keeps its registers.
__device__ __noinline__ bool long_merge_df(uint32_t *err, int64_t D, const int32_t *in_jump, const int32_t *in_src,
                                           const float2 *coef, const float4 *X, int p, int pe, int q, int qe,
                                           float &gr, float &gi) {
    const bool is_long = pe > p && qe > q && (pe - p) + (qe - q) > kLongMerge;
    unsigned longs = __ballot_sync(0xffffffffu, is_long);
    const int lane = threadIdx.x;
    while (longs) {
        const int owner = __ffs(longs) - 1;
        longs &= longs - 1;
        const int op = __shfl_sync(0xffffffffu, p, owner), ope = __shfl_sync(0xffffffffu, pe, owner);
        const int oq = __shfl_sync(0xffffffffu, q, owner), oqe = __shfl_sync(0xffffffffu, qe, owner);
        const bool m_short = ope - op <= oqe - oq;
        const int s0 = m_short ? op : oq, s1 = m_short ? ope : oqe;
        const int l0 = m_short ? oq : op, l1 = m_short ? oqe : ope;
        float sr = 0.f, si = 0.f;
        for (int e = s0 + lane; e < s1; e += 32) {
            const int j = in_jump[e];
            int lo = l0, hi = l1;  // first entry of the longer list with jump >= j
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (in_jump[mid] < j)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const int ep = m_short ? e : lo, eq = m_short ? lo : e;  // row m's entry, row n's
            if (lo < l1 && in_jump[lo] == j &&
                qed_check(err, in_src[ep] >= 0 && in_src[ep] < D && in_src[eq] >= 0 && in_src[eq] < D)) {
                const float2 cp = coef[ep], cq = coef[eq];
                const df c = df_mul({cp.x, cp.y}, {cq.x, cq.y});
                const float4 u = X[(int64_t)in_src[ep] * D + in_src[eq]];
                const float ur = u.x + u.y, ui = u.z + u.w;
                sr = __fmaf_rn(c.hi, ur, __fmaf_rn(c.lo, ur, sr));
                si = __fmaf_rn(c.hi, ui, __fmaf_rn(c.lo, ui, si));
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == owner) {
            gr += sr;
            gi += si;
        }
    }
    return is_long;
}

// Rows of one element block: a block of 32 x 8 threads updates 32 columns and 8 kRows rows;
// thread (x, y) takes the rows 8 r + y, r < kRows, of its column, so the column's jump
// entries are read once for kRows elements and their loads are in flight together.
constexpr int kRows = 2;

// The output of one element: out = B + f (dt L(X))_mn with the accumulated increment (gr, gi),
// written as a double-float, and its FP16 planes when asked for.
template <bool LIE>
__device__ __forceinline__ void lindblad_store(const InstDesc &a, float4 *O, int64_t m, int64_t n, const cdf &b,
                                               float f, float gr, float gi, bool planes) {
    const int64_t D = a.D;
    cdf out;
    out.re = df_add_f(b.re, LIE ? gr : f * gr);
    out.im = df_add_f(b.im, LIE ? gi : f * gi);
    O[m * D + n] = store_cdf(out);
    if (!LIE && !planes) return;
    const int64_t plane = a.Dp * 2 * a.Dp;
    __half h, l;
    df_to_half2(out.re, a.s_rho, h, l);
    a.rho_pl[m * 2 * a.Dp + n] = h;
    a.rho_pl[plane + m * 2 * a.Dp + n] = l;
    df_to_half2(out.im, a.s_rho, h, l);
    a.rho_pl[m * 2 * a.Dp + a.Dp + n] = h;
    a.rho_pl[plane + m * 2 * a.Dp + a.Dp + n] = l;
}

// -(d_m + d_n) dt/2 X_mn in FP32 (d from the double-float damping table)
__device__ __forceinline__ void damping_term(float2 dm, float2 dn, const cdf &v, float &gr, float &gi) {
    const df dl = df_add({dm.x, dm.y}, {dn.x, dn.y});
    gr = -__fmaf_rn(dl.hi, v.re.hi, __fmaf_rn(dl.hi, v.re.lo, dl.lo * v.re.hi));
    gi = -__fmaf_rn(dl.hi, v.im.hi, __fmaf_rn(dl.hi, v.im.lo, dl.lo * v.im.hi));
}

template <bool LIE>
__device__ __forceinline__ void lindblad_update(const TileItem *__restrict__ tiles,
                                                const InstDesc *__restrict__ descs, int xsel, int bsel, int osel,
                                                float f, bool planes, const float4 *X_only = nullptr,
                                                float4 *O_only = nullptr) {
    // set-up tables (damping, padded jump rows) are read while the previous kernel finishes
    const TileItem it = tiles[blockIdx.x];
    const InstDesc a = descs[it.inst];
    const int64_t D = a.D;
    const int64_t n = (int64_t)it.bx * 32 + threadIdx.x;
    const int64_t m0 = (int64_t)it.by * (8 * kRows) + threadIdx.y;
    const bool n_in = n < D;
    const int64_t nc = n_in ? n : 0;
    const float2 dn = a.damp[nc];
    // X_only: out = f dt L(X_only) into O_only (B = 0), for buffers outside the model
    const float4 *X = X_only ? X_only : (LIE ? a.V : state_buf(a, xsel));
    const float4 *B = X_only ? nullptr : (LIE ? a.V : state_buf(a, bsel));
    float4 *O = X_only ? O_only : (LIE ? a.rho : state_buf(a, osel));
    if (a.jtab) {
        // incoming entries by jump: element (m, n) gets c_j(m) c_j(n) X[src_j(m), src_j(n)] for
        // every jump j with an entry in both rows (row entries warp-uniform, column entries
        // read once for the thread's kRows rows)
        const int nj = a.nj;
        int4 tn[kInMax], tm[kRows][kInMax];
        float2 dm[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int64_t m = m0 + 8 * r, mc = m < D ? m : 0;
            dm[r] = a.damp[mc];
#pragma unroll
            for (int j = 0; j < kInMax; ++j)
                tm[r][j] = j < nj ? a.jtab[mc * kInMax + j] : make_int4(-1, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < kInMax; ++j) tn[j] = j < nj ? a.jtab[nc * kInMax + j] : make_int4(-1, 0, 0, 0);
        pdl_wait();
        pdl_trigger();
        float4 v[kRows], u[kRows][kInMax], bv[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int64_t m = m0 + 8 * r;
            const bool inside = m < D && n_in;
            v[r] = X[(inside ? m : 0) * D + nc];
            // the base of a Strang stage comes with the gathers
            if (!LIE) bv[r] = B ? B[(inside ? m : 0) * D + nc] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < kInMax; ++j) {
                const bool hit = inside && tm[r][j].x >= 0 && tn[j].x >= 0 &&
                                 qed_check(a.err, tm[r][j].x < D && tn[j].x < D);
                u[r][j] = hit ? X[(int64_t)tm[r][j].x * D + tn[j].x] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int64_t m = m0 + 8 * r;
            if (!(m < D && n_in)) continue;
            const cdf vv = load_cdf(v[r]);
            float gr, gi;
            damping_term(dm[r], dn, vv, gr, gi);
#pragma unroll
            for (int j = 0; j < kInMax; ++j) {
                if (!(tm[r][j].x >= 0 && tn[j].x >= 0)) continue;
                const df c = df_mul({__int_as_float(tm[r][j].y), __int_as_float(tm[r][j].z)},
                                    {__int_as_float(tn[j].y), __int_as_float(tn[j].z)});
                const float ur = u[r][j].x + u[r][j].y, ui = u[r][j].z + u[r][j].w;
                gr = __fmaf_rn(c.hi, ur, __fmaf_rn(c.lo, ur, gr));
                gi = __fmaf_rn(c.hi, ui, __fmaf_rn(c.lo, ui, gi));
            }
            const cdf b = LIE ? vv : load_cdf(bv[r]);
            lindblad_store<LIE>(a, O, m, n, b, f, gr, gi, planes);
        }
        return;
    }
    if (a.in_tab) {
        // padded incoming tables: the row entries are the same for the whole warp (one row per
        // warp and r), the column's for all kRows rows of the thread
        int4 en[kInMax], em[kRows][kInMax];
        float2 dm[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int64_t m = m0 + 8 * r, mc = m < D ? m : 0;
            dm[r] = a.damp[mc];
#pragma unroll
            for (int i = 0; i < kInMax; ++i) em[r][i] = a.in_tab[mc * kInMax + i];
        }
#pragma unroll
        for (int i = 0; i < kInMax; ++i) en[i] = a.in_tab[nc * kInMax + i];
        pdl_wait();
        pdl_trigger();
        // every load of the kRows elements issued before the first use
        float4 v[kRows], u[kRows][kInMax], bv[kRows];
        float2 cq[kRows][kInMax];
        bool hit[kRows][kInMax];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int64_t m = m0 + 8 * r;
            const bool inside = m < D && n_in;
            if (!LIE) bv[r] = B ? B[(inside ? m : 0) * D + nc] : make_float4(0.f, 0.f, 0.f, 0.f);
            v[r] = X[(inside ? m : 0) * D + nc];
#pragma unroll
            for (int i = 0; i < kInMax; ++i) {
                int src = 0;
                float2 c2 = make_float2(0.f, 0.f);
                bool h = false;
#pragma unroll
                for (int j = 0; j < kInMax; ++j)
                    if (en[j].x == em[r][i].x) {
                        h = true;
                        src = en[j].y;
                        c2 = make_float2(__int_as_float(en[j].z), __int_as_float(en[j].w));
                    }
                hit[r][i] = h && em[r][i].x != kNoJump && inside &&
                            qed_check(a.err, em[r][i].y >= 0 && em[r][i].y < D && src >= 0 && src < D);
                cq[r][i] = c2;
                u[r][i] = hit[r][i] ? X[(int64_t)em[r][i].y * D + src] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int64_t m = m0 + 8 * r;
            if (!(m < D && n_in)) continue;
            const cdf vv = load_cdf(v[r]);
            float gr, gi;
            damping_term(dm[r], dn, vv, gr, gi);
#pragma unroll
            for (int i = 0; i < kInMax; ++i) {
                if (!hit[r][i]) continue;
                const df c = df_mul({__int_as_float(em[r][i].z), __int_as_float(em[r][i].w)}, {cq[r][i].x, cq[r][i].y});
                const float ur = u[r][i].x + u[r][i].y, ui = u[r][i].z + u[r][i].w;
                gr = __fmaf_rn(c.hi, ur, __fmaf_rn(c.lo, ur, gr));
                gi = __fmaf_rn(c.hi, ui, __fmaf_rn(c.lo, ui, gi));
            }
            const cdf b = LIE ? vv : load_cdf(bv[r]);
            lindblad_store<LIE>(a, O, m, n, b, f, gr, gi, planes);
        }
        return;
    }
    // incoming lists: the damping rates and list bounds of the thread's rows (static
    // tables) before the dependency wait, the rows' V elements together after it, then the
    // rows' merges one after another; lanes outside the matrix stay to the end of every row
    // (with clamped indices, no stores), since the warp shares the merge of long jump lists
    float2 dmr[kRows];
    int pr[kRows], per[kRows];
    const int q0 = n_in ? a.in_ptr[n] : 0, qe0 = n_in ? a.in_ptr[n + 1] : 0;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int64_t m = m0 + 8 * r;
        const bool inside = m < D && n_in;
        dmr[r] = a.damp[m < D ? m : 0];
        pr[r] = inside ? a.in_ptr[m] : 0;
        per[r] = inside ? a.in_ptr[m + 1] : 0;
    }
    pdl_wait();
    pdl_trigger();
    float4 vr[kRows], bv[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int64_t m = m0 + 8 * r;
        vr[r] = X[(m < D && n_in ? m : 0) * D + nc];
        if (!LIE) bv[r] = B ? B[(m < D && n_in ? m : 0) * D + nc] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int64_t m = m0 + 8 * r;
        const bool inside = m < D && n_in;
        const cdf v = load_cdf(vr[r]);
        float gr, gi;
        damping_term(dmr[r], dn, v, gr, gi);
        int p = pr[r], pe = per[r];
        int q = inside ? q0 : 0, qe = inside ? qe0 : 0;
        // long lists: merged by the whole warp
        const bool is_long = long_merge_df(a.err, D, a.in_jump, a.in_src, a.coef, X, p, pe, q, qe, gr, gi);
        if (is_long) pe = p;  // done: skip the serial merge
        while (p < pe && q < qe) {  // jumps present in both incoming lists
            const int jp = a.in_jump[p], jq = a.in_jump[q];
            if (jp < jq) {
                ++p;
            } else if (jp > jq) {
                ++q;
            } else if (qed_check(a.err, a.in_src[p] >= 0 && a.in_src[p] < D && a.in_src[q] >= 0 && a.in_src[q] < D)) {
                const float2 cp = a.coef[p], cqq = a.coef[q];
                const df c = df_mul({cp.x, cp.y}, {cqq.x, cqq.y});  // dt c_j(m) c_j(n)
                const float4 uu = X[(int64_t)a.in_src[p] * D + a.in_src[q]];
                const float ur = uu.x + uu.y, ui = uu.z + uu.w;
                gr = __fmaf_rn(c.hi, ur, __fmaf_rn(c.lo, ur, gr));
                gi = __fmaf_rn(c.hi, ui, __fmaf_rn(c.lo, ui, gi));
                ++p;
                ++q;
            }
        }
        if (!inside) continue;
        const cdf b = LIE ? v : load_cdf(bv[r]);
        lindblad_store<LIE>(a, O, m, n, b, f, gr, gi, planes);
    }
}

// The Lie step's update (rho = V + dt L(V) and the next planes) for instances whose incoming
// entries are all in per-jump tables (at most kInMax jumps of monomial form).  The block's
// row and column entries and damping rates are staged in shared memory first, so a thread
// keeps only its kRows elements' loads in registers; with 64 registers four blocks fit on an
// SM, and a dim-512 update (512 blocks) runs as one wave whose table reads overlap the
// previous kernel.
__global__ void __launch_bounds__(256, 4) dissipate_jt_kernel(const TileItem *__restrict__ tiles,
                                                           const InstDesc *__restrict__ descs) {
    constexpr int R = 8 * kRows;
    constexpr int JW = kInMax;
    __shared__ int4 s_row[R][JW], s_col[32][JW];
    __shared__ float2 s_dr[R], s_dc[32];
    const TileItem it = tiles[blockIdx.x];
    const InstDesc a = descs[it.inst];
    // element offsets in 32 bits: the split path holds dimensions below 65536 (split_create)
    const uint32_t D = (uint32_t)a.D;
    const int nj = a.nj;
    const uint32_t n0 = (uint32_t)it.bx * 32, m0 = (uint32_t)it.by * R;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // entries: the block's R rows, then its 32 columns, then both damping vectors
    for (int e = tid; e < (R + 32) * JW + R + 32; e += 256) {
        if (e < R * JW) {
            const int r = e / JW, j = e % JW;
            const uint32_t m = m0 + r;
            s_row[r][j] = j < nj && m < D ? a.jtab[m * JW + j] : make_int4(-1, 0, 0, 0);
        } else if (e < (R + 32) * JW) {
            const int c = (e - R * JW) / JW, j = e % JW;
            const uint32_t n = n0 + c;
            s_col[c][j] = j < nj && n < D ? a.jtab[n * JW + j] : make_int4(-1, 0, 0, 0);
        } else if (e < (R + 32) * JW + R) {
            const int r = e - (R + 32) * JW;
            s_dr[r] = m0 + r < D ? a.damp[m0 + r] : make_float2(0.f, 0.f);
        } else {
            const int c = e - (R + 32) * JW - R;
            s_dc[c] = n0 + c < D ? a.damp[n0 + c] : make_float2(0.f, 0.f);
        }
    }
    const float4 *X = a.V;
    float4 *O = a.rho;
    __syncthreads();
    pdl_wait();
    pdl_trigger();
    const int tx = threadIdx.x;
    const uint32_t n = n0 + tx;
    // the jump terms are formed in FP32 (their size is dt gamma of the result), so each
    // gathered element contributes only the leading words of its real and imaginary parts
    float4 v[kRows];
    float ur[kRows][JW], ui[kRows][JW];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int rr = threadIdx.y + 8 * r;
        const uint32_t m = m0 + rr;
        const bool inside = m < D && n < D;
        v[r] = inside ? X[m * D + n] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < JW; ++j) {
            const int sm = s_row[rr][j].x, sn = s_col[tx][j].x;
            const bool hit = inside && sm >= 0 && sn >= 0 && qed_check(a.err, (uint32_t)sm < D && (uint32_t)sn < D);
            const float *src = (const float *)(X + ((uint32_t)sm * D + (uint32_t)sn));
            ur[r][j] = hit ? src[0] : 0.f;
            ui[r][j] = hit ? src[2] : 0.f;
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int rr = threadIdx.y + 8 * r;
        const uint32_t m = m0 + rr;
        if (!(m < D && n < D)) continue;
        const cdf vv = load_cdf(v[r]);
        float gr, gi;
        damping_term(s_dr[rr], s_dc[tx], vv, gr, gi);
#pragma unroll
        for (int j = 0; j < JW; ++j) {
            const int4 em = s_row[rr][j], en = s_col[tx][j];
            if (!(em.x >= 0 && en.x >= 0)) continue;
            const df c = df_mul({__int_as_float(em.y), __int_as_float(em.z)}, {__int_as_float(en.y), __int_as_float(en.z)});
            gr = __fmaf_rn(c.hi, ur[r][j], __fmaf_rn(c.lo, ur[r][j], gr));
            gi = __fmaf_rn(c.hi, ui[r][j], __fmaf_rn(c.lo, ui[r][j], gi));
        }
        lindblad_store<true>(a, O, m, n, vv, 1.f, gr, gi, true);
    }
}

// Lie step: rho = V + dt L(V), and the next planes.
__global__ void __launch_bounds__(256, 2) dissipate_df_kernel(const TileItem *__restrict__ tiles,
                                                           const InstDesc *__restrict__ descs) {
    lindblad_update<true>(tiles, descs, 1, 1, 0, 1.f, true);
}

// One stage of the Strang step: out = B + f dt L(X).
__global__ void __launch_bounds__(256, 2) lindblad_df_kernel(const TileItem *__restrict__ tiles,
                                                          const InstDesc *__restrict__ descs, int xsel, int bsel,
                                                          int osel, float f, int planes) {
    lindblad_update<false>(tiles, descs, xsel, bsel, osel, f, planes != 0);
}

// out = dt L(X) for a double-float buffer X of a single model (the adjoint's rate terms).
__global__ void __launch_bounds__(256, 2) lindblad_apply_df_kernel(const TileItem *__restrict__ tiles,
                                                                const InstDesc *__restrict__ descs,
                                                                const float4 *X, float4 *out) {
    lindblad_update<false>(tiles, descs, 0, 0, 0, 1.f, false, X, out);
}

__global__ void __launch_bounds__(256) observables_df_kernel(int64_t D, const float4 *st, const double *w,
                                                             const int32_t *ids, double *out) {
    __shared__ double part[256];
    const int o = blockIdx.x;
    const int id = ids[o];
    const int t = threadIdx.x;
    double s = 0.0;
    if (id < D) {
        if (t == 0) {
            const float4 v = st[(int64_t)id * D + id];
            s = (double)v.x + (double)v.y;
        }
    } else {
        const double *wr = w + (int64_t)(id - D) * D;
        for (int64_t k = t; k < D; k += blockDim.x) {
            const float4 v = st[k * D + k];
            s += wr[k] * ((double)v.x + (double)v.y);
        }
    }
    part[t] = s;
    __syncthreads();
    for (int st2 = blockDim.x / 2; st2 > 0; st2 >>= 1) {
        if (t < st2) part[t] += part[t + st2];
        __syncthreads();
    }
    if (t == 0) out[o] = part[0];
}

__global__ void __launch_bounds__(1024) trace_df_kernel(int64_t D, const float4 *st, double *tr, uint32_t *err) {
    __shared__ double part[1024];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t k = t; k < D; k += blockDim.x) {
        const float4 v = st[k * D + k];
        s += (double)v.x + (double)v.y;
    }
    part[t] = s;
    __syncthreads();
    for (int st2 = blockDim.x / 2; st2 > 0; st2 >>= 1) {
        if (t < st2) part[t] += part[t + st2];
        __syncthreads();
    }
    if (t == 0) {
        *tr = part[0];
        if (!isfinite(part[0]) || !(part[0] > 0.0)) atomicOr(err, kErrNonFinite);
    }
}

// rho <- (rho + rho^+) / (2 tr rho) (divide != 0) or (rho + rho^+) / 2 on the double-float
// state (FP64 arithmetic; it runs once every `renorm_every` steps), then the FP16 planes
// again.
__global__ void symmetrise_df_kernel(int64_t D, int64_t Dp, float4 *st, const double *tr, const uint32_t *err,
                                     float s_rho, __half *pl, int divide) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= D || j >= D || j < i) return;
    if (*err & kErrNonFinite) return;
    const double inv = divide ? 1.0 / *tr : 1.0;
    const float4 a = st[i * D + j], b = st[j * D + i];
    double re = 0.5 * (((double)a.x + (double)a.y) + ((double)b.x + (double)b.y)) * inv;
    double im = 0.5 * (((double)a.z + (double)a.w) - ((double)b.z + (double)b.w)) * inv;
    if (i == j) im = 0.0;
    const float rh = (float)re, ih = (float)im;
    const df dre = {rh, (float)(re - (double)rh)}, dim = {ih, (float)(im - (double)ih)};
    st[i * D + j] = make_float4(dre.hi, dre.lo, dim.hi, dim.lo);
    st[j * D + i] = make_float4(dre.hi, dre.lo, -dim.hi, -dim.lo);
    const int64_t plane = Dp * 2 * Dp;
    __half h, l;
    df_to_half2(dre, s_rho, h, l);
    pl[i * 2 * Dp + j] = h;
    pl[plane + i * 2 * Dp + j] = l;
    pl[j * 2 * Dp + i] = h;
    pl[plane + j * 2 * Dp + i] = l;
    df_to_half2(dim, s_rho, h, l);
    pl[i * 2 * Dp + Dp + j] = h;
    pl[plane + i * 2 * Dp + Dp + j] = l;
    df_to_half2(df_neg(dim), s_rho, h, l);
    pl[j * 2 * Dp + Dp + i] = h;
    pl[plane + j * 2 * Dp + Dp + i] = l;
}

double pow2_scale(double maxabs, int target_exp) {
    if (!(maxabs > 0.0) || !std::isfinite(maxabs)) return 1.0;
    int e = (int)std::ceil(std::log2(maxabs));
    return std::ldexp(1.0, target_exp - e);
}

template <class T>
qed_status alloc(T **p, size_t count) {
    if (device_malloc((void **)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed for the split-precision buffers");
        return QED_ENOMEM;
    }
    return QED_OK;
}

#define SPLIT_TRY(expr)                 \
    do {                                \
        qed_status st_ = (expr);        \
        if (st_ != QED_OK) return st_;  \
    } while (0)

const TcSegs kSegs1 = {4, {0, 0, 1, 2, 0, 0}, {0, 1, 0, 0, 0, 0}};  // Delta(hi,mid,lo) x rho(hi,lo)
const TcSegs kSegs2 = {3, {0, 1, 0, 0, 0, 0}, {0, 0, 1, 0, 0, 0}};  // W(hi,lo) x Delta(hi,mid,lo)
const int kSeg1Pairs[8] = {0, 0, 0, 1, 1, 0, 2, 0};
const int kSeg2Pairs[6] = {0, 0, 1, 0, 0, 1};

template <class T>
qed_status upload(T **dst, const std::vector<T> &v) {
    SPLIT_TRY(alloc(dst, std::max<size_t>(v.size(), 1)));
    if (!v.empty()) QED_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return QED_OK;
}

// The plans of a model's two products: GEMM1 [W_re; W_im] = A1 . rho^T (2Dp x Dp, K 2Dp, four
// plane pairs), GEMM2 [X_re | X_im] = W . B2^T (Dp x 2Dp, K 2Dp, three plane pairs).  Widths and
// splits = CTAs per cluster (on-chip reduction of the split-K slices) as given, or 0 for the
// planner's rule (256-wide tiles once the tiles that run fill half the SMs).
bool plan_products(SplitState &S, TcGemm &g1, TcGemm &g2, int splits1, int bn1, int splits2, int bn2 = 0) {
    const int Dp = (int)S.Dp;
    if (bn2 == 0) {
        // GEMM2 runs only the tiles on or above the diagonal: nm (nm + 1) / 2 of them when 256
        // wide (nm = Dp / 128), which must fill half the SMs
        const int nm = Dp / kTcBM;
        bn2 = nm * (nm + 1) >= S.num_sms ? 256 : 128;
    }
    return tc_gemm_plan(g1, S.a1, 3, S.rho_pl, 2, 2 * Dp, Dp, 2 * Dp, 4, kSeg1Pairs, S.num_sms, splits1, bn1, true) &&
           tc_gemm_plan(g2, S.w_pl, 2, S.b2, 3, Dp, 2 * Dp, 2 * Dp, 3, kSeg2Pairs, S.num_sms, splits2, bn2, true);
}

// Descriptors, jobs and work lists of a batch.  With `single` set (one model on its own)
// the products keep their plans (split-K slices reduced inside clusters); in a batch every
// product runs unsplit, largest first, since the batch itself fills the GPU.  GEMM1 skips
// tiles that lie wholly in the zero padding (rows or columns >= D); GEMM2 runs the tiles on
// or above the diagonal only (its epilogue writes both halves of the Hermitian V).
qed_status build_batch(Batch &b, qed_model *const *ms, int n, bool single, int batch_bn1 = kTcBNMax,
                       int batch_bn2 = kTcBNMax) {
    b.release();
    b.n = n;
    b.scheme = ms[0]->scheme;
    for (int i = 1; i < n; ++i)
        if (ms[i]->scheme != b.scheme) {
            set_error("batched evolution: all models must use one time-stepping scheme");
            return QED_EINVAL;
        }
    std::vector<InstDesc> desc((size_t)n);
    std::vector<GemmJob> jobs1((size_t)n), jobs2((size_t)n);
    std::vector<CUtensorMap> maps((size_t)(4 * n));
    std::vector<GemmItem> it1, it2;
    std::vector<TileItem> et;
    for (int i = 0; i < n; ++i) {
        qed_model *m = ms[i];
        SplitState &S = *m->sp;
        InstDesc &d = desc[(size_t)i];
        const int64_t D = m->D, Dp = S.Dp;
        d.D = D;
        d.Dp = Dp;
        d.s_rho = (float)S.scale_rho;
        d.rho = S.rho_df[0];
        d.V = S.rho_df[1];
        d.Y = S.y_df;
        d.phase = S.phase_df;
        d.damp = S.damp_df;
        d.in_ptr = m->in_ptr;
        d.in_jump = m->in_jump;
        d.in_src = m->in_src;
        d.coef = S.coef_df;
        d.in_tab = S.in_tab;
        d.jtab = S.jtab;
        d.nj = S.nj;
        d.rho_pl = S.rho_pl;
        d.err = m->err;
        TcGemm bg1 = S.g1, bg2 = S.g2;
        if (!single && !plan_products(S, bg1, bg2, 1, batch_bn1, 1, batch_bn2)) return QED_ECUDA;
        auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
        if (!pow2(bg1.splits) || bg1.splits > kTcMaxCluster || !pow2(bg2.splits) || bg2.splits > kTcMaxClusterV ||
            (bg2.bn != 128 && bg2.bn != 256)) {
            set_error("split step: product plan outside the cluster epilogue's limits");
            return QED_EINVAL;
        }
        maps[(size_t)(4 * i + 0)] = bg1.a;
        maps[(size_t)(4 * i + 1)] = bg1.b;
        maps[(size_t)(4 * i + 2)] = bg2.a;
        maps[(size_t)(4 * i + 3)] = bg2.b;
        const TcGemm *gs[2] = {&bg1, &bg2};
        GemmJob *js[2] = {&jobs1[(size_t)i], &jobs2[(size_t)i]};
        for (int q = 0; q < 2; ++q) {
            const TcGemm &g = *gs[q];
            GemmJob &j = *js[q];
            j.M = g.M;
            j.N = g.N;
            j.kb_per_seg = g.K / kTcBK;
            j.kb_per_split = g.kb_per_split;
            j.out = nullptr;
            j.gate = m->gate_armed ? m->gate : nullptr;
            j.gate_budget = m->gate_budget;
            j.mode = q == 0 ? kEpiW : kEpiV;
            j.tx_bytes = tc_stage_tx_bytes(g, j.mode);
            j.epi = TcEpilogue();
            j.epi.D = D;
            j.epi.Dp = Dp;
            j.epi.w32 = S.w32;
            if (q == 0) {
                j.epi.inv = (float)(1.0 / (S.scale_delta * S.scale_rho));
                j.epi.s_w = (float)S.scale_w;
                j.epi.w_pl = S.w_pl;
            } else {
                j.epi.inv = (float)(1.0 / (S.scale_w * S.scale_delta));
                j.epi.rho = S.rho_df[0];
                j.epi.phase = S.phase_df;
                j.epi.V = S.rho_df[1];
            }
            if (i == 0) {
                (q == 0 ? b.cs1 : b.cs2) = g.splits;
                (q == 0 ? b.bn1 : b.bn2) = g.bn;
            } else if (g.splits != (q == 0 ? b.cs1 : b.cs2) || g.bn != (q == 0 ? b.bn1 : b.bn2)) {
                set_error("batched evolution: every instance of a launch needs the same tile plan");
                return QED_EINVAL;
            }
        }
        // GEMM1 tiles: 128 rows of [W_re; W_im] x bn1 columns; wholly-padding tiles skipped
        for (int tm = 0; tm < bg1.M / kTcBM; ++tm) {
            if ((tm * kTcBM) % Dp >= D) continue;
            for (int tn = 0; tn * bg1.bn < bg1.N; ++tn) {
                if ((int64_t)tn * bg1.bn >= D) continue;
                for (int sp = 0; sp < bg1.splits; ++sp) it1.push_back({i, tm, tn, sp});
            }
        }
        // GEMM2 tiles: 128 rows m x (64 c2) complex columns n, on or above the diagonal
        const int c2 = bg2.bn / 128;
        for (int tm = 0; tm < bg2.M / kTcBM; ++tm) {
            if ((int64_t)tm * kTcBM >= D) continue;
            for (int tj = 2 * tm / c2; tj < bg2.N / bg2.bn; ++tj) {
                if ((int64_t)tj * 64 * c2 >= D) continue;
                for (int sp = 0; sp < bg2.splits; ++sp) it2.push_back({i, tm, tj, sp});
            }
        }
        for (int by = 0; by < (D + 8 * kRows - 1) / (8 * kRows); ++by)
            for (int bx = 0; bx < (D + 31) / 32; ++bx) et.push_back({i, bx, by, 0});
    }
    if (!single) {
        // longest products first, so the tail of the grouped launch is short (unsplit:
        // every item is a cluster of one)
        auto by_cost = [&](const GemmItem &x, const GemmItem &y) {
            return jobs1[(size_t)x.job].kb_per_seg > jobs1[(size_t)y.job].kb_per_seg;
        };
        std::stable_sort(it1.begin(), it1.end(), by_cost);
        std::stable_sort(it2.begin(), it2.end(), by_cost);
    }
    SPLIT_TRY(upload(&b.maps, maps));
    for (int i = 0; i < n; ++i) {
        jobs1[(size_t)i].map_a = b.maps + 4 * i + 0;
        jobs1[(size_t)i].map_b = b.maps + 4 * i + 1;
        jobs2[(size_t)i].map_a = b.maps + 4 * i + 2;
        jobs2[(size_t)i].map_b = b.maps + 4 * i + 3;
    }
    SPLIT_TRY(upload(&b.desc, desc));
    SPLIT_TRY(upload(&b.jobs1, jobs1));
    SPLIT_TRY(upload(&b.jobs2, jobs2));
    SPLIT_TRY(upload(&b.items1, it1));
    SPLIT_TRY(upload(&b.items2, it2));
    SPLIT_TRY(upload(&b.etiles, et));
    b.n_items1 = (int)it1.size();
    b.n_items2 = (int)it2.size();
    b.n_etiles = (int)et.size();
    b.jt = std::all_of(desc.begin(), desc.end(), [](const InstDesc &d) { return d.jtab != nullptr; });
    if (single) {
        SplitState &S = *ms[0]->sp;
        b.single = true;
        b.D = ms[0]->D;
        b.g1 = S.g1;
        b.g2 = S.g2;
        b.j1 = jobs1[0];
        b.j2 = jobs2[0];
        if (tc_gemm_single_ctas(b.g1, kEpiW, b.D) * 1 != b.n_items1 ||
            tc_gemm_single_ctas(b.g2, kEpiV, b.D) != b.n_items2) {
            set_error("split step: tile lists of the single-model launch disagree");
            return QED_ECUDA;
        }
    }
    if (!tc_gemm_prepare_grouped()) return QED_ECUDA;
    return QED_OK;
}

void launch_gemm1(const Batch &b, uint32_t *err, cudaStream_t s) {
    if (b.single)
        tc_gemm_single_launch(b.g1, b.j1, kSegs1, b.D, err, s);
    else
        tc_gemm_grouped_launch(b.items1, b.n_items1, b.jobs1, kSegs1, b.bn1, kEpiW, b.cs1, err, s);
}
void launch_gemm2(const Batch &b, uint32_t *err, cudaStream_t s) {
    if (b.single)
        tc_gemm_single_launch(b.g2, b.j2, kSegs2, b.D, err, s);
    else
        tc_gemm_grouped_launch(b.items2, b.n_items2, b.jobs2, kSegs2, b.bn2, kEpiV, b.cs2, err, s);
}
void launch_dissipate(const Batch &b, cudaStream_t s) {
    launch_pdl(b.jt ? dissipate_jt_kernel : dissipate_df_kernel, dim3(b.n_etiles), dim3(32, 8), 0, s, b.etiles,
               b.desc);
    count_launches(1);
}
void launch_lindblad(const Batch &b, int xsel, int bsel, int osel, float f, int planes, cudaStream_t s) {
    launch_pdl(lindblad_df_kernel, dim3(b.n_etiles), dim3(32, 8), 0, s, b.etiles, b.desc, xsel, bsel, osel, f,
               planes);
    count_launches(1);
}
// The two stages of one explicit-midpoint half step of the Lindblad flow (step dt/2):
// Y = X + (dt/4) L(X), then rho = X + (dt/2) L(Y), with its planes when the next kernel is
// GEMM1 (the leading half step; the trailing one is always followed by the next leading
// half step, a renormalisation or the end of the run, none of which read the planes).
void launch_half_lindblad(const Batch &b, int xsel, int planes, cudaStream_t s) {
    launch_lindblad(b, xsel, xsel, 2, 0.25f, 0, s);
    launch_lindblad(b, 2, xsel, 0, 0.5f, planes, s);
}

}  // namespace

qed_status split_prepare(qed_model *m, cudaStream_t s) {
    const int64_t D = m->D;
    const int64_t Dp = (D + kTcBM - 1) / kTcBM * kTcBM;
    const size_t W2 = (size_t)(2 * Dp) * (size_t)(2 * Dp);
    if (D >= 65536) {
        // (its buffers would exceed any device's memory; the Lindblad kernels index in 32 bits)
        set_error("split precision: dimensions up to 65535");
        return QED_EINVAL;
    }
    if (!m->sp) {
        m->sp = new SplitState();
        SplitState &S = *m->sp;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&S.num_sms, cudaDevAttrMultiProcessorCount, dev);
        S.Dp = Dp;
        const size_t pl = (size_t)Dp * 2 * Dp * 2;
        SPLIT_TRY(alloc(&S.a1, W2 * 3));
        SPLIT_TRY(alloc(&S.b2, W2 * 3));
        SPLIT_TRY(alloc(&S.rho_pl, pl));
        SPLIT_TRY(alloc(&S.w_pl, pl));
        SPLIT_TRY(alloc(&S.w32, (size_t)2 * Dp * Dp));
        SPLIT_TRY(alloc(&S.rho_df[0], (size_t)(D * D)));
        SPLIT_TRY(alloc(&S.rho_df[1], (size_t)(D * D)));
        SPLIT_TRY(alloc(&S.y_df, (size_t)(D * D)));
        SPLIT_TRY(alloc(&S.phase_df, (size_t)D));
        // zero padding: tiles of GEMM1 that lie wholly in it are never written
        QED_CUDA_TRY(cudaMemset(S.rho_pl, 0, pl * sizeof(__half)));
        QED_CUDA_TRY(cudaMemset(S.w_pl, 0, pl * sizeof(__half)));
        QED_CUDA_TRY(cudaMemset(S.w32, 0, (size_t)2 * Dp * Dp * sizeof(float)));
        // the planner's split-K factors become the cluster sizes of the on-chip reduction
        static_assert(kTcMaxAutoSplits <= kTcMaxCluster, "plans must fit the cluster epilogues");
        if (!plan_products(S, S.g1, S.g2, 0, 0, 0)) return QED_ECUDA;

        SPLIT_TRY(alloc(&S.damp_df, (size_t)D));
        // sqrt(dt) * coefficient of the incoming jump entries as double-floats
        auto split_f = [](double x) { const float h = (float)x; return make_float2(h, (float)(x - (double)h)); };
        std::vector<double> coef((size_t)m->n_in);
        if (m->n_in > 0)
            QED_CUDA_TRY(cudaMemcpy(coef.data(), m->in_coef, (size_t)m->n_in * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<float2> cdf_((size_t)std::max<int64_t>(m->n_in, 1));
        for (int64_t e = 0; e < m->n_in; ++e) cdf_[(size_t)e] = split_f(std::sqrt(m->dt) * coef[(size_t)e]);
        SPLIT_TRY(alloc(&S.coef_df, cdf_.size()));
        QED_CUDA_TRY(cudaMemcpy(S.coef_df, cdf_.data(), cdf_.size() * sizeof(float2), cudaMemcpyHostToDevice));
        // the padded table when no row has more than kInMax incoming entries
        std::vector<int32_t> ptr((size_t)D + 1), jmp((size_t)std::max<int64_t>(m->n_in, 1)),
            src((size_t)std::max<int64_t>(m->n_in, 1));
        QED_CUDA_TRY(cudaMemcpy(ptr.data(), m->in_ptr, ptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (m->n_in > 0) {
            QED_CUDA_TRY(cudaMemcpy(jmp.data(), m->in_jump, (size_t)m->n_in * sizeof(int32_t), cudaMemcpyDeviceToHost));
            QED_CUDA_TRY(cudaMemcpy(src.data(), m->in_src, (size_t)m->n_in * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
        int32_t widest = 0;
        for (int64_t k = 0; k < D; ++k) widest = std::max(widest, ptr[(size_t)k + 1] - ptr[(size_t)k]);
        if (widest <= kInMax) {
            std::vector<int4> tab((size_t)D * kInMax, make_int4(kNoJump, 0, 0, 0));
            for (int64_t k = 0; k < D; ++k)
                for (int32_t e = ptr[(size_t)k]; e < ptr[(size_t)k + 1]; ++e) {
                    const float2 c = cdf_[(size_t)e];
                    int f_hi = 0, f_lo = 0;
                    std::memcpy(&f_hi, &c.x, 4);
                    std::memcpy(&f_lo, &c.y, 4);
                    tab[(size_t)(k * kInMax + (e - ptr[(size_t)k]))] = make_int4(jmp[(size_t)e], src[(size_t)e], f_hi, f_lo);
                }
            SPLIT_TRY(alloc(&S.in_tab, tab.size()));
            QED_CUDA_TRY(cudaMemcpy(S.in_tab, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice));
        }
        // with at most kInMax jumps, and (monomial operators) at most one incoming entry per
        // state and jump, the entries indexed by jump: the Lindblad kernels then read the
        // pairs (m, n) of each jump directly instead of matching the two rows' lists
        const int nj = (int)m->host.gamma.size();
        if (nj >= 1 && nj <= kInMax) {
            std::vector<int4> jt((size_t)D * kInMax, make_int4(-1, 0, 0, 0));
            bool unique = true;
            for (int64_t k = 0; k < D && unique; ++k)
                for (int32_t e = ptr[(size_t)k]; e < ptr[(size_t)k + 1]; ++e) {
                    int4 &slot = jt[(size_t)(k * kInMax + jmp[(size_t)e])];
                    if (slot.x >= 0) {
                        unique = false;
                        break;
                    }
                    const float2 c = cdf_[(size_t)e];
                    int f_hi = 0, f_lo = 0;
                    std::memcpy(&f_hi, &c.x, 4);
                    std::memcpy(&f_lo, &c.y, 4);
                    slot = make_int4(src[(size_t)e], f_hi, f_lo, 0);
                }
            if (unique) {
                SPLIT_TRY(alloc(&S.jtab, jt.size()));
                QED_CUDA_TRY(cudaMemcpy(S.jtab, jt.data(), jt.size() * sizeof(int4), cudaMemcpyHostToDevice));
                S.nj = nj;
            }
        }
    }
    SplitState &S = *m->sp;
    const bool eff = m->scheme == QED_SCHEME_EFFECTIVE;
    {
        // per-row phases P_k and dt/2 d_k (zero for the effective step, whose propagator holds
        // the anticommutator) as double-floats
        auto split_f = [](double x) { const float h = (float)x; return make_float2(h, (float)(x - (double)h)); };
        std::vector<double2> ph((size_t)D);
        QED_CUDA_TRY(cudaMemcpy(ph.data(), m->phase, (size_t)D * sizeof(double2), cudaMemcpyDeviceToHost));
        std::vector<float4> pdf((size_t)D);
        for (int64_t k = 0; k < D; ++k) {
            const float rh = (float)ph[(size_t)k].x, ih = (float)ph[(size_t)k].y;
            pdf[(size_t)k] = make_float4(rh, (float)(ph[(size_t)k].x - rh), ih, (float)(ph[(size_t)k].y - ih));
        }
        QED_CUDA_TRY(cudaMemcpy(S.phase_df, pdf.data(), (size_t)D * sizeof(float4), cudaMemcpyHostToDevice));
        std::vector<double> anti((size_t)D);
        QED_CUDA_TRY(cudaMemcpy(anti.data(), m->anti, (size_t)D * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<float2> damp((size_t)D);
        for (int64_t k = 0; k < D; ++k) damp[(size_t)k] = split_f(eff ? 0.0 : 0.5 * m->dt * anti[(size_t)k]);
        QED_CUDA_TRY(cudaMemcpy(S.damp_df, damp.data(), (size_t)D * sizeof(float2), cudaMemcpyHostToDevice));
    }
    // Delta into work1, its scales from a host copy, then the constant planes
    make_delta_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, m->U, m->phase, m->work1, eff ? 0 : 1);
    count_launches(1);
    std::vector<double2> h((size_t)(D * D));
    QED_CUDA_TRY(cudaMemcpyAsync(h.data(), m->work1, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    double maxabs = 0.0, maxrow = 0.0;
    for (int64_t k = 0; k < D; ++k) {
        double row = 0.0;
        for (int64_t l = 0; l < D; ++l) {
            double a = std::hypot(h[(size_t)(k * D + l)].x, h[(size_t)(k * D + l)].y);
            maxabs = std::max(maxabs, a);
            row += a;
        }
        maxrow = std::max(maxrow, row);
    }
    // largest scaled magnitude 2^14 (FP16 max 65504); |rho_kl| <= 1, |W_kl| <= max row sum of |Delta|
    S.scale_delta = pow2_scale(maxabs, 14);
    S.scale_rho = std::ldexp(1.0, 14);
    S.scale_w = pow2_scale(maxrow, 14);
    static_planes_kernel<<<blocks_for((int64_t)W2, 256), 256, 0, s>>>(D, Dp, m->work1, S.scale_delta, S.a1, S.b2);
    count_launches(1);
    QED_CUDA_TRY(cudaGetLastError());
    qed_model *self[1] = {m};
    return build_batch(S.self, self, 1, true);
}

qed_status split_begin(qed_model *m, const double2 *rho, cudaStream_t s) {
    SplitState &S = *m->sp;
    dim3 grid(blocks_for(m->D, 256), (unsigned)m->D);
    import_kernel<<<grid, 256, 0, s>>>(m->D, S.Dp, rho, (float)S.scale_rho, S.rho_df[0], S.rho_pl);
    count_launches(1);
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}

void split_check_density(qed_model *m, const double2 *rho, cudaStream_t s) {
    dim3 grid(blocks_for(m->D, 32), blocks_for(m->D, 8));
    check_density_kernel<<<grid, dim3(32, 8), 0, s>>>(m->D, rho, m->err, m->scheme != QED_SCHEME_EFFECTIVE);
    count_launches(1);
}

void batch_step(const Batch &b, uint32_t *err, cudaStream_t s) {
    if (b.scheme == QED_SCHEME_STRANG) launch_half_lindblad(b, 0, 1, s);  // rho <- E(dt/2) rho
    launch_gemm1(b, err, s);  // W and its planes (split-K slices summed inside each cluster)
    launch_gemm2(b, err, s);  // X on and above the diagonal; its epilogue writes V = U rho U^+
    if (b.scheme == QED_SCHEME_STRANG)
        launch_half_lindblad(b, 1, 0, s);  // rho <- E(dt/2) V
    else
        launch_dissipate(b, s);
}

void split_step(qed_model *m, cudaStream_t s) { batch_step(m->sp->self, m->err, s); }

// Chooses the tile width and split-K factor (CTAs per cluster) of each of the model's two
// products by timing whole steps: GEMM1's candidates (128- and 256-wide tiles, 1, 2, 4 or 8
// slices) with GEMM2 as planned, then GEMM2's (128- and 256-wide, 1, 2 or 4 slices) with the
// best GEMM1.  Plans whose slices would not be a power of two are skipped.  Overwrites the
// internal state (qed_evolve imports rho again) and replaces the step tables; the caller
// drops its captured graphs.
qed_status split_autotune(qed_model *m, cudaStream_t s, int steps, std::string &choice) {
    SplitState &S = *m->sp;
    qed_model *self[1] = {m};
    auto candidates = [&](int which, std::vector<TcGemm> &out) -> qed_status {
        for (int bn : {128, 256}) {
            for (int sp : {1, 2, 4, 8}) {
                if (which == 2 && sp > kTcMaxClusterV) continue;
                TcGemm g1, g2;
                if (!plan_products(S, g1, g2, which == 1 ? sp : S.g1.splits, which == 1 ? bn : S.g1.bn,
                                   which == 2 ? sp : S.g2.splits, which == 2 ? bn : S.g2.bn))
                    return QED_ECUDA;
                const TcGemm &g = which == 1 ? g1 : g2;
                bool seen = (g.splits & (g.splits - 1)) != 0;
                for (const auto &h : out) seen = seen || (h.bn == g.bn && h.splits == g.splits);
                if (!seen) out.push_back(g);
            }
        }
        return QED_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QED_CUDA_TRY(cudaEventCreate(&e0));
    QED_CUDA_TRY(cudaEventCreate(&e1));
    auto time_steps = [&](float &ms) -> qed_status {
        QED_CUDA_TRY(cudaStreamSynchronize(s));
        SPLIT_TRY(build_batch(S.self, self, 1, true));
        for (int i = 0; i < 2; ++i) batch_step(S.self, m->err, s);
        QED_CUDA_TRY(cudaEventRecord(e0, s));
        for (int i = 0; i < steps; ++i) batch_step(S.self, m->err, s);
        QED_CUDA_TRY(cudaEventRecord(e1, s));
        QED_CUDA_TRY(cudaEventSynchronize(e1));
        QED_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        return QED_OK;
    };
    qed_status st = QED_OK;
    float best = 0.f;
    TcGemm g1 = S.g1, g2 = S.g2;
    std::vector<TcGemm> c1, c2;
    if ((st = candidates(1, c1)) == QED_OK && (st = candidates(2, c2)) == QED_OK && (st = time_steps(best)) == QED_OK) {
        for (const auto &g : c1) {
            S.g1 = g;
            S.g2 = g2;
            float t = 0.f;
            if ((st = time_steps(t)) != QED_OK) break;
            if (t < best) best = t, g1 = g;
        }
        for (size_t i = 0; st == QED_OK && i < c2.size(); ++i) {
            S.g1 = g1;
            S.g2 = c2[i];
            float t = 0.f;
            if ((st = time_steps(t)) != QED_OK) break;
            if (t < best) best = t, g2 = c2[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    S.g1 = g1;
    S.g2 = g2;
    if (st != QED_OK) return st;
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    SPLIT_TRY(build_batch(S.self, self, 1, true));
    choice = "gemm1 " + std::to_string(g1.bn) + "-wide x" + std::to_string(g1.splits) + " slices, gemm2 " +
             std::to_string(g2.bn) + "-wide x" + std::to_string(g2.splits) + " slices, " +
             std::to_string(1e3 * best / steps) + " us per step";
    return QED_OK;
}

// The batched counterpart: the grouped launches share one plan, so the candidates are the
// tile widths of the two products (GEMM1 256 or 128, GEMM2 128 or 256; both unsplit), each
// pair timed on `steps` whole batched steps from a zero state.  The winner is kept in every
// model of the batch.
qed_status split_autotune_batched(qed_model *const *ms, int n, cudaStream_t s, int steps, std::string &choice) {
    for (int i = 0; i < n; ++i) {
        SplitState &S = *ms[i]->sp;
        QED_CUDA_TRY(cudaMemsetAsync(S.rho_df[0], 0, (size_t)(ms[i]->D * ms[i]->D) * sizeof(float4), s));
        QED_CUDA_TRY(cudaMemsetAsync(S.rho_pl, 0, (size_t)S.Dp * 2 * S.Dp * 2 * sizeof(__half), s));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QED_CUDA_TRY(cudaEventCreate(&e0));
    QED_CUDA_TRY(cudaEventCreate(&e1));
    Batch b;
    qed_status st = QED_OK;
    float best = -1.f;
    int best1 = kTcBNMax, best2 = kTcBNMax;
    std::string times;
    const int plans[4][2] = {{256, 256}, {128, 256}, {256, 128}, {128, 128}};
    for (const auto &pl : plans) {
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            set_error(std::string("autotune (batched): ") + cudaGetErrorString(cudaGetLastError()));
            st = QED_ECUDA;
            break;
        }
        if ((st = build_batch(b, ms, n, false, pl[0], pl[1])) != QED_OK) break;
        for (int i = 0; i < 2; ++i) batch_step(b, ms[0]->err, s);
        float t = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = QED_ECUDA; break; }
        for (int i = 0; i < steps; ++i) batch_step(b, ms[0]->err, s);
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            set_error(std::string("autotune (batched): ") + cudaGetErrorString(cudaGetLastError()));
            st = QED_ECUDA;
            break;
        }
        times += (times.empty() ? "" : ", ") + std::to_string(pl[0]) + "/" + std::to_string(pl[1]) + " " +
                 std::to_string(1e3 * t / steps) + " us";
        if (best < 0.f || t < best) best = t, best1 = pl[0], best2 = pl[1];
    }
    cudaStreamSynchronize(s);
    b.release();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != QED_OK) return st;
    for (int i = 0; i < n; ++i) ms[i]->sp->batch_bn1 = best1, ms[i]->sp->batch_bn2 = best2;
    choice = "gemm1 " + std::to_string(best1) + "-wide, gemm2 " + std::to_string(best2) +
             "-wide (batched step, gemm1/gemm2 widths: " + times + ")";
    return QED_OK;
}

qed_status split_set_plan(qed_model *m, int bn1, int splits1, int bn2, int splits2, cudaStream_t s) {
    SplitState &S = *m->sp;
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    if ((bn1 != 128 && bn1 != 256) || (bn2 != 128 && bn2 != 256) || !pow2(splits1) || splits1 > kTcMaxCluster ||
        !pow2(splits2) || splits2 > kTcMaxClusterV) {
        set_error("qed_set_plan: widths 128 or 256, slices a power of two (GEMM1 <= 8, GEMM2 <= 4)");
        return QED_EINVAL;
    }
    TcGemm g1, g2;
    if (!plan_products(S, g1, g2, splits1, bn1, splits2, bn2)) return QED_ECUDA;
    if (g1.splits != splits1 || g2.splits != splits2) {
        set_error("qed_set_plan: more K slices than the product's 64-wide K blocks allow");
        return QED_EINVAL;
    }
    S.g1 = g1;
    S.g2 = g2;
    S.batch_bn1 = bn1;
    S.batch_bn2 = bn2;
    return split_rebuild(m, s);
}

void split_lindblad_stage(qed_model *m, int xsel, int bsel, int osel, float f, int planes, cudaStream_t s) {
    launch_lindblad(m->sp->self, xsel, bsel, osel, f, planes, s);
}

void split_apply_lindblad(qed_model *m, const float4 *X, float4 *out, cudaStream_t s) {
    const Batch &b = m->sp->self;
    launch_pdl(lindblad_apply_df_kernel, dim3(b.n_etiles), dim3(32, 8), 0, s, b.etiles, b.desc, X, out);
    count_launches(1);
}

void split_products(qed_model *m, cudaStream_t s) {
    launch_gemm1(m->sp->self, m->err, s);
    launch_gemm2(m->sp->self, m->err, s);
}

float4 *split_ybuf(qed_model *m) { return m->sp->y_df; }

qed_status split_rebuild(qed_model *m, cudaStream_t s) {
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    qed_model *self[1] = {m};
    return build_batch(m->sp->self, self, 1, true);
}

void split_set_scheme(qed_model *m, int scheme) {
    if (m->sp) m->sp->self.scheme = scheme;
}

// Each kernel of the Lie step replayed `reps` times back to back from a CUDA graph (the way
// the step loop runs them: programmatic dependent launch overlapping one launch's set-up
// with the previous one's tail), after one full step so that W, V and the planes hold
// this state's values.  Each kernel only reads what the others write and overwrites its
// own outputs with the same values, so the replay repeats identical work.  ms[c] = mean
// milliseconds per launch.
qed_status split_profile_replay(qed_model *m, cudaStream_t s, int reps, std::vector<double> &ms, std::string &label) {
    const Batch &b = m->sp->self;
    if (b.scheme != QED_SCHEME_LIE) {
        set_error("qed_profile_replay: the Lie step only");
        return QED_EUNSUPPORTED;
    }
    batch_step(b, m->err, s);
    cudaStream_t cap = nullptr;
    QED_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    qed_status st = QED_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = QED_ECUDA;
    ms.assign(3, 0.0);
    for (int c = 0; c < 3 && st == QED_OK; ++c) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = QED_ECUDA;
            break;
        }
        const int64_t before = launches();
        for (int r = 0; r < reps; ++r) {
            if (c == 0) launch_gemm1(b, m->err, cap);
            else if (c == 1) launch_gemm2(b, m->err, cap);
            else launch_dissipate(b, cap);
        }
        count_launches(-(launches() - before));
        const cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) st = QED_ECUDA;
        if (graph) cudaGraphDestroy(graph);
        float t = 0.f;
        if (st == QED_OK && (cudaGraphLaunch(exec, s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
                             cudaGraphLaunch(exec, s) != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            st = QED_ECUDA;
        count_launches(2 * (int64_t)reps);
        ms[(size_t)c] = (double)t / reps;
        if (exec) cudaGraphExecDestroy(exec);
    }
    if (st == QED_ECUDA) set_error(std::string("qed_profile_replay: ") + cudaGetErrorString(cudaGetLastError()));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(cap);
    label = "gemm1_tc,gemm2_tc_v,dissipate";
    return st;
}

int split_step_timed(qed_model *m, cudaStream_t s, std::string &label) {
    const Batch &b = m->sp->self;
    if (b.scheme == QED_SCHEME_STRANG) {
        int e = 0;
        cudaEventRecord(m->ev[e++], s);
        launch_lindblad(b, 0, 0, 2, 0.25f, 0, s);
        cudaEventRecord(m->ev[e++], s);
        launch_lindblad(b, 2, 0, 0, 0.5f, 1, s);
        cudaEventRecord(m->ev[e++], s);
        launch_gemm1(b, m->err, s);
        cudaEventRecord(m->ev[e++], s);
        launch_gemm2(b, m->err, s);
        cudaEventRecord(m->ev[e++], s);
        launch_lindblad(b, 1, 1, 2, 0.25f, 0, s);
        cudaEventRecord(m->ev[e++], s);
        launch_lindblad(b, 2, 1, 0, 0.5f, 0, s);
        cudaEventRecord(m->ev[e++], s);
        label = "lindblad_a,lindblad_b,gemm1_tc,gemm2_tc_v,lindblad_c,lindblad_d";
        return 6;
    }
    cudaEventRecord(m->ev[0], s);
    launch_gemm1(b, m->err, s);
    cudaEventRecord(m->ev[1], s);
    launch_gemm2(b, m->err, s);
    cudaEventRecord(m->ev[2], s);
    launch_dissipate(b, s);
    cudaEventRecord(m->ev[3], s);
    label = "gemm1_tc,gemm2_tc_v,dissipate";
    return 3;
}

void split_renorm(qed_model *m, cudaStream_t s) {
    SplitState &S = *m->sp;
    trace_df_kernel<<<1, 1024, 0, s>>>(m->D, S.rho_df[0], m->scalars, m->err);
    dim3 block(32, 8);
    dim3 grid(blocks_for(m->D, 32), blocks_for(m->D, 8));
    // the effective step's own trace drift is part of its result: symmetrise only
    symmetrise_df_kernel<<<grid, block, 0, s>>>(m->D, S.Dp, S.rho_df[0], m->scalars, m->err,
                                                (float)S.scale_rho, S.rho_pl, m->scheme != QED_SCHEME_EFFECTIVE);
    count_launches(2);
}

void split_observables(qed_model *m, const int32_t *ids, int32_t n_obs, double *out, cudaStream_t s) {
    if (n_obs <= 0) return;
    observables_df_kernel<<<n_obs, 256, 0, s>>>(m->D, m->sp->rho_df[0], m->obs_w, ids, out);
    count_launches(1);
}

void split_end(qed_model *m, double2 *rho, cudaStream_t s) {
    export_kernel<<<blocks_for(m->D * m->D, 256), 256, 0, s>>>(m->D, m->sp->rho_df[0], rho);
    count_launches(1);
}

__global__ void populations_kernel(int64_t D, const float4 *st, double *out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    const float4 v = st[k * D + k];
    out[k] = (double)v.x + (double)v.y;
}

void split_populations(qed_model *m, double *out, cudaStream_t s) {
    populations_kernel<<<blocks_for(m->D, 256), 256, 0, s>>>(m->D, m->sp->rho_df[0], out);
    count_launches(1);
}

qed_status split_batch_create(qed_model *const *ms, int n, Batch **out) {
    Batch *b = new Batch();
    // the tuned tile widths when every model of the batch carries the same ones
    int bn1 = ms[0]->sp->batch_bn1, bn2 = ms[0]->sp->batch_bn2;
    for (int i = 1; i < n; ++i)
        if (ms[i]->sp->batch_bn1 != bn1 || ms[i]->sp->batch_bn2 != bn2) bn1 = kTcBNMax, bn2 = kTcBNMax;
    qed_status st = build_batch(*b, ms, n, false, bn1, bn2);
    if (st != QED_OK) {
        b->release();
        delete b;
        return st;
    }
    *out = b;
    return QED_OK;
}

void split_batch_step(const Batch *b, uint32_t *err, cudaStream_t s) { batch_step(*b, err, s); }

void split_batch_destroy(Batch *b) {
    if (!b) return;
    b->release();
    delete b;
}

float4 *split_state(qed_model *m) { return m->sp->rho_df[0]; }
float4 *split_vbuf(qed_model *m) { return m->sp->rho_df[1]; }
void split_dissipate_only(qed_model *m, cudaStream_t s) { launch_dissipate(m->sp->self, s); }
void split_refresh_planes(qed_model *m, cudaStream_t s) {
    SplitState &S = *m->sp;
    dim3 grid(blocks_for(m->D, 256), (unsigned)m->D);
    planes_from_state_kernel<<<grid, 256, 0, s>>>(m->D, S.Dp, S.rho_df[0], (float)S.scale_rho, S.rho_pl);
    count_launches(1);
}

void split_release(qed_model *m) {
    if (!m->sp) return;
    SplitState &S = *m->sp;
    S.self.release();
    void *ptrs[] = {S.a1,       S.b2,       S.rho_pl,   S.w_pl,    S.w32,    S.rho_df[0], S.rho_df[1],
                    S.phase_df, S.damp_df, S.coef_df, S.in_tab, S.y_df, S.jtab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m->sp;
    m->sp = nullptr;
}

}  // namespace qed
