// Split-precision step in increment form.
//
// With E_k = H_kk and P = diag(exp(-i E_k dt)), the propagator factors exactly as
// U = P (I + Delta), Delta = P^-1 U - I, so the "unitary evolution" of Sec. 4.2 is
//     V = U rho U^+ = P (rho + W + W^+ + X) P^+,   W = Delta rho,  X = W Delta^+.
// rho stays FP64; only the small increments W and X go through the tensor cores, with
// every operand split into an FP16 hi part and an FP16 lo part (power-of-two scaled) and
// the three products hi*hi + hi*lo + lo*hi accumulated in FP32.  Complex products use
// the real embedding, with the signs folded into the constant operands:
//   GEMM1  [W_re; W_im] (2Dp x Dp)  = [[D_re, D_im], [D_im, -D_re]] . [rho_re | rho_im]^T
//   GEMM2  [X_re | X_im] (Dp x 2Dp) = [W_re | W_im] . [[D_re, D_im], [-D_im, D_re]]^T
// (rho^T = conj(rho) for the Hermitian rho, so the row-major rho planes are the K-major
// operand directly.)  The Lindblad update of Eq. (3) then runs on V in FP64.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gemm_tc.h"
#include "kernels.h"
#include "split.h"

namespace qed {

namespace {

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ void split_half(double x, __half &hi, __half &lo) {
    hi = __double2half(x);
    lo = __double2half(x - (double)__half2float(hi));
}

// Delta = conj(P_k) U_kl - delta_kl   (|P_k| = 1, so P^-1 = conj(P))
__global__ void make_delta_kernel(int64_t D, const double2 *U, const double2 *P, double2 *Dl) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    int64_t k = idx / D, l = idx % D;
    double2 u = U[idx], p = P[k];
    double2 d = make_double2(p.x * u.x + p.y * u.y, p.x * u.y - p.y * u.x);
    if (k == l) d.x -= 1.0;
    Dl[idx] = d;
}

// a1 = [[Dre, Dim], [Dim, -Dre]] and b2 = [[Dre, Dim], [-Dim, Dre]], 2Dp x 2Dp, hi/lo planes.
__global__ void static_planes_kernel(int64_t D, int64_t Dp, const double2 *Dl, double s, __half *a1, __half *b2) {
    const int64_t W2 = 2 * Dp;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= W2 * W2) return;
    int64_t r = idx / W2, c = idx % W2;
    int64_t rk = r % Dp, cm = c % Dp;
    bool rlo = r >= Dp, clo = c >= Dp;
    double va = 0.0, vb = 0.0;
    if (rk < D && cm < D) {
        double2 d = Dl[rk * D + cm];
        if (!rlo && !clo) { va = d.x; vb = d.x; }
        else if (!rlo && clo) { va = d.y; vb = d.y; }
        else if (rlo && !clo) { va = d.y; vb = -d.y; }
        else { va = -d.x; vb = d.x; }
    }
    __half h, l;
    split_half(va * s, h, l);
    a1[idx] = h;
    a1[W2 * W2 + idx] = l;
    split_half(vb * s, h, l);
    b2[idx] = h;
    b2[W2 * W2 + idx] = l;
}

// rho planes: row l = [rho_re[l, :] | rho_im[l, :]] (Dp x 2Dp), scaled, hi/lo.
__global__ void rho_planes_kernel(int64_t D, int64_t Dp, const double2 *rho, double s, __half *pl) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t l = blockIdx.y;
    if (m >= D || l >= D) return;
    double2 v = rho[l * D + m];
    __half h, lo;
    const int64_t plane = Dp * 2 * Dp;
    split_half(v.x * s, h, lo);
    pl[l * 2 * Dp + m] = h;
    pl[plane + l * 2 * Dp + m] = lo;
    split_half(v.y * s, h, lo);
    pl[l * 2 * Dp + Dp + m] = h;
    pl[plane + l * 2 * Dp + Dp + m] = lo;
}

// W = sum of the split-K partials of GEMM1 (rows r < Dp real, r >= Dp imaginary), in FP32,
// and its hi/lo planes as GEMM2's A operand: row k = [W_re[k, :] | W_im[k, :]].
__global__ void w_reduce_kernel(int64_t Dp, int splits, const float *part, double inv_scale, double s_w, float *w32,
                                __half *wpl) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (l >= Dp) return;
    const int64_t stride = 2 * Dp * Dp;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += (double)part[s * stride + r * Dp + l];
    const double w = acc * inv_scale;
    w32[r * Dp + l] = (float)w;
    const int64_t k = r % Dp;
    const int64_t col = (r >= Dp ? Dp : 0) + l;
    __half h, lo;
    split_half(w * s_w, h, lo);
    wpl[k * 2 * Dp + col] = h;
    wpl[Dp * 2 * Dp + k * 2 * Dp + col] = lo;
}

// V_kl = P_k conj(P_l) (rho_kl + W_kl + conj(W_lk) + X_kl)
__global__ void form_v_kernel(int64_t D, int64_t Dp, int splits, const double2 *__restrict__ rho,
                              const float *__restrict__ w32, const float *__restrict__ part, double inv_scale,
                              const double2 *__restrict__ P, double2 *__restrict__ V) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (k >= D || l >= D) return;
    const int64_t stride = Dp * 2 * Dp;
    double xr = 0.0, xi = 0.0;
    for (int s = 0; s < splits; ++s) {
        xr += (double)part[s * stride + k * 2 * Dp + l];
        xi += (double)part[s * stride + k * 2 * Dp + Dp + l];
    }
    const double2 r = rho[k * D + l];
    double sr = r.x + (double)w32[k * Dp + l] + (double)w32[l * Dp + k] + xr * inv_scale;
    double si = r.y + (double)w32[Dp * Dp + k * Dp + l] - (double)w32[Dp * Dp + l * Dp + k] + xi * inv_scale;
    const double2 pk = P[k], pl = P[l];
    // phase = P_k conj(P_l)
    const double2 ph = make_double2(pk.x * pl.x + pk.y * pl.y, pk.y * pl.x - pk.x * pl.y);
    V[k * D + l] = make_double2(ph.x * sr - ph.y * si, ph.x * si + ph.y * sr);
}

// Lindblad update of Eq. (3) on V (as in the FP64 path) that also writes the rho planes.
__global__ void dissipate_split_kernel(int64_t D, int64_t Dp, const double2 *__restrict__ V, double2 *__restrict__ rho,
                                       const double *__restrict__ anti, const int32_t *__restrict__ in_ptr,
                                       const int32_t *__restrict__ in_jump, const int32_t *__restrict__ in_src,
                                       const double *__restrict__ in_coef, double dt, double s_rho,
                                       __half *__restrict__ pl) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (m >= D || n >= D) return;
    double2 v = V[m * D + n];
    double f = 1.0 - 0.5 * dt * (anti[m] + anti[n]);
    double2 out = make_double2(v.x * f, v.y * f);
    int a = in_ptr[m], ae = in_ptr[m + 1];
    int b = in_ptr[n], be = in_ptr[n + 1];
    while (a < ae && b < be) {
        int ja = in_jump[a], jb = in_jump[b];
        if (ja < jb) {
            ++a;
        } else if (ja > jb) {
            ++b;
        } else {
            double c = dt * in_coef[a] * in_coef[b];
            double2 g = V[(int64_t)in_src[a] * D + in_src[b]];
            out.x = fma(c, g.x, out.x);
            out.y = fma(c, g.y, out.y);
            ++a;
            ++b;
        }
    }
    rho[m * D + n] = out;
    __half h, lo;
    const int64_t plane = Dp * 2 * Dp;
    split_half(out.x * s_rho, h, lo);
    pl[m * 2 * Dp + n] = h;
    pl[plane + m * 2 * Dp + n] = lo;
    split_half(out.y * s_rho, h, lo);
    pl[m * 2 * Dp + Dp + n] = h;
    pl[plane + m * 2 * Dp + Dp + n] = lo;
}

double pow2_scale(double maxabs, int target_exp) {
    if (!(maxabs > 0.0) || !std::isfinite(maxabs)) return 1.0;
    int e = (int)std::ceil(std::log2(maxabs));
    return std::ldexp(1.0, target_exp - e);
}

struct SplitState {
    TcGemm g1, g2;
    int num_sms = 148;
};

SplitState *state(qed_model *m) { return (SplitState *)m->sp.tmaps; }

}  // namespace

qed_status split_prepare(qed_model *m, cudaStream_t s) {
    SplitPlanes &sp = m->sp;
    const int64_t D = m->D;
    const int64_t Dp = (D + kTcBM - 1) / kTcBM * kTcBM;
    const size_t W2 = (size_t)(2 * Dp) * (size_t)(2 * Dp);
    if (!sp.tmaps) {
        SplitState *st = new SplitState();
        sp.tmaps = st;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, dev);
        sp.Dp = Dp;
        auto alloc = [&](void **p, size_t bytes) -> qed_status {
            if (cudaMalloc(p, bytes) != cudaSuccess) {
                cudaGetLastError();
                set_error("cudaMalloc failed for the split-precision buffers");
                return QED_ENOMEM;
            }
            return QED_OK;
        };
        qed_status st_;
        if ((st_ = alloc(&sp.a1, W2 * 2 * sizeof(__half))) != QED_OK) return st_;
        if ((st_ = alloc(&sp.b2, W2 * 2 * sizeof(__half))) != QED_OK) return st_;
        if ((st_ = alloc(&sp.rho_pl, (size_t)Dp * 2 * Dp * 2 * sizeof(__half))) != QED_OK) return st_;
        if ((st_ = alloc(&sp.w_pl, (size_t)Dp * 2 * Dp * 2 * sizeof(__half))) != QED_OK) return st_;
        if ((st_ = alloc((void **)&sp.w32, (size_t)2 * Dp * Dp * sizeof(float))) != QED_OK) return st_;
        QED_CUDA_TRY(cudaMemset(sp.rho_pl, 0, (size_t)Dp * 2 * Dp * 2 * sizeof(__half)));
        QED_CUDA_TRY(cudaMemset(sp.w_pl, 0, (size_t)Dp * 2 * Dp * 2 * sizeof(__half)));
        QED_CUDA_TRY(cudaMemset(sp.w32, 0, (size_t)2 * Dp * Dp * sizeof(float)));
        if (!tc_gemm_plan(st->g1, sp.a1, sp.rho_pl, (int)(2 * Dp), (int)Dp, (int)(2 * Dp), st->num_sms))
            return QED_ECUDA;
        if (!tc_gemm_plan(st->g2, sp.w_pl, sp.b2, (int)Dp, (int)(2 * Dp), (int)(2 * Dp), st->num_sms))
            return QED_ECUDA;
        sp.partial_elems = (int64_t)std::max(st->g1.splits, st->g2.splits) * 2 * Dp * Dp;
        if ((st_ = alloc((void **)&sp.partial, (size_t)sp.partial_elems * sizeof(float))) != QED_OK) return st_;
    }
    // Delta into work1, its scale from the host copy, then the constant planes
    make_delta_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, m->U, m->phase, m->work1);
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
    sp.scale_delta = pow2_scale(maxabs, 14);
    sp.scale_rho = std::ldexp(1.0, 14);
    sp.scale_w = pow2_scale(maxrow, 14);
    static_planes_kernel<<<blocks_for((int64_t)W2, 256), 256, 0, s>>>(D, Dp, m->work1, sp.scale_delta,
                                                                      (__half *)sp.a1, (__half *)sp.b2);
    count_launches(1);
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}

qed_status split_begin(qed_model *m, double2 *rho, cudaStream_t s) {
    SplitPlanes &sp = m->sp;
    dim3 grid(blocks_for(m->D, 256), (unsigned)m->D);
    rho_planes_kernel<<<grid, 256, 0, s>>>(m->D, sp.Dp, rho, sp.scale_rho, (__half *)sp.rho_pl);
    count_launches(1);
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}

static void launch_w_reduce(qed_model *m, cudaStream_t s) {
    SplitPlanes &sp = m->sp;
    SplitState *st = state(m);
    dim3 grid(blocks_for(sp.Dp, 256), (unsigned)(2 * sp.Dp));
    w_reduce_kernel<<<grid, 256, 0, s>>>(sp.Dp, st->g1.splits, sp.partial, 1.0 / (sp.scale_delta * sp.scale_rho),
                                         sp.scale_w, sp.w32, (__half *)sp.w_pl);
    count_launches(1);
}

static void launch_form_v(qed_model *m, cudaStream_t s, const double2 *rho) {
    SplitPlanes &sp = m->sp;
    SplitState *st = state(m);
    dim3 block(32, 8);
    dim3 grid(blocks_for(m->D, 32), blocks_for(m->D, 8));
    form_v_kernel<<<grid, block, 0, s>>>(m->D, sp.Dp, st->g2.splits, rho, sp.w32, sp.partial,
                                         1.0 / (sp.scale_w * sp.scale_delta), m->phase, m->work2);
    count_launches(1);
}

static void launch_dissipate(qed_model *m, cudaStream_t s, double2 *rho) {
    SplitPlanes &sp = m->sp;
    dim3 block(32, 8);
    dim3 grid(blocks_for(m->D, 32), blocks_for(m->D, 8));
    dissipate_split_kernel<<<grid, block, 0, s>>>(m->D, sp.Dp, m->work2, rho, m->anti, m->in_ptr, m->in_jump,
                                                  m->in_src, m->in_coef, m->dt, sp.scale_rho, (__half *)sp.rho_pl);
    count_launches(1);
}

void split_step(qed_model *m, double2 *rho, cudaStream_t s) {
    SplitState *st = state(m);
    tc_gemm_launch(st->g1, m->sp.partial, m->err, s);
    launch_w_reduce(m, s);
    tc_gemm_launch(st->g2, m->sp.partial, m->err, s);
    launch_form_v(m, s, rho);
    launch_dissipate(m, s, rho);
}

int split_step_timed(qed_model *m, double2 *rho, cudaStream_t s, std::string &label) {
    SplitState *st = state(m);
    cudaEventRecord(m->ev[0], s);
    tc_gemm_launch(st->g1, m->sp.partial, m->err, s);
    cudaEventRecord(m->ev[1], s);
    launch_w_reduce(m, s);
    cudaEventRecord(m->ev[2], s);
    tc_gemm_launch(st->g2, m->sp.partial, m->err, s);
    cudaEventRecord(m->ev[3], s);
    launch_form_v(m, s, rho);
    cudaEventRecord(m->ev[4], s);
    launch_dissipate(m, s, rho);
    cudaEventRecord(m->ev[5], s);
    label = "gemm1_tc,w_reduce,gemm2_tc,form_v,dissipate_split";
    return 5;
}

void split_renorm(qed_model *m, double2 *rho, cudaStream_t s) {
    renormalise(s, m->D, rho, m->scalars, m->err);
    split_begin(m, rho, s);
}

void split_sync_rho(qed_model *, double2 *, cudaStream_t) {}

void split_release(qed_model *m) {
    SplitPlanes &sp = m->sp;
    void *ptrs[] = {sp.a1, sp.b2, sp.rho_pl, sp.w_pl, sp.w32, sp.partial};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete state(m);
    sp.tmaps = nullptr;
}

}  // namespace qed
