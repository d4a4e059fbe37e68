// Discrete adjoint of the QME step (Eq. 2 with the Lindblad term of Eq. 3, Lie split as
// in qed_evolve): gradients of L = tr(diag(o) rho_N) with respect to the couplings g,
// the hoppings zeta and the rates gamma.
//
// Forward map: V_n = U rho_n U^+,  rho_{n+1} = J(V_n),  J(V) = V + dt sum_j gamma_j D_j(V),
// D_j(V) = A_j V A_j^+ - 1/2 {A_j^+ A_j, V}.  Co-state: lambda_N = diag(o), and per step
//     kappa = J^+(lambda_{n+1})        (J's Hilbert-Schmidt adjoint: A -> A^+ in the gathers)
//     dL/dgamma_j += dt tr(lambda_{n+1} D_j(V_n))
//     M += rho_n U^+ kappa
//     lambda_n = U^+ kappa U.
// For a Hamiltonian parameter theta, dL/dtheta = 2 Re tr(dU/dtheta M) with
// dU/dtheta = L_exp(X, -i dt dH/dtheta), X = -i dt H; since tr(L_exp(X, E) M) =
// tr(L_exp(X, M) E), one Frechet derivative G = L_exp(X, M) serves every parameter:
// dL/dtheta = 2 dt Im tr(G dH/dtheta).  G comes from the Pade-13 approximant of exp and its
// directional derivative, evaluated together (the upper-right block of
// exp([[X, M], [0, X]]), Najfeld and Havel; Higham 2008, Sec. 10.6; Al-Mohy and Higham
// 2009).  rho is checkpointed every k steps and each segment but the last recomputed
// (storing its rho_n and V_n) while stepping the co-state back; the forward pass stores
// the last segment directly, so k >= n_steps runs without recomputation.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "gemm_tc.h"
#include "kernels.h"
#include "model.h"
#include "split.h"

namespace qed {

struct AdjointState {
    // outgoing jump lists per row k (A_j |k> = c |dst>), sorted by jump, c * sqrt(gamma_j)
    int32_t *out_ptr = nullptr, *out_jump = nullptr, *out_dst = nullptr;
    double *out_coef = nullptr;
    // per-jump entries (CSR over jumps): src, dst, raw coefficient
    int32_t *je_ptr = nullptr, *je_src = nullptr, *je_dst = nullptr;
    double *je_coef = nullptr;
    int32_t n_jumps = 0;
    // Hamiltonian entries per parameter (CSR over g then zeta): row, col, unit amplitude
    int32_t *pe_ptr = nullptr, *pe_row = nullptr, *pe_col = nullptr;
    double *pe_unit = nullptr;
    int32_t n_g = 0, n_zeta = 0;
    double2 *H = nullptr;  // dense H (device)
    double h_norm1 = 0.0;
    int32_t n_out = 0;
    // split precision: the backward model (U^+, conjugate phases, outgoing jump lists),
    // whose step kappa -> J^+(U^+ kappa U) is the co-state step, and the tensor-core
    // product rho_n lambda_n
    qed_model *twin = nullptr;
    __half *a_pl = nullptr;   // [2][Dp][2Dp]   rows m: [rho_re | rho_im]
    __half *b_pl = nullptr;   // [2][2Dp][2Dp]  [[lam_re, lam_im], [-lam_im, lam_re]]
    float *c_slices = nullptr;
    TcGemm g;
    int64_t Dp = 0;
};

namespace {

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class T>
qed_status up(T **dst, const std::vector<T> &v) {
    const size_t n = std::max<size_t>(v.size(), 1);
    if (device_malloc((void **)dst, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed for the adjoint tables");
        return QED_ENOMEM;
    }
    if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("cudaMemcpy failed for the adjoint tables");
        return QED_ECUDA;
    }
    return QED_OK;
}

#define ADJ_TRY(expr)                   \
    do {                                \
        qed_status st_ = (expr);        \
        if (st_ != QED_OK) return st_;  \
    } while (0)

qed_status setup(qed_model *m) {
    if (m->adj) return QED_OK;
    AdjointState *a = new AdjointState();
    m->adj = a;
    const HostModel &hm = m->host;
    const int64_t D = m->D;
    // outgoing lists
    std::vector<std::vector<JumpEntry>> rows((size_t)D);
    for (const auto &e : hm.jumps) rows[(size_t)e.src].push_back(e);
    std::vector<int32_t> ptr((size_t)D + 1, 0), jj, dst;
    std::vector<double> coef;
    for (int64_t k = 0; k < D; ++k) {
        auto &v = rows[(size_t)k];
        std::sort(v.begin(), v.end(), [](const JumpEntry &x, const JumpEntry &y) { return x.jump < y.jump; });
        for (const auto &e : v) {
            jj.push_back(e.jump);
            dst.push_back((int32_t)e.dst);
            coef.push_back(e.coef * std::sqrt(hm.gamma[(size_t)e.jump]));
        }
        ptr[(size_t)k + 1] = (int32_t)jj.size();
    }
    a->n_out = (int32_t)jj.size();
    ADJ_TRY(up(&a->out_ptr, ptr));
    ADJ_TRY(up(&a->out_jump, jj));
    ADJ_TRY(up(&a->out_dst, dst));
    ADJ_TRY(up(&a->out_coef, coef));
    // per-jump entries
    a->n_jumps = (int32_t)hm.gamma.size();
    std::vector<std::vector<JumpEntry>> per((size_t)a->n_jumps);
    for (const auto &e : hm.jumps) per[(size_t)e.jump].push_back(e);
    std::vector<int32_t> jp(1, 0), js, jd;
    std::vector<double> jc;
    for (const auto &v : per) {
        for (const auto &e : v) {
            js.push_back((int32_t)e.src);
            jd.push_back((int32_t)e.dst);
            jc.push_back(e.coef);
        }
        jp.push_back((int32_t)js.size());
    }
    ADJ_TRY(up(&a->je_ptr, jp));
    ADJ_TRY(up(&a->je_src, js));
    ADJ_TRY(up(&a->je_dst, jd));
    ADJ_TRY(up(&a->je_coef, jc));
    // Hamiltonian entries per parameter: g (param 1) then zeta (param 2)
    a->n_g = (int32_t)hm.g.size();
    a->n_zeta = (int32_t)hm.zeta.size();
    const int np = a->n_g + a->n_zeta;
    std::vector<std::vector<const HostModel::HEntry *>> pe((size_t)np);
    for (const auto &e : hm.h_entries) {
        if (e.param == 1) pe[(size_t)e.which].push_back(&e);
        if (e.param == 2) pe[(size_t)(a->n_g + e.which)].push_back(&e);
    }
    std::vector<int32_t> pp(1, 0), pr, pc;
    std::vector<double> pu;
    for (const auto &v : pe) {
        for (const auto *e : v) {
            pr.push_back((int32_t)e->row);
            pc.push_back((int32_t)e->col);
            pu.push_back(e->unit);
        }
        pp.push_back((int32_t)pr.size());
    }
    ADJ_TRY(up(&a->pe_ptr, pp));
    ADJ_TRY(up(&a->pe_row, pr));
    ADJ_TRY(up(&a->pe_col, pc));
    ADJ_TRY(up(&a->pe_unit, pu));
    std::vector<cplx> Hd;
    dense_hamiltonian(hm, Hd);
    for (int64_t c = 0; c < D; ++c) {
        double col = 0.0;
        for (int64_t r = 0; r < D; ++r) col += std::abs(Hd[(size_t)(r * D + c)]);
        a->h_norm1 = std::max(a->h_norm1, col);
    }
    std::vector<double2> h2(Hd.size());
    for (size_t i = 0; i < Hd.size(); ++i) h2[i] = make_double2(Hd[i].real(), Hd[i].imag());
    ADJ_TRY(up(&a->H, h2));
    return QED_OK;
}

__global__ void set_diag_kernel(int64_t D, const double *o, double2 *X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    const int64_t r = idx / D, c = idx % D;
    X[idx] = make_double2(r == c ? o[r] : 0.0, 0.0);
}

__global__ void __launch_bounds__(256) loss_kernel(int64_t D, const double2 *rho, const double *o, double *loss) {
    __shared__ double part[256];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t k = t; k < D; k += blockDim.x) s += o[k] * rho[k * D + k].x;
    part[t] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (t < st) part[t] += part[t + st];
        __syncthreads();
    }
    if (t == 0) *loss = part[0];
}

// r_k = Re (lambda V)_kk = Re sum_n lambda_kn conj(V_kn)  (V Hermitian); one warp per row
__global__ void rowdot_kernel(int64_t D, const double2 *lam, const double2 *V, double *r) {
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (k >= D) return;
    double s = 0.0;
    for (int64_t n = lane; n < D; n += 32) {
        const double2 a = lam[k * D + n], b = V[k * D + n];
        s += a.x * b.x + a.y * b.y;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) r[k] = s;
}

// grad_gamma_j += dt [ sum_{e,f in A_j} c_e c_f Re(lambda[d_f][d_e] V[s_e][s_f]) - sum_e c_e^2 r[s_e] ]
__global__ void __launch_bounds__(256) gamma_grad_kernel(int64_t D, const int32_t *je_ptr, const int32_t *je_src,
                                                         const int32_t *je_dst, const double *je_coef,
                                                         const double2 *lam, const double2 *V, const double *r,
                                                         double dt, double *grad) {
    __shared__ double part[256];
    const int j = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t e0 = je_ptr[j], ne = je_ptr[j + 1] - e0;
    double s = 0.0;
    for (int64_t idx = t; idx < ne * ne; idx += blockDim.x) {
        const int64_t e = e0 + idx / ne, f = e0 + idx % ne;
        const double2 l = lam[(int64_t)je_dst[f] * D + je_dst[e]];
        const double2 v = V[(int64_t)je_src[e] * D + je_src[f]];
        s += je_coef[e] * je_coef[f] * (l.x * v.x - l.y * v.y);
    }
    for (int64_t e = e0 + t; e < e0 + ne; e += blockDim.x) s -= je_coef[e] * je_coef[e] * r[je_src[e]];
    part[t] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (t < st) part[t] += part[t + st];
        __syncthreads();
    }
    if (t == 0) grad[j] += dt * part[0];
}

// grad[p] = 2 dt Im sum_e unit_e G[col_e][row_e], G = L_exp(X, M)
__global__ void param_grad_kernel(int64_t D, int np, const int32_t *pe_ptr, const int32_t *pe_row,
                                  const int32_t *pe_col, const double *pe_unit, const double2 *G, double scale,
                                  double *grad_g, int n_g, double *grad_zeta) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int e = pe_ptr[p]; e < pe_ptr[p + 1]; ++e) s += pe_unit[e] * G[(int64_t)pe_col[e] * D + pe_row[e]].y;
    if (p < n_g)
        grad_g[p] = scale * s;
    else
        grad_zeta[p - n_g] = scale * s;
}

struct Buffers {
    std::vector<void *> ptrs;
    ~Buffers() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    qed_status get(T **p, size_t count) {
        if (device_malloc((void **)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the adjoint work space");
            return QED_ENOMEM;
        }
        ptrs.push_back(*p);
        return QED_OK;
    }
};

// ---------------------------------------------------------------- split precision
__global__ void conj_transpose_kernel(int64_t D, const double2 *U, double2 *Ut) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    const int64_t r = idx / D, c = idx % D;
    const double2 u = U[c * D + r];
    Ut[idx] = make_double2(u.x, -u.y);
}

__global__ void conj_kernel(int64_t n, const double2 *x, double2 *y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_double2(x[i].x, -x[i].y);
}

__global__ void set_diag_df_kernel(int64_t D, const double *o, float4 *X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    const int64_t r = idx / D, c = idx % D;
    float h = 0.f, l = 0.f;
    if (r == c) {
        h = (float)o[r];
        l = (float)(o[r] - (double)h);
    }
    X[idx] = make_float4(h, l, 0.f, 0.f);
}

__device__ __forceinline__ double2 dfc(const float4 v) {
    return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

__global__ void __launch_bounds__(256) loss_df_kernel(int64_t D, const float4 *st, const double *o, double *loss) {
    __shared__ double part[256];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t k = t; k < D; k += blockDim.x) s += o[k] * dfc(st[k * D + k]).x;
    part[t] = s;
    __syncthreads();
    for (int st2 = blockDim.x / 2; st2 > 0; st2 >>= 1) {
        if (t < st2) part[t] += part[t + st2];
        __syncthreads();
    }
    if (t == 0) *loss = part[0];
}

__global__ void rowdot_df_kernel(int64_t D, const float4 *lam, const float4 *V, double *r) {
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (k >= D) return;
    double s = 0.0;
    for (int64_t n = lane; n < D; n += 32) {
        const double2 a = dfc(lam[k * D + n]), b = dfc(V[k * D + n]);
        s += a.x * b.x + a.y * b.y;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) r[k] = s;
}

__global__ void __launch_bounds__(256) gamma_grad_df_kernel(int64_t D, const int32_t *je_ptr, const int32_t *je_src,
                                                            const int32_t *je_dst, const double *je_coef,
                                                            const float4 *lam, const float4 *V, const double *r,
                                                            double dt, double *grad) {
    __shared__ double part[256];
    const int j = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t e0 = je_ptr[j], ne = je_ptr[j + 1] - e0;
    double s = 0.0;
    for (int64_t idx = t; idx < ne * ne; idx += blockDim.x) {
        const int64_t e = e0 + idx / ne, f = e0 + idx % ne;
        const double2 l = dfc(lam[(int64_t)je_dst[f] * D + je_dst[e]]);
        const double2 v = dfc(V[(int64_t)je_src[e] * D + je_src[f]]);
        s += je_coef[e] * je_coef[f] * (l.x * v.x - l.y * v.y);
    }
    for (int64_t e = e0 + t; e < e0 + ne; e += blockDim.x) s -= je_coef[e] * je_coef[e] * r[je_src[e]];
    part[t] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (t < st) part[t] += part[t + st];
        __syncthreads();
    }
    if (t == 0) grad[j] += dt * part[0];
}

__device__ __forceinline__ void half2_of(float4 v, bool im, float s, __half &h, __half &l) {
    const float hi = (im ? v.z : v.x) * s, lo = (im ? v.w : v.y) * s;
    h = __float2half_rn(hi);
    l = __float2half_rn((hi - __half2float(h)) + lo);
}

// A planes of rho_n: rows m = [rho_re[m, :] | rho_im[m, :]] (Dp x 2Dp), hi / lo
__global__ void a_planes_kernel(int64_t D, int64_t Dp, const float4 *st, float s, __half *pl) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.y;
    if (n >= D) return;
    const float4 v = st[m * D + n];
    const int64_t plane = Dp * 2 * Dp;
    __half h, l;
    half2_of(v, false, s, h, l);
    pl[m * 2 * Dp + n] = h;
    pl[plane + m * 2 * Dp + n] = l;
    half2_of(v, true, s, h, l);
    pl[m * 2 * Dp + Dp + n] = h;
    pl[plane + m * 2 * Dp + Dp + n] = l;
}

// B planes of lambda_n: [[lam_re, lam_im], [-lam_im, lam_re]] (2Dp x 2Dp), hi / lo.  The
// product takes B transposed (K-major); for Hermitian lambda that is the same matrix.
__global__ void b_planes_kernel(int64_t D, int64_t Dp, const float4 *lam, float s, __half *pl) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.y;
    if (n >= D) return;
    const float4 v = lam[m * D + n];
    const float4 neg = make_float4(-v.x, -v.y, -v.z, -v.w);
    const int64_t W2 = 2 * Dp, plane = W2 * W2;
    __half h, l;
    half2_of(v, false, s, h, l);  // re, upper left and lower right
    pl[m * W2 + n] = h;
    pl[plane + m * W2 + n] = l;
    pl[(Dp + m) * W2 + Dp + n] = h;
    pl[plane + (Dp + m) * W2 + Dp + n] = l;
    half2_of(v, true, s, h, l);  // im, upper right
    pl[m * W2 + Dp + n] = h;
    pl[plane + m * W2 + Dp + n] = l;
    half2_of(neg, true, s, h, l);  // -im, lower left
    pl[(Dp + m) * W2 + n] = h;
    pl[plane + (Dp + m) * W2 + n] = l;
}

// Nacc += (sum of the slices) / scale, the product being [C_re | C_im] (Dp x 2Dp)
__global__ void acc_kernel(int64_t D, int64_t Dp, int splits, const float *sl, double inv, double2 *Nacc) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.y;
    if (n >= D) return;
    double re = 0.0, im = 0.0;
    const int64_t stride = Dp * 2 * Dp;
    for (int q = 0; q < splits; ++q) {
        re += sl[q * stride + m * 2 * Dp + n];
        im += sl[q * stride + m * 2 * Dp + Dp + n];
    }
    double2 a = Nacc[m * D + n];
    a.x += re * inv;
    a.y += im * inv;
    Nacc[m * D + n] = a;
}

qed_status make_twin(qed_model *m, cudaStream_t s) {
    AdjointState &a = *m->adj;
    if (a.twin) return QED_OK;
    qed_model *t = new qed_model();
    a.twin = t;
    const int64_t D = m->D;
    const size_t DD = (size_t)(D * D);
    t->D = D;
    t->dt = m->dt;
    t->prec = m->prec;
    t->renorm_every = 0;
    auto get = [&](void **p, size_t bytes) -> qed_status {
        if (device_malloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the backward model");
            return QED_ENOMEM;
        }
        return QED_OK;
    };
    ADJ_TRY(get((void **)&t->U, DD * 16));
    ADJ_TRY(get((void **)&t->work1, DD * 16));
    ADJ_TRY(get((void **)&t->work2, DD * 16));
    ADJ_TRY(get((void **)&t->phase, (size_t)D * 16));
    ADJ_TRY(get((void **)&t->anti, (size_t)D * 8));
    ADJ_TRY(get((void **)&t->in_ptr, (size_t)(D + 1) * 4));
    ADJ_TRY(get((void **)&t->in_jump, (size_t)a.n_out * 4));
    ADJ_TRY(get((void **)&t->in_src, (size_t)a.n_out * 4));
    ADJ_TRY(get((void **)&t->in_coef, (size_t)a.n_out * 8));
    ADJ_TRY(get((void **)&t->scalars, 16 * 8));
    ADJ_TRY(get((void **)&t->err, 4));
    QED_CUDA_TRY(cudaMallocHost((void **)&t->err_host, sizeof(uint32_t)));
    QED_CUDA_TRY(cudaMemsetAsync(t->err, 0, 4, s));
    t->n_in = a.n_out;
    conj_transpose_kernel<<<blocks_for((int64_t)DD, 256), 256, 0, s>>>(D, m->U, t->U);
    conj_kernel<<<blocks_for(D, 256), 256, 0, s>>>(D, m->phase, t->phase);
    count_launches(2);
    QED_CUDA_TRY(cudaMemcpyAsync(t->anti, m->anti, (size_t)D * 8, cudaMemcpyDeviceToDevice, s));
    QED_CUDA_TRY(cudaMemcpyAsync(t->in_ptr, a.out_ptr, (size_t)(D + 1) * 4, cudaMemcpyDeviceToDevice, s));
    if (a.n_out > 0) {
        QED_CUDA_TRY(cudaMemcpyAsync(t->in_jump, a.out_jump, (size_t)a.n_out * 4, cudaMemcpyDeviceToDevice, s));
        QED_CUDA_TRY(cudaMemcpyAsync(t->in_src, a.out_dst, (size_t)a.n_out * 4, cudaMemcpyDeviceToDevice, s));
        QED_CUDA_TRY(cudaMemcpyAsync(t->in_coef, a.out_coef, (size_t)a.n_out * 8, cudaMemcpyDeviceToDevice, s));
    }
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    ADJ_TRY(split_prepare(t, s));
    // the product rho_n lambda_n
    a.Dp = (D + kTcBM - 1) / kTcBM * kTcBM;
    const int64_t Dp = a.Dp;
    ADJ_TRY(get((void **)&a.a_pl, (size_t)2 * Dp * 2 * Dp * 2));
    ADJ_TRY(get((void **)&a.b_pl, (size_t)2 * (2 * Dp) * (2 * Dp) * 2));
    QED_CUDA_TRY(cudaMemset(a.a_pl, 0, (size_t)2 * Dp * 2 * Dp * 2));
    QED_CUDA_TRY(cudaMemset(a.b_pl, 0, (size_t)2 * (2 * Dp) * (2 * Dp) * 2));
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int seg[6] = {0, 0, 0, 1, 1, 0};
    if (!tc_gemm_plan(a.g, a.a_pl, 2, a.b_pl, 2, (int)Dp, (int)(2 * Dp), (int)(2 * Dp), 3, seg, sms))
        return QED_ECUDA;
    ADJ_TRY(get((void **)&a.c_slices, (size_t)a.g.splits * Dp * 2 * Dp * 4));
    return QED_OK;
}

// G = L_exp(X, M), X = -i dt H, contracted with dH/dtheta for every g and zeta.
qed_status frechet_gradients(qed_model *m, Buffers &B, const double2 *Macc, double *grad_g, double *grad_zeta,
                             cudaStream_t s) {
    NvtxRange range("adjoint: Frechet derivative and parameter gradients");
    AdjointState &a = *m->adj;
    const int64_t D = m->D;
    const size_t DD = (size_t)(D * D);
    const double dt = m->dt;
    if (a.n_g + a.n_zeta > 0) {
        double2 *X = nullptr, *R = nullptr, *G = nullptr;
        ADJ_TRY(B.get(&X, DD));
        ADJ_TRY(B.get(&R, DD));
        ADJ_TRY(B.get(&G, DD));
        scale_minus_i(s, D, dt, a.H, X);
        ADJ_TRY(expm_frechet_pade13(s, D, X, Macc, dt * a.h_norm1, R, G, m->err));
        const int np = a.n_g + a.n_zeta;
        param_grad_kernel<<<blocks_for(np, 128), 128, 0, s>>>(D, np, a.pe_ptr, a.pe_row, a.pe_col, a.pe_unit, G,
                                                              2.0 * dt, grad_g, a.n_g, grad_zeta);
        count_launches(1);
    }
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    QED_CUDA_TRY(cudaGetLastError());
    uint32_t flags = 0;
    QED_CUDA_TRY(cudaMemcpy(&flags, m->err, 4, cudaMemcpyDeviceToHost));
    if (flags & kErrSingular) {
        QED_CUDA_TRY(cudaMemset(m->err, 0, 4));
        set_error("qed_adjoint: singular Pade denominator in the Frechet derivative");
        return QED_ENUMERIC;
    }
    return QED_OK;
}

// The adjoint on the split-precision path: the forward steps and the segment recomputes
// are qed_evolve's steps, the co-state steps are the backward model's steps, and
// M = (sum_n rho_n lambda_n) U^+ is accumulated from one tensor-core product per step.
qed_status adjoint_split(qed_model *m, const void *rho0, int64_t N, int64_t k, const double *obs_diag, double *loss,
                         double *grad_g, double *grad_zeta, double *grad_gamma, cudaStream_t s) {
    {
        const qed_status st = make_twin(m, s);
        if (st != QED_OK) {  // nothing half-built is kept for the next call
            cudaStreamSynchronize(s);
            adjoint_release(m);
            return st;
        }
    }
    AdjointState &a = *m->adj;
    qed_model *t = a.twin;
    k = std::min<int64_t>(k, std::max<int64_t>(N, 1));
    const int64_t D = m->D, Dp = a.Dp;
    const size_t DD = (size_t)(D * D);
    const int64_t n_ck = N > 0 ? (N - 1) / k + 1 : 0;
    const double dt = m->dt;
    // The co-state is linear in o: run it for o / 2^e with max |o / 2^e| in (1/2, 1], so that
    // |lambda_kl| <= 1 like |rho_kl| (the co-state map is unital and contractive) and the
    // backward model's FP16 scales hold, and scale the gradients by 2^e.
    std::vector<double> ho((size_t)D);
    QED_CUDA_TRY(cudaMemcpyAsync(ho.data(), obs_diag, (size_t)D * 8, cudaMemcpyDeviceToHost, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    double omax = 0.0;
    for (double x : ho) omax = std::max(omax, std::abs(x));
    const int e = omax > 0.0 ? (int)std::ceil(std::log2(omax)) : 0;
    const double o_scale = std::ldexp(1.0, e);
    for (double &x : ho) x = std::ldexp(x, -e);
    const double s_a = std::ldexp(1.0, 14), s_b = std::ldexp(1.0, 14);
    Buffers B;
    float4 *ck = nullptr, *seg_rho = nullptr, *seg_v = nullptr;
    double2 *Nacc = nullptr, *Macc = nullptr;
    double *r = nullptr, *o_s = nullptr;
    ADJ_TRY(B.get(&o_s, (size_t)D));
    QED_CUDA_TRY(cudaMemcpyAsync(o_s, ho.data(), (size_t)D * 8, cudaMemcpyHostToDevice, s));
    ADJ_TRY(B.get(&ck, DD * (size_t)std::max<int64_t>(n_ck, 1)));
    ADJ_TRY(B.get(&seg_rho, DD * (size_t)k));
    ADJ_TRY(B.get(&seg_v, DD * (size_t)k));
    ADJ_TRY(B.get(&Nacc, DD));
    ADJ_TRY(B.get(&Macc, DD));
    ADJ_TRY(B.get(&r, (size_t)D));
    // forward with checkpoints of the double-float state
    const int64_t last0 = (n_ck - 1) * k;  // the last segment is stored by the forward pass
    split_check_density(m, (const double2 *)rho0, s);
    ADJ_TRY(split_begin(m, (const double2 *)rho0, s));
    for (int64_t n = 0; n < N; ++n) {
        if (n % k == 0 && n < last0)
            QED_CUDA_TRY(cudaMemcpyAsync(ck + (size_t)(n / k) * DD, split_state(m), DD * 16, cudaMemcpyDeviceToDevice, s));
        if (n >= last0)
            QED_CUDA_TRY(cudaMemcpyAsync(seg_rho + (size_t)(n - last0) * DD, split_state(m), DD * 16,
                                         cudaMemcpyDeviceToDevice, s));
        split_step(m, s);
        if (n >= last0)
            QED_CUDA_TRY(cudaMemcpyAsync(seg_v + (size_t)(n - last0) * DD, split_vbuf(m), DD * 16,
                                         cudaMemcpyDeviceToDevice, s));
    }
    loss_df_kernel<<<1, 256, 0, s>>>(D, split_state(m), obs_diag, loss);
    // co-state: lambda_N = diag(o) in the backward model's V buffer, kappa_N = J^+(lambda_N)
    set_diag_df_kernel<<<blocks_for((int64_t)DD, 256), 256, 0, s>>>(D, o_s, split_vbuf(t));
    count_launches(2);
    split_dissipate_only(t, s);
    QED_CUDA_TRY(cudaMemsetAsync(Nacc, 0, DD * 16, s));
    if (a.n_jumps > 0) QED_CUDA_TRY(cudaMemsetAsync(grad_gamma, 0, (size_t)a.n_jumps * 8, s));
    const dim3 rows(blocks_for(D, 256), (unsigned)D);
    for (int64_t c = n_ck - 1; c >= 0; --c) {
        const int64_t s0 = c * k, s1 = std::min(N, s0 + k);
        if (c < n_ck - 1) {
            QED_CUDA_TRY(cudaMemcpyAsync(split_state(m), ck + (size_t)c * DD, DD * 16, cudaMemcpyDeviceToDevice, s));
            split_refresh_planes(m, s);
        }
        for (int64_t n = s0; n < s1 && c < n_ck - 1; ++n) {
            QED_CUDA_TRY(cudaMemcpyAsync(seg_rho + (size_t)(n - s0) * DD, split_state(m), DD * 16,
                                         cudaMemcpyDeviceToDevice, s));
            split_step(m, s);
            QED_CUDA_TRY(cudaMemcpyAsync(seg_v + (size_t)(n - s0) * DD, split_vbuf(m), DD * 16,
                                         cudaMemcpyDeviceToDevice, s));
        }
        for (int64_t n = s1 - 1; n >= s0; --n) {
            const float4 *rn = seg_rho + (size_t)(n - s0) * DD, *vn = seg_v + (size_t)(n - s0) * DD;
            if (a.n_jumps > 0) {  // lambda_{n+1} is still in the backward model's V buffer
                rowdot_df_kernel<<<blocks_for(D, 8), 256, 0, s>>>(D, split_vbuf(t), vn, r);
                gamma_grad_df_kernel<<<a.n_jumps, 256, 0, s>>>(D, a.je_ptr, a.je_src, a.je_dst, a.je_coef,
                                                               split_vbuf(t), vn, r, dt * o_scale, grad_gamma);
                count_launches(2);
            }
            split_step(t, s);  // kappa_{n+1} -> lambda_n (V buffer) -> kappa_n (state)
            // Nacc += rho_n lambda_n on the tensor cores
            a_planes_kernel<<<rows, 256, 0, s>>>(D, Dp, rn, (float)s_a, a.a_pl);
            b_planes_kernel<<<rows, 256, 0, s>>>(D, Dp, split_vbuf(t), (float)s_b, a.b_pl);
            count_launches(2);
            QED_CUDA_TRY(tc_gemm_launch(a.g, a.c_slices, m->err, s));
            acc_kernel<<<rows, 256, 0, s>>>(D, Dp, a.g.splits, a.c_slices, o_scale / (s_a * s_b), Nacc);
            count_launches(1);
        }
    }
    // M = Nacc U^+, then the Frechet contraction
    zgemm(s, D, D, D, 1.0, Nacc, D, m->U, D, true, 0.0, Macc, D);
    ADJ_TRY(frechet_gradients(m, B, Macc, grad_g, grad_zeta, s));
    uint32_t flags[2] = {0, 0};
    QED_CUDA_TRY(cudaMemcpy(&flags[0], m->err, 4, cudaMemcpyDeviceToHost));
    QED_CUDA_TRY(cudaMemcpy(&flags[1], t->err, 4, cudaMemcpyDeviceToHost));
    if ((flags[0] | flags[1]) & kErrTimeout) {
        QED_CUDA_TRY(cudaMemset(m->err, 0, 4));
        QED_CUDA_TRY(cudaMemset(t->err, 0, 4));
        set_error("qed_adjoint: a bounded device wait ran out");
        return QED_ETIMEOUT;
    }
    if (flags[0] & kErrNotDensity) {
        QED_CUDA_TRY(cudaMemset(m->err, 0, 4));
        set_error("qed_adjoint: split precision needs a Hermitian rho0 of unit trace");
        return QED_EINVAL;
    }
    return QED_OK;
}

// The adjoint of the Strang step in split precision.  Forward: X_n = E(rho_n), V_n =
// U X_n U^+, rho_{n+1} = E(V_n), E the explicit-midpoint half step (tau = dt/2) of the
// Lindblad term, run as the model's own stages so that rho_n, X_n and V_n of a segment are
// kept.  Backward: the twin model (U^+, conjugate phases, the outgoing jump lists, i.e. the
// adjoint Lindblad term) runs the same stages on the co-state: kappa_n = E^+(lambda_{n+1})
// (its first stage T = lambda + tau/2 L^+ lambda in the stage buffer), mu_n = U^+ kappa_n U
// (its V buffer), lambda_n = E^+(mu_n).  M = (sum_n X_n mu_n) U^+ with one FP16 hi/lo
// tensor-core product per step accumulated in FP64; every rate gradient gets
// tau tr(T D_j Y) + tau^2/2 tr(Lam D_j(L Y)) from each half step (Lam, Y) = (lambda_{n+1},
// V_n) and (mu_n, rho_n), L Y applied by the forward model's Lindblad kernel.
qed_status adjoint_strang_split(qed_model *m, const void *rho0, int64_t N, int64_t k, const double *obs_diag,
                                double *loss, double *grad_g, double *grad_zeta, double *grad_gamma, cudaStream_t s) {
    {
        const qed_status st = make_twin(m, s);
        if (st != QED_OK) {  // nothing half-built is kept for the next call
            cudaStreamSynchronize(s);
            adjoint_release(m);
            return st;
        }
    }
    AdjointState &a = *m->adj;
    qed_model *t = a.twin;
    k = std::min<int64_t>(k, std::max<int64_t>(N, 1));
    const int64_t D = m->D, Dp = a.Dp;
    const size_t DD = (size_t)(D * D);
    const int64_t n_ck = N > 0 ? (N - 1) / k + 1 : 0;
    const double dt = m->dt, tau = 0.5 * dt;
    // the co-state runs for o / 2^e (see adjoint_split)
    std::vector<double> ho((size_t)D);
    QED_CUDA_TRY(cudaMemcpyAsync(ho.data(), obs_diag, (size_t)D * 8, cudaMemcpyDeviceToHost, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    double omax = 0.0;
    for (double x : ho) omax = std::max(omax, std::abs(x));
    const int e = omax > 0.0 ? (int)std::ceil(std::log2(omax)) : 0;
    const double o_scale = std::ldexp(1.0, e);
    for (double &x : ho) x = std::ldexp(x, -e);
    const double s_a = std::ldexp(1.0, 14), s_b = std::ldexp(1.0, 14);
    Buffers B;
    float4 *ck = nullptr, *seg_rho = nullptr, *seg_x = nullptr, *seg_v = nullptr, *Ly = nullptr;
    double2 *Nacc = nullptr, *Macc = nullptr;
    double *r = nullptr, *o_s = nullptr;
    ADJ_TRY(B.get(&o_s, (size_t)D));
    QED_CUDA_TRY(cudaMemcpyAsync(o_s, ho.data(), (size_t)D * 8, cudaMemcpyHostToDevice, s));
    ADJ_TRY(B.get(&ck, DD * (size_t)std::max<int64_t>(n_ck, 1)));
    ADJ_TRY(B.get(&seg_rho, DD * (size_t)k));
    ADJ_TRY(B.get(&seg_x, DD * (size_t)k));
    ADJ_TRY(B.get(&seg_v, DD * (size_t)k));
    ADJ_TRY(B.get(&Ly, DD));
    ADJ_TRY(B.get(&Nacc, DD));
    ADJ_TRY(B.get(&Macc, DD));
    ADJ_TRY(B.get(&r, (size_t)D));
    auto copy = [&](float4 *dst, const float4 *src) {
        return cudaMemcpyAsync(dst, src, DD * 16, cudaMemcpyDeviceToDevice, s);
    };
    // one forward step of the state (in place), keeping X_n and V_n when asked
    auto fwd_step = [&](float4 *x_out, float4 *v_out) -> cudaError_t {
        split_lindblad_stage(m, 0, 0, 2, 0.25f, 0, s);  // Y = rho + dt/4 L(rho)
        split_lindblad_stage(m, 2, 0, 0, 0.5f, 1, s);   // X_n = rho + dt/2 L(Y), and its planes
        cudaError_t ce = x_out ? copy(x_out, split_state(m)) : cudaSuccess;
        split_products(m, s);                           // V_n = U X_n U^+
        if (ce == cudaSuccess && v_out) ce = copy(v_out, split_vbuf(m));
        split_lindblad_stage(m, 1, 1, 2, 0.25f, 0, s);
        split_lindblad_stage(m, 2, 1, 0, 0.5f, 0, s);   // rho_{n+1} = E(V_n)
        return ce;
    };
    auto rate = [&](const float4 *Lam, const float4 *Y, double scale) {
        rowdot_df_kernel<<<blocks_for(D, 8), 256, 0, s>>>(D, Lam, Y, r);
        gamma_grad_df_kernel<<<a.n_jumps, 256, 0, s>>>(D, a.je_ptr, a.je_src, a.je_dst, a.je_coef, Lam, Y, r, scale,
                                                       grad_gamma);
        count_launches(2);
    };
    const int64_t last0 = (n_ck - 1) * k;  // the last segment is stored by the forward pass
    split_check_density(m, (const double2 *)rho0, s);
    ADJ_TRY(split_begin(m, (const double2 *)rho0, s));
    for (int64_t n = 0; n < N; ++n) {
        if (n % k == 0 && n < last0) QED_CUDA_TRY(copy(ck + (size_t)(n / k) * DD, split_state(m)));
        const bool keep = n >= last0;
        const size_t o = keep ? (size_t)(n - last0) * DD : 0;
        if (keep) QED_CUDA_TRY(copy(seg_rho + o, split_state(m)));
        QED_CUDA_TRY(fwd_step(keep ? seg_x + o : nullptr, keep ? seg_v + o : nullptr));
    }
    loss_df_kernel<<<1, 256, 0, s>>>(D, split_state(m), obs_diag, loss);
    set_diag_df_kernel<<<blocks_for((int64_t)DD, 256), 256, 0, s>>>(D, o_s, split_state(t));  // lambda_N
    count_launches(2);
    QED_CUDA_TRY(cudaMemsetAsync(Nacc, 0, DD * 16, s));
    if (a.n_jumps > 0) QED_CUDA_TRY(cudaMemsetAsync(grad_gamma, 0, (size_t)a.n_jumps * 8, s));
    const dim3 rows(blocks_for(D, 256), (unsigned)D);
    const double r1 = o_scale * tau, r2 = o_scale * 0.5 * tau * tau / dt;  // Ly holds dt L(Y)
    for (int64_t c = n_ck - 1; c >= 0; --c) {
        const int64_t s0 = c * k, s1 = std::min(N, s0 + k);
        if (c < n_ck - 1) {  // recompute the segment, keeping rho_n, X_n and V_n
            QED_CUDA_TRY(copy(split_state(m), ck + (size_t)c * DD));
            for (int64_t n = s0; n < s1; ++n) {
                const size_t o = (size_t)(n - s0) * DD;
                QED_CUDA_TRY(copy(seg_rho + o, split_state(m)));
                QED_CUDA_TRY(fwd_step(seg_x + o, seg_v + o));
            }
        }
        for (int64_t n = s1 - 1; n >= s0; --n) {
            const size_t o = (size_t)(n - s0) * DD;
            const float4 *rn = seg_rho + o, *xn = seg_x + o, *vn = seg_v + o;
            // kappa_n = E^+(lambda_{n+1}) with the rate terms of the trailing half step
            if (a.n_jumps > 0) {
                split_apply_lindblad(m, vn, Ly, s);
                rate(split_state(t), Ly, r2);
            }
            split_lindblad_stage(t, 0, 0, 2, 0.25f, 0, s);
            if (a.n_jumps > 0) rate(split_ybuf(t), vn, r1);
            split_lindblad_stage(t, 2, 0, 0, 0.5f, 1, s);
            // mu_n = U^+ kappa_n U;  Nacc += X_n mu_n on the tensor cores
            split_products(t, s);
            a_planes_kernel<<<rows, 256, 0, s>>>(D, Dp, xn, (float)s_a, a.a_pl);
            b_planes_kernel<<<rows, 256, 0, s>>>(D, Dp, split_vbuf(t), (float)s_b, a.b_pl);
            count_launches(2);
            QED_CUDA_TRY(tc_gemm_launch(a.g, a.c_slices, m->err, s));
            acc_kernel<<<rows, 256, 0, s>>>(D, Dp, a.g.splits, a.c_slices, o_scale / (s_a * s_b), Nacc);
            count_launches(1);
            // lambda_n = E^+(mu_n) with the rate terms of the leading half step
            if (a.n_jumps > 0) {
                split_apply_lindblad(m, rn, Ly, s);
                rate(split_vbuf(t), Ly, r2);
            }
            split_lindblad_stage(t, 1, 1, 2, 0.25f, 0, s);
            if (a.n_jumps > 0) rate(split_ybuf(t), rn, r1);
            split_lindblad_stage(t, 2, 1, 0, 0.5f, 0, s);
        }
    }
    // M = Nacc U^+, then the Frechet contraction
    zgemm(s, D, D, D, 1.0, Nacc, D, m->U, D, true, 0.0, Macc, D);
    ADJ_TRY(frechet_gradients(m, B, Macc, grad_g, grad_zeta, s));
    uint32_t flags[2] = {0, 0};
    QED_CUDA_TRY(cudaMemcpy(&flags[0], m->err, 4, cudaMemcpyDeviceToHost));
    QED_CUDA_TRY(cudaMemcpy(&flags[1], t->err, 4, cudaMemcpyDeviceToHost));
    if ((flags[0] | flags[1]) & kErrTimeout) {
        QED_CUDA_TRY(cudaMemset(m->err, 0, 4));
        QED_CUDA_TRY(cudaMemset(t->err, 0, 4));
        set_error("qed_adjoint: a bounded device wait ran out");
        return QED_ETIMEOUT;
    }
    if (flags[0] & kErrNotDensity) {
        QED_CUDA_TRY(cudaMemset(m->err, 0, 4));
        set_error("qed_adjoint: split precision needs a Hermitian rho0 of unit trace");
        return QED_EINVAL;
    }
    return QED_OK;
}

// The adjoint of the Strang step on the FP64 path.  Forward: X_n = E(rho_n),
// V_n = U X_n U^+, rho_{n+1} = E(V_n), E the explicit-midpoint half step (tau = dt/2) of the
// Lindblad term.  Backward: kappa_n = E^+(lambda_{n+1}), mu_n = U^+ kappa_n U,
// lambda_n = E^+(mu_n), with E^+(Lam) = Lam + tau L^+(T), T = Lam + tau/2 L^+(Lam) (L^+ from
// the outgoing jump lists); M = sum_n X_n U^+ kappa_n for the Frechet contraction; every rate
// gradient gets tau tr(T D_j(Y)) + tau^2/2 tr(Lam D_j(L Y)) from each half step (Lam, Y) =
// (lambda_{n+1}, V_n) and (mu_n, rho_n).
qed_status adjoint_strang_f64(qed_model *m, const void *rho0, int64_t N, int64_t k, const double *obs_diag,
                              double *loss, double *grad_g, double *grad_zeta, double *grad_gamma, cudaStream_t s) {
    AdjointState &a = *m->adj;
    const int64_t D = m->D;
    const size_t DD = (size_t)(D * D);
    k = std::min<int64_t>(k, std::max<int64_t>(N, 1));
    const int64_t n_ck = N > 0 ? (N - 1) / k + 1 : 0;
    const double tau = 0.5 * m->dt;
    Buffers B;
    double2 *ck = nullptr, *seg_rho = nullptr, *seg_x = nullptr, *seg_v = nullptr, *rho = nullptr, *lam = nullptr,
            *kap = nullptr, *mu = nullptr, *T1 = nullptr, *Ly = nullptr, *Z = nullptr, *Macc = nullptr, *T = nullptr;
    double *r = nullptr;
    ADJ_TRY(B.get(&ck, DD * (size_t)std::max<int64_t>(n_ck, 1)));
    ADJ_TRY(B.get(&seg_rho, DD * (size_t)k));
    ADJ_TRY(B.get(&seg_x, DD * (size_t)k));
    ADJ_TRY(B.get(&seg_v, DD * (size_t)k));
    for (double2 **q : {&rho, &lam, &kap, &mu, &T1, &Ly, &Z, &Macc, &T}) ADJ_TRY(B.get(q, DD));
    ADJ_TRY(B.get(&r, (size_t)D));
    QED_CUDA_TRY(cudaMemsetAsync(Z, 0, DD * 16, s));
    // forward L stages (incoming lists) and backward L^+ stages (outgoing lists)
    auto fwd = [&](const double2 *X, const double2 *Bv, double2 *out, double t) {
        lindblad_axpy_f64(s, D, X, Bv, out, m->anti, m->in_ptr, m->in_jump, m->in_src, m->in_coef, t);
    };
    auto bwd = [&](const double2 *X, const double2 *Bv, double2 *out, double t) {
        lindblad_axpy_f64(s, D, X, Bv, out, m->anti, a.out_ptr, a.out_jump, a.out_dst, a.out_coef, t);
    };
    // one forward step from rho (in place), keeping X and V
    auto step = [&](double2 *x, double2 *v) {
        fwd(rho, rho, T1, 0.5 * tau);
        fwd(T1, rho, x, tau);
        zgemm(s, D, D, D, 1.0, m->U, D, x, D, false, 0.0, T, D);
        zgemm(s, D, D, D, 1.0, T, D, m->U, D, true, 0.0, v, D);
        fwd(v, v, T1, 0.5 * tau);
        fwd(T1, v, rho, tau);
    };
    auto rate = [&](const double2 *Lam, const double2 *Y, double scale) {
        rowdot_kernel<<<blocks_for(D, 8), 256, 0, s>>>(D, Lam, Y, r);
        gamma_grad_kernel<<<a.n_jumps, 256, 0, s>>>(D, a.je_ptr, a.je_src, a.je_dst, a.je_coef, Lam, Y, r, scale,
                                                    grad_gamma);
        count_launches(2);
    };
    const int64_t last0 = (n_ck - 1) * k;  // the last segment is stored by the forward pass
    QED_CUDA_TRY(cudaMemcpyAsync(rho, rho0, DD * 16, cudaMemcpyDeviceToDevice, s));
    for (int64_t n = 0; n < N; ++n) {
        if (n % k == 0 && n < last0)
            QED_CUDA_TRY(cudaMemcpyAsync(ck + (size_t)(n / k) * DD, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
        const bool keep = n >= last0;
        const size_t o = keep ? (size_t)(n - last0) * DD : 0;
        if (keep) QED_CUDA_TRY(cudaMemcpyAsync(seg_rho + o, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
        step(keep ? seg_x + o : Ly, keep ? seg_v + o : mu);
    }
    loss_kernel<<<1, 256, 0, s>>>(D, rho, obs_diag, loss);
    set_diag_kernel<<<blocks_for((int64_t)DD, 256), 256, 0, s>>>(D, obs_diag, lam);
    count_launches(2);
    QED_CUDA_TRY(cudaMemsetAsync(Macc, 0, DD * 16, s));
    if (a.n_jumps > 0) QED_CUDA_TRY(cudaMemsetAsync(grad_gamma, 0, (size_t)a.n_jumps * 8, s));
    for (int64_t c = n_ck - 1; c >= 0; --c) {
        const int64_t s0 = c * k, s1 = std::min(N, s0 + k);
        if (c < n_ck - 1) {  // recompute the segment, keeping rho_n, X_n and V_n
            QED_CUDA_TRY(cudaMemcpyAsync(rho, ck + (size_t)c * DD, DD * 16, cudaMemcpyDeviceToDevice, s));
            for (int64_t n = s0; n < s1; ++n) {
                const size_t o = (size_t)(n - s0) * DD;
                QED_CUDA_TRY(cudaMemcpyAsync(seg_rho + o, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
                step(seg_x + o, seg_v + o);
            }
        }
        for (int64_t n = s1 - 1; n >= s0; --n) {
            const size_t o = (size_t)(n - s0) * DD;
            const double2 *rn = seg_rho + o, *xn = seg_x + o, *vn = seg_v + o;
            // kappa_n = E^+(lambda_{n+1}), its stage T1
            bwd(lam, lam, T1, 0.5 * tau);
            bwd(T1, lam, kap, tau);
            if (a.n_jumps > 0) {
                fwd(vn, Z, Ly, 1.0);  // L(V_n)
                rate(T1, vn, tau);
                rate(lam, Ly, 0.5 * tau * tau);
            }
            // M += X_n U^+ kappa_n;  mu_n = U^+ kappa_n U
            zgemm(s, D, D, D, 1.0, xn, D, m->U, D, true, 0.0, T, D);
            zgemm(s, D, D, D, 1.0, T, D, kap, D, false, 1.0, Macc, D);
            zgemm(s, D, D, D, 1.0, kap, D, m->U, D, false, 0.0, T, D);
            zgemm_ex(s, D, D, D, 1.0, m->U, D, true, T, D, false, 0.0, mu, D);
            // lambda_n = E^+(mu_n), its stage T1
            bwd(mu, mu, T1, 0.5 * tau);
            bwd(T1, mu, lam, tau);
            if (a.n_jumps > 0) {
                fwd(rn, Z, Ly, 1.0);  // L(rho_n)
                rate(T1, rn, tau);
                rate(mu, Ly, 0.5 * tau * tau);
            }
        }
    }
    return frechet_gradients(m, B, Macc, grad_g, grad_zeta, s);
}

}  // namespace

void adjoint_release(qed_model *m) {
    AdjointState *a = m->adj;
    if (!a) return;
    void *ptrs[] = {a->out_ptr, a->out_jump, a->out_dst, a->out_coef, a->je_ptr, a->je_src,   a->je_dst, a->je_coef,
                    a->pe_ptr,  a->pe_row,   a->pe_col,  a->pe_unit,  a->H,      a->a_pl,     a->b_pl,   a->c_slices};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (a->twin) qed_free(a->twin);
    delete a;
    m->adj = nullptr;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_adjoint(qed_model *m, const void *rho0, int64_t n_steps, int32_t checkpoint_every,
                                  const double *obs_diag, double *loss, double *grad_g, double *grad_zeta,
                                  double *grad_gamma, qed_stream stream) {
    if (!m || !rho0 || !obs_diag || !loss) {
        set_error("qed_adjoint: NULL argument");
        return QED_EINVAL;
    }
    if (n_steps < 0 || checkpoint_every <= 0) {
        set_error("qed_adjoint: n_steps >= 0 and checkpoint_every > 0 required");
        return QED_EINVAL;
    }
    if (m->scheme == QED_SCHEME_EFFECTIVE) {
        set_error("qed_adjoint: the effective-Hamiltonian step is not differentiated");
        return QED_EUNSUPPORTED;
    }
    NvtxRange range("qed_adjoint");
    {
        // a failed set-up (e.g. out of device memory) leaves no half-built tables behind
        const qed_status st = setup(m);
        if (st != QED_OK) {
            adjoint_release(m);
            return st;
        }
    }
    AdjointState &a = *m->adj;
    if ((a.n_g > 0 && !grad_g) || (a.n_zeta > 0 && !grad_zeta) || (a.n_jumps > 0 && !grad_gamma)) {
        set_error("qed_adjoint: gradient buffers missing");
        return QED_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (m->prec != QED_FP64 && m->scheme == QED_SCHEME_STRANG)
        return adjoint_strang_split(m, rho0, n_steps, checkpoint_every, obs_diag, loss, grad_g, grad_zeta, grad_gamma,
                                    s);
    if (m->prec != QED_FP64)
        return adjoint_split(m, rho0, n_steps, checkpoint_every, obs_diag, loss, grad_g, grad_zeta, grad_gamma, s);
    if (m->scheme == QED_SCHEME_STRANG)
        return adjoint_strang_f64(m, rho0, n_steps, checkpoint_every, obs_diag, loss, grad_g, grad_zeta, grad_gamma,
                                  s);
    const int64_t D = m->D;
    const size_t DD = (size_t)(D * D);
    const int64_t N = n_steps, k = std::min<int64_t>(checkpoint_every, std::max<int64_t>(n_steps, 1));
    const int64_t n_ck = N > 0 ? (N - 1) / k + 1 : 0;
    const double dt = m->dt;
    Buffers B;
    double2 *ck = nullptr, *seg_rho = nullptr, *seg_v = nullptr, *rho = nullptr, *lam = nullptr, *kap = nullptr,
            *Macc = nullptr, *T = nullptr;
    double *r = nullptr;
    ADJ_TRY(B.get(&ck, DD * (size_t)std::max<int64_t>(n_ck, 1)));
    ADJ_TRY(B.get(&seg_rho, DD * (size_t)k));
    ADJ_TRY(B.get(&seg_v, DD * (size_t)k));
    ADJ_TRY(B.get(&rho, DD));
    ADJ_TRY(B.get(&lam, DD));
    ADJ_TRY(B.get(&kap, DD));
    ADJ_TRY(B.get(&Macc, DD));
    ADJ_TRY(B.get(&T, DD));
    ADJ_TRY(B.get(&r, (size_t)D));
    // forward with checkpoints (FP64 step: V = (U rho) U^+, then Eq. 3)
    const int64_t last0 = (n_ck - 1) * k;  // the last segment is stored by the forward pass
    QED_CUDA_TRY(cudaMemcpyAsync(rho, rho0, DD * 16, cudaMemcpyDeviceToDevice, s));
    for (int64_t n = 0; n < N; ++n) {
        if (n % k == 0 && n < last0)
            QED_CUDA_TRY(cudaMemcpyAsync(ck + (size_t)(n / k) * DD, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
        double2 *vn = m->work2;
        if (n >= last0) {
            QED_CUDA_TRY(cudaMemcpyAsync(seg_rho + (size_t)(n - last0) * DD, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
            vn = seg_v + (size_t)(n - last0) * DD;
        }
        zgemm(s, D, D, D, 1.0, m->U, D, rho, D, false, 0.0, m->work1, D);
        zgemm(s, D, D, D, 1.0, m->work1, D, m->U, D, true, 0.0, vn, D);
        dissipate_f64(s, D, vn, rho, m->anti, m->in_ptr, m->in_jump, m->in_src, m->in_coef, dt);
    }
    loss_kernel<<<1, 256, 0, s>>>(D, rho, obs_diag, loss);
    count_launches(1);
    // co-state
    set_diag_kernel<<<blocks_for((int64_t)DD, 256), 256, 0, s>>>(D, obs_diag, lam);
    count_launches(1);
    QED_CUDA_TRY(cudaMemsetAsync(Macc, 0, DD * 16, s));
    if (a.n_jumps > 0) QED_CUDA_TRY(cudaMemsetAsync(grad_gamma, 0, (size_t)a.n_jumps * 8, s));
    for (int64_t c = n_ck - 1; c >= 0; --c) {
        const int64_t s0 = c * k, s1 = std::min(N, s0 + k);
        // recompute the segment, storing rho_n and V_n
        if (c < n_ck - 1)
            QED_CUDA_TRY(cudaMemcpyAsync(rho, ck + (size_t)c * DD, DD * 16, cudaMemcpyDeviceToDevice, s));
        for (int64_t n = s0; n < s1 && c < n_ck - 1; ++n) {
            double2 *vn = seg_v + (size_t)(n - s0) * DD;
            QED_CUDA_TRY(cudaMemcpyAsync(seg_rho + (size_t)(n - s0) * DD, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
            zgemm(s, D, D, D, 1.0, m->U, D, rho, D, false, 0.0, m->work1, D);
            zgemm(s, D, D, D, 1.0, m->work1, D, m->U, D, true, 0.0, vn, D);
            dissipate_f64(s, D, vn, rho, m->anti, m->in_ptr, m->in_jump, m->in_src, m->in_coef, dt);
        }
        for (int64_t n = s1 - 1; n >= s0; --n) {
            const double2 *rn = seg_rho + (size_t)(n - s0) * DD, *vn = seg_v + (size_t)(n - s0) * DD;
            // dL/dgamma_j += dt tr(lambda_{n+1} D_j(V_n))
            if (a.n_jumps > 0) {
                rowdot_kernel<<<blocks_for(D, 8), 256, 0, s>>>(D, lam, vn, r);
                gamma_grad_kernel<<<a.n_jumps, 256, 0, s>>>(D, a.je_ptr, a.je_src, a.je_dst, a.je_coef, lam, vn, r,
                                                            dt, grad_gamma);
                count_launches(2);
            }
            // kappa = J^+(lambda_{n+1}): the Lindblad update with the outgoing lists
            dissipate_f64(s, D, lam, kap, m->anti, a.out_ptr, a.out_jump, a.out_dst, a.out_coef, dt);
            // M += rho_n U^+ kappa
            zgemm(s, D, D, D, 1.0, rn, D, m->U, D, true, 0.0, T, D);
            zgemm(s, D, D, D, 1.0, T, D, kap, D, false, 1.0, Macc, D);
            // lambda_n = U^+ kappa U
            zgemm(s, D, D, D, 1.0, kap, D, m->U, D, false, 0.0, T, D);
            zgemm_ex(s, D, D, D, 1.0, m->U, D, true, T, D, false, 0.0, lam, D);
        }
    }
    ADJ_TRY(frechet_gradients(m, B, Macc, grad_g, grad_zeta, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}
