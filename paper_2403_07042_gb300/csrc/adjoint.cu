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
// dL/dtheta = 2 dt Im tr(G dH/dtheta).  G is the upper-right block of
// exp([[X, M], [0, X]]) (Najfeld and Havel; Higham 2008, Sec. 10.6), computed with the same
// Pade-13 routine as U.  rho is checkpointed every k steps and each segment recomputed
// (storing its rho_n and V_n) while stepping the co-state back.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.h"
#include "model.h"

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
};

namespace {

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class T>
qed_status up(T **dst, const std::vector<T> &v) {
    const size_t n = std::max<size_t>(v.size(), 1);
    if (cudaMalloc((void **)dst, n * sizeof(T)) != cudaSuccess) {
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

// B = [[X, tau M], [0, X]] with X = -i dt H (2D x 2D)
__global__ void block_kernel(int64_t D, const double2 *H, double dt, const double2 *M, double tau, double2 *B) {
    const int64_t W = 2 * D;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= W * W) return;
    const int64_t r = idx / W, c = idx % W;
    double2 v = make_double2(0.0, 0.0);
    if ((r < D) == (c < D)) {
        const double2 h = H[(r % D) * D + (c % D)];
        v = make_double2(dt * h.y, -dt * h.x);
    } else if (r < D && c >= D) {
        const double2 x = M[r * D + (c - D)];
        v = make_double2(tau * x.x, tau * x.y);
    }
    B[idx] = v;
}

// grad[p] = 2 dt Im sum_e unit_e G[col_e][row_e] / tau, G the upper-right block of R
__global__ void param_grad_kernel(int64_t D, int np, const int32_t *pe_ptr, const int32_t *pe_row,
                                  const int32_t *pe_col, const double *pe_unit, const double2 *R, double scale,
                                  double *grad_g, int n_g, double *grad_zeta) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int e = pe_ptr[p]; e < pe_ptr[p + 1]; ++e) s += pe_unit[e] * R[(int64_t)pe_col[e] * 2 * D + D + pe_row[e]].y;
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
        if (cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed for the adjoint work space");
            return QED_ENOMEM;
        }
        ptrs.push_back(*p);
        return QED_OK;
    }
};

}  // namespace

void adjoint_release(qed_model *m) {
    AdjointState *a = m->adj;
    if (!a) return;
    void *ptrs[] = {a->out_ptr, a->out_jump, a->out_dst, a->out_coef, a->je_ptr,  a->je_src, a->je_dst,
                    a->je_coef, a->pe_ptr,   a->pe_row,  a->pe_col,   a->pe_unit, a->H};
    for (void *p : ptrs)
        if (p) cudaFree(p);
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
    ADJ_TRY(setup(m));
    AdjointState &a = *m->adj;
    if ((a.n_g > 0 && !grad_g) || (a.n_zeta > 0 && !grad_zeta) || (a.n_jumps > 0 && !grad_gamma)) {
        set_error("qed_adjoint: gradient buffers missing");
        return QED_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t D = m->D;
    const size_t DD = (size_t)(D * D);
    const int64_t N = n_steps, k = checkpoint_every;
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
    QED_CUDA_TRY(cudaMemcpyAsync(rho, rho0, DD * 16, cudaMemcpyDeviceToDevice, s));
    for (int64_t n = 0; n < N; ++n) {
        if (n % k == 0)
            QED_CUDA_TRY(cudaMemcpyAsync(ck + (size_t)(n / k) * DD, rho, DD * 16, cudaMemcpyDeviceToDevice, s));
        zgemm(s, D, D, D, 1.0, m->U, D, rho, D, false, 0.0, m->work1, D);
        zgemm(s, D, D, D, 1.0, m->work1, D, m->U, D, true, 0.0, m->work2, D);
        dissipate_f64(s, D, m->work2, rho, m->anti, m->in_ptr, m->in_jump, m->in_src, m->in_coef, dt);
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
        QED_CUDA_TRY(cudaMemcpyAsync(rho, ck + (size_t)c * DD, DD * 16, cudaMemcpyDeviceToDevice, s));
        for (int64_t n = s0; n < s1; ++n) {
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
    // G = L_exp(X, M): upper-right block of exp([[X, tau M], [0, X]])
    if (a.n_g + a.n_zeta > 0) {
        std::vector<double2> hM(DD);
        QED_CUDA_TRY(cudaMemcpyAsync(hM.data(), Macc, DD * 16, cudaMemcpyDeviceToHost, s));
        QED_CUDA_TRY(cudaStreamSynchronize(s));
        double mnorm = 0.0;
        for (int64_t cc = 0; cc < D; ++cc) {
            double col = 0.0;
            for (int64_t rr = 0; rr < D; ++rr) col += std::hypot(hM[(size_t)(rr * D + cc)].x, hM[(size_t)(rr * D + cc)].y);
            mnorm = std::max(mnorm, col);
        }
        const double xnorm = dt * a.h_norm1;
        double tau = 1.0;
        if (mnorm > 0.0 && xnorm > 0.0) tau = std::ldexp(1.0, (int)std::floor(std::log2(xnorm / mnorm)));
        double2 *blk = nullptr, *R = nullptr;
        ADJ_TRY(B.get(&blk, 4 * DD));
        ADJ_TRY(B.get(&R, 4 * DD));
        block_kernel<<<blocks_for((int64_t)(4 * DD), 256), 256, 0, s>>>(D, a.H, dt, Macc, tau, blk);
        count_launches(1);
        ADJ_TRY(expm_pade13(s, 2 * D, blk, xnorm + tau * mnorm, R, m->err));
        const int np = a.n_g + a.n_zeta;
        param_grad_kernel<<<blocks_for(np, 128), 128, 0, s>>>(D, np, a.pe_ptr, a.pe_row, a.pe_col, a.pe_unit, R,
                                                              2.0 * dt / tau, grad_g, a.n_g, grad_zeta);
        count_launches(1);
    }
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}
