// The C ABI of libqed (declared in include/qed.h): argument checks, model lifetime,
// the propagator stage and the step loop.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "kernels.h"
#include "model.h"
#include "split.h"

namespace qed {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

namespace {
std::atomic<int64_t> g_alloc_budget{-1};  // bytes the library may still allocate (< 0: no limit)
}

cudaError_t device_malloc(void **p, size_t bytes) {
    int64_t left = g_alloc_budget.load();
    while (left >= 0) {
        if ((int64_t)bytes > left) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_budget.compare_exchange_weak(left, left - (int64_t)bytes)) break;
    }
    return cudaMalloc(p, bytes);
}

namespace {

qed_status einval(const std::string &msg) {
    set_error(msg);
    return QED_EINVAL;
}

template <class T>
qed_status dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = device_malloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? QED_ENOMEM : QED_ECUDA;
    }
    return QED_OK;
}

#define QED_TRY(expr)                       \
    do {                                    \
        qed_status st_ = (expr);            \
        if (st_ != QED_OK) return st_;      \
    } while (0)

void release(qed_model *m) {
    if (!m) return;
    for (auto &g : m->graph)
        if (g) cudaGraphExecDestroy(g);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    void *ptrs[] = {m->U,      m->work1,   m->work2, m->work3,       m->phase,   m->anti, m->in_ptr,
                    m->in_jump, m->in_src, m->in_coef, m->obs_w, m->obs_ids_dev, m->scalars, m->err,
                    m->rho_int, m->gate, m->anti_zero};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->err_host) cudaFreeHost(m->err_host);
    split_release(m);
    adjoint_release(m);
    for (auto &e : m->ev)
        if (e) cudaEventDestroy(e);
    delete m;
}

qed_status upload_tables(qed_model *m) {
    const HostModel &hm = m->host;
    const int64_t D = m->D;
    // incoming jump lists, grouped by destination row and sorted by jump id
    std::vector<std::vector<JumpEntry>> rows((size_t)D);
    for (const auto &e : hm.jumps) rows[(size_t)e.dst].push_back(e);
    std::vector<int32_t> ptr((size_t)D + 1, 0), jump, src;
    std::vector<double> coef;
    int32_t max_in = 0;
    for (int64_t r = 0; r < D; ++r) {
        auto &v = rows[(size_t)r];
        std::sort(v.begin(), v.end(), [](const JumpEntry &a, const JumpEntry &b) { return a.jump < b.jump; });
        for (const auto &e : v) {
            jump.push_back(e.jump);
            src.push_back((int32_t)e.src);
            coef.push_back(e.coef * std::sqrt(hm.gamma[(size_t)e.jump]));
        }
        ptr[(size_t)r + 1] = (int32_t)jump.size();
        max_in = std::max(max_in, (int32_t)v.size());
    }
    m->n_in = (int64_t)jump.size();
    m->max_in = max_in;
    QED_TRY(dev_alloc(&m->in_ptr, ptr.size()));
    QED_TRY(dev_alloc(&m->in_jump, jump.size()));
    QED_TRY(dev_alloc(&m->in_src, src.size()));
    QED_TRY(dev_alloc(&m->in_coef, coef.size()));
    QED_CUDA_TRY(cudaMemcpy(m->in_ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice));
    if (!jump.empty()) {
        QED_CUDA_TRY(cudaMemcpy(m->in_jump, jump.data(), jump.size() * 4, cudaMemcpyHostToDevice));
        QED_CUDA_TRY(cudaMemcpy(m->in_src, src.data(), src.size() * 4, cudaMemcpyHostToDevice));
        QED_CUDA_TRY(cudaMemcpy(m->in_coef, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice));
    }
    QED_TRY(dev_alloc(&m->anti, (size_t)D));
    QED_CUDA_TRY(cudaMemcpy(m->anti, hm.anti_diag.data(), (size_t)D * 8, cudaMemcpyHostToDevice));
    // observables: trace, photons per cavity, atoms, extra digits
    const Layout &L = hm.layout;
    const int nd = L.n_digits();
    std::vector<int> digit_of;
    for (int p : L.photon_digit) digit_of.push_back(p);
    for (int p : L.atom_digit) digit_of.push_back(p);
    for (int p : L.extra_digit) digit_of.push_back(p);
    m->n_named = 1 + (int32_t)digit_of.size();
    std::vector<double> w((size_t)m->n_named * (size_t)D, 0.0);
    for (int64_t k = 0; k < D; ++k) {
        w[(size_t)k] = 1.0;
        for (size_t q = 0; q < digit_of.size(); ++q)
            w[(size_t)(q + 1) * (size_t)D + (size_t)k] = hm.digits[(size_t)k * nd + digit_of[q]];
    }
    QED_TRY(dev_alloc(&m->obs_w, w.size()));
    QED_CUDA_TRY(cudaMemcpy(m->obs_w, w.data(), w.size() * 8, cudaMemcpyHostToDevice));
    QED_TRY(dev_alloc(&m->phase, (size_t)D));  // values: compute_propagator
    return QED_OK;
}

qed_status ensure_ids(qed_model *m, int32_t n_obs, const int32_t *ids, cudaStream_t s) {
    if (n_obs <= 0) return QED_OK;
    if (!ids) return einval("obs_ids is NULL");
    const int32_t lim = (int32_t)m->D + m->n_named;
    for (int32_t o = 0; o < n_obs; ++o)
        if (ids[o] < 0 || ids[o] >= lim) return einval("observable id out of range");
    if (n_obs > m->obs_ids_cap) {
        if (m->obs_ids_dev) {
            cudaStreamSynchronize(s);
            cudaFree(m->obs_ids_dev);
            m->obs_ids_dev = nullptr;
        }
        QED_TRY(dev_alloc(&m->obs_ids_dev, (size_t)n_obs));
        m->obs_ids_cap = n_obs;
    }
    QED_CUDA_TRY(cudaMemcpyAsync(m->obs_ids_dev, ids, (size_t)n_obs * 4, cudaMemcpyHostToDevice, s));
    return QED_OK;
}


// One FP64 step.  Lie: V = (U rho) U^+, then the Euler update of Eq. 3 into rho.  Strang:
// rho <- E(dt/2) rho, V = U rho U^+, rho <- E(dt/2) V, each E(t) X = X + t L(X + t/2 L(X))
// as two stages through work3.  With `ev`, records an event before every kernel and after
// the last; returns the number of kernels and names them in `label`.
int step_f64(qed_model *m, double2 *rho, cudaStream_t s, cudaEvent_t *ev = nullptr, std::string *label = nullptr) {
    const int64_t D = m->D;
    const double dt = m->dt;
    const bool strang = m->scheme == QED_SCHEME_STRANG;
    // the effective-Hamiltonian step: U is U_eff and the anticommutator is inside it
    const double *anti = m->scheme == QED_SCHEME_EFFECTIVE ? m->anti_zero : m->anti;
    int e = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord(ev[e], s);
        ++e;
    };
    auto stage = [&](const double2 *X, const double2 *B, double2 *out, double tau) {
        lindblad_axpy_f64(s, D, X, B, out, anti, m->in_ptr, m->in_jump, m->in_src, m->in_coef, tau);
    };
    if (strang) {
        mark();
        stage(rho, rho, m->work3, 0.25 * dt);
        mark();
        stage(m->work3, rho, rho, 0.5 * dt);
    }
    mark();
    zgemm(s, D, D, D, 1.0, m->U, D, rho, D, false, 0.0, m->work1, D);
    mark();
    zgemm(s, D, D, D, 1.0, m->work1, D, m->U, D, true, 0.0, m->work2, D);
    mark();
    if (strang) {
        stage(m->work2, m->work2, m->work3, 0.25 * dt);
        mark();
        stage(m->work3, m->work2, rho, 0.5 * dt);
    } else {
        dissipate_f64(s, D, m->work2, rho, anti, m->in_ptr, m->in_jump, m->in_src, m->in_coef, dt);
    }
    mark();
    if (label)
        *label = strang ? "lindblad_a,lindblad_b,zgemm_f64_1,zgemm_f64_2,lindblad_c,lindblad_d"
                        : "zgemm_f64_1,zgemm_f64_2,dissipate_f64";
    return e - 1;
}

void one_step(qed_model *m, cudaStream_t s) {
    if (m->prec == QED_FP64)
        step_f64(m, m->rho_int, s);
    else
        split_step(m, s);
}

constexpr int64_t kGraphSteps = 16;

// Captures the step sequences (1 and kGraphSteps steps) into CUDA graphs on a
// library-owned stream.  Falls back to direct launches if capture is unavailable.
qed_status ensure_graphs(qed_model *m) {
    if (m->graph[0] || m->graphs_off) return QED_OK;
    if (!m->cap_stream) QED_CUDA_TRY(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    const int64_t counts[2] = {1, kGraphSteps};
    for (int g = 0; g < 2; ++g) {
        const int64_t before = launches();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            m->graphs_off = true;
            return QED_OK;
        }
        for (int64_t k = 0; k < counts[g]; ++k) one_step(m, m->cap_stream);
        cudaError_t e = cudaStreamEndCapture(m->cap_stream, &graph);
        const int64_t captured = launches() - before;
        count_launches(-captured);  // captured, not launched
        if (e != cudaSuccess || !graph) {
            cudaGetLastError();
            m->graphs_off = true;
            return QED_OK;
        }
        e = cudaGraphInstantiate(&m->graph[g], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            m->graph[g] = nullptr;
            m->graphs_off = true;
            return QED_OK;
        }
        m->graph_kernels[g] = captured;
    }
    return QED_OK;
}

// k consecutive steps with nothing to record or renormalise in between.
qed_status run_steps(qed_model *m, int64_t k, cudaStream_t s) {
    if (m->graphs_off) {
        for (int64_t i = 0; i < k; ++i) one_step(m, s);
        return QED_OK;
    }
    for (; k >= kGraphSteps; k -= kGraphSteps) {
        QED_CUDA_TRY(cudaGraphLaunch(m->graph[1], s));
        count_launches(m->graph_kernels[1]);
    }
    for (; k > 0; --k) {
        QED_CUDA_TRY(cudaGraphLaunch(m->graph[0], s));
        count_launches(m->graph_kernels[0]);
    }
    return QED_OK;
}

int64_t next_multiple_after(int64_t off, int64_t i, int64_t every) {
    // smallest p > i with (off + p) % every == 0
    return i + (every - (off + i) % every);
}

// The propagator of a scheme into m->U and the diagonal phases into m->phase ("Taylor
// approximation" stage, Sec. 4.2): for the Lie and Strang steps U = exp(-i H dt) (Pade-13 on
// the Hermitian H) and P_k = exp(-i H_kk dt); for the effective-Hamiltonian step
// U = exp(X), X = -i dt H - (dt/2) diag(d) with d_k = sum_j gamma_j (A_j^+ A_j)_kk (every
// jump operator of this library is a monomial, so A_j^+ A_j is diagonal), and
// P_k = exp(-i H_kk dt - d_k dt/2).  Synchronises `s`.
qed_status compute_propagator(qed_model *m, int scheme, cudaStream_t s) {
    NvtxRange range("propagator (Pade-13 exp(-i H dt))");
    const int64_t D = m->D;
    const double dt = m->dt;
    const HostModel &hm = m->host;
    const bool eff = scheme == QED_SCHEME_EFFECTIVE;
    std::vector<cplx> Hd;
    dense_hamiltonian(hm, Hd);
    if (eff)
        for (int64_t k = 0; k < D; ++k) {
            // X = -i dt H - (dt/2) diag(d), stored in place of H
            for (int64_t l = 0; l < D; ++l) Hd[(size_t)(k * D + l)] *= cplx(0.0, -dt);
            Hd[(size_t)(k * D + k)] -= 0.5 * dt * hm.anti_diag[(size_t)k];
        }
    double norm1 = 0.0;
    for (int64_t c = 0; c < D; ++c) {
        double col = 0.0;
        for (int64_t r = 0; r < D; ++r) col += std::abs(Hd[(size_t)(r * D + c)]);
        norm1 = std::max(norm1, col);
    }
    QED_CUDA_TRY(cudaMemcpyAsync(m->work1, Hd.data(), (size_t)(D * D) * 16, cudaMemcpyHostToDevice, s));
    if (eff)
        QED_TRY(expm_pade13(s, D, m->work1, norm1, m->U, m->err));
    else
        QED_TRY(propagator(s, D, dt, m->work1, norm1, m->U, m->err));
    QED_CUDA_TRY(cudaMemcpy(m->err_host, m->err, 4, cudaMemcpyDeviceToHost));
    if (*m->err_host & kErrSingular) {
        set_error("singular Pade denominator");
        return QED_ENUMERIC;
    }
    std::vector<double> diag((size_t)D, 0.0);
    for (const auto &e : hm.h_entries)
        if (e.row == e.col) diag[(size_t)e.row] += entry_coefficient(hm, e) * e.unit;
    std::vector<double2> ph((size_t)D);
    for (int64_t k = 0; k < D; ++k) {
        const double amp = eff ? std::exp(-0.5 * dt * hm.anti_diag[(size_t)k]) : 1.0;
        ph[(size_t)k] = make_double2(amp * std::cos(diag[(size_t)k] * dt), -amp * std::sin(diag[(size_t)k] * dt));
    }
    QED_CUDA_TRY(cudaMemcpy(m->phase, ph.data(), (size_t)D * 16, cudaMemcpyHostToDevice));
    return QED_OK;
}

// Device side of a model whose host model m->host is built: operators, tables, U, and
// the split-precision state.  Synchronises `s`.
qed_status build_device(qed_model *m, double dt, qed_precision prec, cudaStream_t s) {
    m->D = m->host.dim;
    m->dt = dt;
    m->prec = prec;
    const int64_t D = m->D;
    const size_t DD = (size_t)(D * D);
    QED_TRY(dev_alloc(&m->U, DD));
    QED_TRY(dev_alloc(&m->work1, DD));
    QED_TRY(dev_alloc(&m->work2, DD));
    QED_TRY(dev_alloc(&m->scalars, 16));
    QED_TRY(dev_alloc(&m->err, 1));
    QED_TRY(dev_alloc(&m->gate, 1));
    QED_CUDA_TRY(cudaMallocHost((void **)&m->err_host, sizeof(uint32_t)));
    *m->err_host = 0;
    QED_CUDA_TRY(cudaMemset(m->err, 0, sizeof(uint32_t)));
    QED_TRY(upload_tables(m));
    for (auto &e : m->ev) QED_CUDA_TRY(cudaEventCreate(&e));
    QED_TRY(compute_propagator(m, QED_SCHEME_LIE, s));
    if (prec != QED_FP64) QED_TRY(split_prepare(m, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    return QED_OK;
}

}  // namespace

}  // namespace qed

using namespace qed;

extern "C" {

const char *qed_last_error(void) { return g_last_error.c_str(); }

qed_status qed_launch_count(int64_t *count) {
    if (!count) return einval("count is NULL");
    *count = launches();
    return QED_OK;
}

qed_status qed_spec_dim(const qed_spec *spec, int64_t *dim, int32_t *n_digits) {
    if (!dim) return einval("dim is NULL");
    HostModel hm;
    std::string err;
    qed_status st = build_host_model(spec, hm, err, false);
    if (st != QED_OK) { set_error(err); return st; }
    *dim = hm.dim;
    if (n_digits) *n_digits = hm.layout.n_digits();
    return QED_OK;
}

qed_status qed_spec_basis(const qed_spec *spec, int32_t *digits, int64_t capacity) {
    HostModel hm;
    std::string err;
    qed_status st = build_host_model(spec, hm, err, false);
    if (st != QED_OK) { set_error(err); return st; }
    if (!digits || capacity < (int64_t)hm.digits.size()) return einval("digits buffer too small");
    for (size_t i = 0; i < hm.digits.size(); ++i) digits[i] = hm.digits[i];
    return QED_OK;
}

qed_status qed_spec_hamiltonian(const qed_spec *spec, double *H, int64_t capacity) {
    HostModel hm;
    std::string err;
    qed_status st = build_host_model(spec, hm, err, true);
    if (st != QED_OK) { set_error(err); return st; }
    if (!H || capacity < hm.dim * hm.dim) return einval("H buffer too small");
    std::vector<cplx> Hd;
    dense_hamiltonian(hm, Hd);
    std::memcpy(H, Hd.data(), Hd.size() * sizeof(cplx));
    return QED_OK;
}

qed_status qed_spec_jump(const qed_spec *spec, int32_t j, double *A, int64_t capacity) {
    HostModel hm;
    std::string err;
    qed_status st = build_host_model(spec, hm, err, true);
    if (st != QED_OK) { set_error(err); return st; }
    if (j < 0 || j >= (int32_t)hm.gamma.size()) return einval("jump index out of range");
    if (!A || capacity < hm.dim * hm.dim) return einval("A buffer too small");
    std::memset(A, 0, (size_t)(hm.dim * hm.dim) * 16);
    for (const auto &e : hm.jumps)
        if (e.jump == j) A[2 * (e.dst * hm.dim + e.src)] += e.coef;
    return QED_OK;
}

qed_status qed_spec_restricted(const qed_spec *spec, const int64_t *keep, int64_t n, int32_t j, double *out,
                               int64_t capacity, double *d) {
    if (!keep || n <= 0 || !out) return einval("qed_spec_restricted: bad argument");
    HostModel hm, sub;
    std::string err;
    qed_status st = build_host_model(spec, hm, err, true);
    if (st != QED_OK) { set_error(err); return st; }
    if (!restrict_host_model(hm, std::vector<int64_t>(keep, keep + n), sub, err)) return einval(err);
    if (capacity < n * n) return einval("qed_spec_restricted: buffer too small");
    if (j >= (int32_t)sub.gamma.size()) return einval("jump index out of range");
    if (j < 0) {
        std::vector<cplx> Hd;
        dense_hamiltonian(sub, Hd);
        std::memcpy(out, Hd.data(), Hd.size() * sizeof(cplx));
    } else {
        std::memset(out, 0, (size_t)(n * n) * 16);
        for (const auto &e : sub.jumps)
            if (e.jump == j) out[2 * (e.dst * n + e.src)] += e.coef;
    }
    if (d) std::copy(sub.anti_diag.begin(), sub.anti_diag.end(), d);
    return QED_OK;
}

qed_status qed_build(const qed_spec *spec, double dt, qed_precision prec, qed_stream stream, qed_model **out) {
    NvtxRange range("qed_build");
    if (!out) return einval("out is NULL");
    *out = nullptr;
    if (!(dt > 0.0) || !std::isfinite(dt)) return einval("dt must be finite and > 0");
    if (prec != QED_FP64 && prec != QED_SPLIT_FP16x2) {
        set_error("precision not implemented by this library");
        return QED_EUNSUPPORTED;
    }
    std::unique_ptr<qed_model, void (*)(qed_model *)> m(new qed_model(), release);
    std::string err;
    qed_status st = build_host_model(spec, m->host, err, true);
    if (st != QED_OK) { set_error(err); return st; }
    QED_TRY(build_device(m.get(), dt, prec, (cudaStream_t)stream));
    *out = m.release();
    return QED_OK;
}

qed_status qed_free(qed_model *m) {
    if (!m) return einval("model is NULL");
    cudaDeviceSynchronize();
    release(m);
    return QED_OK;
}

qed_status qed_dim(const qed_model *m, int64_t *dim) {
    if (!m || !dim) return einval("NULL argument");
    *dim = m->D;
    return QED_OK;
}

qed_status qed_basis_labels(const qed_model *m, int32_t *digits) {
    if (!m || !digits) return einval("NULL argument");
    for (size_t i = 0; i < m->host.digits.size(); ++i) digits[i] = m->host.digits[i];
    return QED_OK;
}

qed_status qed_basis_index(const qed_model *m, const int32_t *digits, int64_t *index) {
    if (!m || !digits || !index) return einval("NULL argument");
    const int nd = m->host.layout.n_digits();
    std::vector<uint8_t> d((size_t)nd);
    for (int i = 0; i < nd; ++i) {
        if (digits[i] < 0 || digits[i] >= m->host.layout.radix[(size_t)i]) {
            *index = -1;
            return einval("digit out of range");
        }
        d[(size_t)i] = (uint8_t)digits[i];
    }
    auto it = m->host.index.find(state_key(d.data(), nd));
    *index = it == m->host.index.end() ? -1 : it->second;
    if (*index < 0) return einval("state not in the basis");
    return QED_OK;
}

qed_status qed_n_observables(const qed_model *m, int32_t *n) {
    if (!m || !n) return einval("NULL argument");
    *n = (int32_t)m->D + m->n_named;
    return QED_OK;
}

qed_status qed_set_renorm_every(qed_model *m, int32_t every) {
    if (!m || every < 0) return einval("bad argument");
    m->renorm_every = every;
    return QED_OK;
}

qed_status qed_autotune(qed_model *m, int32_t steps, char *choice, int32_t choice_cap, qed_stream stream) {
    if (!m || steps <= 0) return einval("qed_autotune: NULL model or steps <= 0");
    NvtxRange range("qed_autotune");
    std::string c = "FP64 model: no tile choices";
    if (m->prec != QED_FP64) {
        // the captured step graphs hold the old step tables
        QED_CUDA_TRY(cudaDeviceSynchronize());
        for (auto &g : m->graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        QED_TRY(split_autotune(m, (cudaStream_t)stream, steps, c));
        QED_TRY(qed_sync_status(m, stream));
    }
    if (choice && choice_cap > 0) {
        std::strncpy(choice, c.c_str(), (size_t)choice_cap - 1);
        choice[choice_cap - 1] = 0;
    }
    return QED_OK;
}

qed_status qed_set_plan(qed_model *m, int32_t gemm1_bn, int32_t gemm1_splits, int32_t gemm2_bn, int32_t gemm2_splits,
                        qed_stream stream) {
    if (!m) return einval("qed_set_plan: NULL model");
    if (m->prec == QED_FP64) {
        set_error("qed_set_plan: FP64 models have no tile plan");
        return QED_EUNSUPPORTED;
    }
    // the captured step graphs hold the old step tables
    QED_CUDA_TRY(cudaDeviceSynchronize());
    for (auto &g : m->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return split_set_plan(m, gemm1_bn, gemm1_splits, gemm2_bn, gemm2_splits, (cudaStream_t)stream);
}

qed_status qed_autotune_batched(int32_t n, qed_model *const *ms, int32_t steps, char *choice, int32_t choice_cap,
                                qed_stream stream) {
    if (n <= 0 || !ms || steps <= 0) return einval("qed_autotune_batched: need n > 0 models and steps > 0");
    for (int32_t i = 0; i < n; ++i) {
        if (!ms[i]) return einval("qed_autotune_batched: NULL model");
        if (ms[i]->prec == QED_FP64) return einval("qed_autotune_batched: FP64 instances have no grouped launches");
        for (int32_t j = 0; j < i; ++j)
            if (ms[j] == ms[i]) return einval("qed_autotune_batched: a model appears twice");
    }
    NvtxRange range("qed_autotune_batched");
    std::string c;
    QED_TRY(split_autotune_batched(ms, n, (cudaStream_t)stream, steps, c));
    for (int32_t i = 0; i < n; ++i) QED_TRY(qed_sync_status(ms[i], stream));
    if (choice && choice_cap > 0) {
        std::strncpy(choice, c.c_str(), (size_t)choice_cap - 1);
        choice[choice_cap - 1] = 0;
    }
    return QED_OK;
}

qed_status qed_set_wait_gate(qed_model *m, int32_t closed, int64_t budget_cycles, qed_stream stream) {
    if (!m || budget_cycles < 0) return einval("qed_set_wait_gate: NULL model or negative budget");
    if (m->prec == QED_FP64) {
        set_error("qed_set_wait_gate: the FP64 path has no bounded waits");
        return QED_EUNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t one = 1u;
    QED_CUDA_TRY(cudaMemcpyAsync(m->gate, &one, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    m->gate_armed = closed != 0;
    m->gate_budget = budget_cycles;
    // the captured step graphs hold the old kernel parameters
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    for (auto &g : m->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return split_rebuild(m, s);
}

qed_status qed_set_alloc_budget(int64_t bytes) {
    g_alloc_budget.store(bytes < 0 ? -1 : bytes);
    return QED_OK;
}

qed_status qed_set_scheme(qed_model *m, int32_t scheme) {
    if (!m || (scheme != QED_SCHEME_LIE && scheme != QED_SCHEME_STRANG && scheme != QED_SCHEME_EFFECTIVE))
        return einval("bad scheme");
    if (scheme == m->scheme) return QED_OK;
    if (scheme == QED_SCHEME_STRANG && m->prec == QED_FP64 && !m->work3)
        QED_TRY(dev_alloc(&m->work3, (size_t)(m->D * m->D)));
    if (scheme == QED_SCHEME_EFFECTIVE && !m->anti_zero) {
        QED_TRY(dev_alloc(&m->anti_zero, (size_t)m->D));
        QED_CUDA_TRY(cudaMemset(m->anti_zero, 0, (size_t)m->D * sizeof(double)));
    }
    // the captured step graphs belong to the old scheme
    QED_CUDA_TRY(cudaDeviceSynchronize());
    for (auto &g : m->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    const bool new_u = (scheme == QED_SCHEME_EFFECTIVE) != (m->scheme == QED_SCHEME_EFFECTIVE);
    m->scheme = scheme;
    if (new_u) {
        // the effective step has its own propagator, phases and (no) damping table
        QED_TRY(compute_propagator(m, scheme, nullptr));
        if (m->prec != QED_FP64) QED_TRY(split_prepare(m, nullptr));
    }
    split_set_scheme(m, scheme);
    QED_CUDA_TRY(cudaDeviceSynchronize());
    return QED_OK;
}

qed_status qed_evolve(qed_model *m, void *rho_v, int64_t n_steps, int64_t step_offset, int32_t record_every,
                      int32_t n_obs, const int32_t *obs_ids, double *records, qed_stream stream) {
    if (!m || !rho_v) return einval("NULL model or rho");
    if (n_steps < 0 || step_offset < 0) return einval("negative step count");
    if (n_obs < 0) return einval("negative n_obs");
    if (n_obs > 0 && (record_every <= 0 || !records)) return einval("records need record_every > 0 and a buffer");
    NvtxRange range("qed_evolve");
    cudaStream_t s = (cudaStream_t)stream;
    QED_TRY(ensure_ids(m, n_obs, obs_ids, s));
    double2 *rho = (double2 *)rho_v;
    const int64_t D = m->D;
    const bool split = m->prec != QED_FP64;
    if (split) {
        split_check_density(m, rho, s);
        QED_TRY(split_begin(m, rho, s));
    } else {
        if (!m->rho_int) QED_TRY(dev_alloc(&m->rho_int, (size_t)(D * D)));
        QED_CUDA_TRY(cudaMemcpyAsync(m->rho_int, rho, (size_t)(D * D) * 16, cudaMemcpyDeviceToDevice, s));
    }
    QED_TRY(ensure_graphs(m));
    const bool renorm = split && m->renorm_every > 0;
    int64_t row = 0;
    auto record = [&](int64_t p) {
        if (n_obs > 0 && (step_offset + p) % record_every == 0) {
            if (split)
                split_observables(m, m->obs_ids_dev, n_obs, records + row * n_obs, s);
            else
                observables(s, D, m->rho_int, m->obs_w, m->obs_ids_dev, n_obs, records + row * n_obs);
            ++row;
        }
    };
    record(0);
    for (int64_t i = 0; i < n_steps;) {
        int64_t p = n_steps;
        if (n_obs > 0) p = std::min(p, next_multiple_after(step_offset, i, record_every));
        if (renorm) p = std::min(p, next_multiple_after(step_offset, i, m->renorm_every));
        QED_TRY(run_steps(m, p - i, s));
        i = p;
        if (renorm && (step_offset + p) % m->renorm_every == 0) split_renorm(m, s);
        record(p);
    }
    if (split)
        split_end(m, rho, s);
    else
        QED_CUDA_TRY(cudaMemcpyAsync(rho, m->rho_int, (size_t)(D * D) * 16, cudaMemcpyDeviceToDevice, s));
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}

qed_status qed_evolve_batched(int32_t n, qed_model *const *ms, void *const *rhos, int64_t n_steps,
                              int32_t record_every, double *const *records, qed_stream stream) {
    if (n <= 0 || !ms || !rhos) return einval("qed_evolve_batched: need n > 0 models and rho pointers");
    if (n_steps < 0) return einval("qed_evolve_batched: negative step count");
    if (records && record_every <= 0) return einval("qed_evolve_batched: records need record_every > 0");
    NvtxRange range("qed_evolve_batched");
    cudaStream_t s = (cudaStream_t)stream;
    const bool split = ms[0] && ms[0]->prec != QED_FP64;
    for (int32_t i = 0; i < n; ++i) {
        if (!ms[i] || !rhos[i]) return einval("qed_evolve_batched: NULL model or rho");
        if ((ms[i]->prec != QED_FP64) != split) return einval("qed_evolve_batched: mixed precisions in one batch");
        for (int32_t j = 0; j < i; ++j)
            if (ms[j] == ms[i]) return einval("qed_evolve_batched: a model appears twice");
    }
    if (!split) {
        // FP64 instances run one after another (each with its own step graphs)
        for (int32_t i = 0; i < n; ++i) {
            qed_model *m = ms[i];
            std::vector<int32_t> ids;
            if (records && records[i])
                for (int64_t k = 0; k < m->D; ++k) ids.push_back((int32_t)k);
            QED_TRY(qed_evolve(m, rhos[i], n_steps, 0, record_every, (int32_t)ids.size(), ids.data(),
                               records ? records[i] : nullptr, stream));
        }
        return QED_OK;
    }
    for (int32_t i = 0; i < n; ++i) {
        split_check_density(ms[i], (const double2 *)rhos[i], s);
        QED_TRY(split_begin(ms[i], (const double2 *)rhos[i], s));
    }
    Batch *b = nullptr;
    QED_TRY(split_batch_create(ms, n, &b));
    // the step loop as graphs of 1 and kGraphSteps grouped steps
    cudaStream_t cap = nullptr;
    cudaGraphExec_t g[2] = {nullptr, nullptr};
    int64_t gk[2] = {0, 0};
    bool graphs = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
    const int64_t counts[2] = {1, kGraphSteps};
    for (int q = 0; q < 2 && graphs; ++q) {
        const int64_t before = launches();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { graphs = false; break; }
        for (int64_t k = 0; k < counts[q]; ++k) split_batch_step(b, ms[0]->err, cap);
        const cudaError_t e = cudaStreamEndCapture(cap, &graph);
        gk[q] = launches() - before;
        count_launches(-gk[q]);
        if (e != cudaSuccess || !graph || cudaGraphInstantiate(&g[q], graph, 0) != cudaSuccess) graphs = false;
        if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    auto run = [&](int64_t k) -> qed_status {
        if (!graphs) {
            for (; k > 0; --k) split_batch_step(b, ms[0]->err, s);
            return QED_OK;
        }
        for (; k >= kGraphSteps; k -= kGraphSteps) {
            QED_CUDA_TRY(cudaGraphLaunch(g[1], s));
            count_launches(gk[1]);
        }
        for (; k > 0; --k) {
            QED_CUDA_TRY(cudaGraphLaunch(g[0], s));
            count_launches(gk[0]);
        }
        return QED_OK;
    };
    int64_t row = 0;
    auto record = [&](int64_t p) {
        if (records && p % record_every == 0) {
            for (int32_t i = 0; i < n; ++i)
                if (records[i]) split_populations(ms[i], records[i] + row * ms[i]->D, s);
            ++row;
        }
    };
    qed_status st = QED_OK;
    record(0);
    for (int64_t i = 0; i < n_steps && st == QED_OK;) {
        int64_t p = n_steps;
        if (records) p = std::min(p, next_multiple_after(0, i, record_every));
        for (int32_t q = 0; q < n; ++q)
            if (ms[q]->renorm_every > 0) p = std::min(p, next_multiple_after(0, i, ms[q]->renorm_every));
        st = run(p - i);
        i = p;
        for (int32_t q = 0; q < n; ++q)
            if (ms[q]->renorm_every > 0 && p % ms[q]->renorm_every == 0) split_renorm(ms[q], s);
        record(p);
    }
    for (int32_t i = 0; i < n; ++i) split_end(ms[i], (double2 *)rhos[i], s);
    // the graphs and the batch tables are released once this call's work has finished
    cudaStreamSynchronize(s);
    for (auto &x : g)
        if (x) cudaGraphExecDestroy(x);
    if (cap) cudaStreamDestroy(cap);
    split_batch_destroy(b);
    if (st != QED_OK) return st;
    QED_CUDA_TRY(cudaGetLastError());
    // the call has synchronised: report device-side errors (a rejected rho, a bounded wait
    // that ran out) of every instance now
    for (int32_t i = 0; i < n; ++i) QED_TRY(qed_sync_status(ms[i], stream));
    return QED_OK;
}

qed_status qed_observables(const qed_model *m_c, const void *rho, int32_t n_obs, const int32_t *obs_ids, double *out,
                           qed_stream stream) {
    qed_model *m = const_cast<qed_model *>(m_c);
    if (!m || !rho || !out) return einval("NULL argument");
    if (n_obs <= 0) return einval("n_obs must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    QED_TRY(ensure_ids(m, n_obs, obs_ids, s));
    observables(s, m->D, (const double2 *)rho, m->obs_w, m->obs_ids_dev, n_obs, out);
    QED_CUDA_TRY(cudaGetLastError());
    return QED_OK;
}

qed_status qed_sync_status(qed_model *m, qed_stream stream) {
    if (!m) return einval("NULL model");
    cudaStream_t s = (cudaStream_t)stream;
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    QED_CUDA_TRY(cudaGetLastError());
    QED_CUDA_TRY(cudaMemcpy(m->err_host, m->err, 4, cudaMemcpyDeviceToHost));
    uint32_t e = *m->err_host;
    QED_CUDA_TRY(cudaMemset(m->err, 0, 4));
    if (e & kErrTimeout) { set_error("a bounded device wait ran out"); return QED_ETIMEOUT; }
    if (e & kErrNonFinite) { set_error("non-finite or non-positive trace at renormalisation"); return QED_ENUMERIC; }
    if (e & kErrSingular) { set_error("singular matrix"); return QED_ENUMERIC; }
    if (e & kErrBounds) {
        set_error("a device bounds check failed (QED_CHECKS build): an index read from a table was out of range");
        return QED_ECUDA;
    }
    if (e & kErrNotDensity) {
        set_error("split precision needs a Hermitian rho of unit trace (|rho_mn - conj(rho_nm)| <= 1e-8, "
                  "|tr rho - 1| <= 1e-6); that rho was evolved regardless and the result is not meaningful");
        return QED_EINVAL;
    }
    return QED_OK;
}

qed_status qed_set_U(qed_model *m, const void *U, qed_stream stream) {
    if (!m || !U) return einval("NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    QED_CUDA_TRY(cudaMemcpyAsync(m->U, U, (size_t)(m->D * m->D) * 16, cudaMemcpyDeviceToDevice, s));
    if (m->prec != QED_FP64) QED_TRY(split_prepare(m, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    return QED_OK;
}

qed_status qed_get_U(const qed_model *m, void *U, qed_stream stream) {
    if (!m || !U) return einval("NULL argument");
    QED_CUDA_TRY(cudaMemcpyAsync(U, m->U, (size_t)(m->D * m->D) * 16, cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
    return QED_OK;
}

qed_status qed_select_states(qed_model *m, const void *rho0, int64_t steps_per_round, int32_t n_rounds, double eps,
                             qed_model **out_model, void *rho_out, int64_t *keep, int64_t *n_keep, int64_t *sizes,
                             qed_stream stream) {
    if (!m || !rho0 || !out_model || !rho_out || !keep || !n_keep) return einval("NULL argument");
    if (steps_per_round <= 0 || n_rounds <= 0 || !(eps >= 0.0)) return einval("bad selection parameters");
    NvtxRange range("qed_select_states");
    *out_model = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    using Owned = std::unique_ptr<qed_model, void (*)(qed_model *)>;
    Owned owned(nullptr, release);  // the current reduced model, once one exists
    qed_model *cur = m;
    const int64_t D0 = m->D;
    double2 *rho = nullptr, *rho_next = nullptr;
    double *p0 = nullptr, *p1 = nullptr;
    int32_t *flag = nullptr;
    int64_t *idx = nullptr;
    struct Free {
        std::vector<void *> p;
        ~Free() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } guard;
    QED_TRY(dev_alloc(&rho, (size_t)(D0 * D0)));
    guard.p.push_back(rho);
    QED_TRY(dev_alloc(&rho_next, (size_t)(D0 * D0)));
    guard.p.push_back(rho_next);
    QED_TRY(dev_alloc(&p0, (size_t)D0));
    guard.p.push_back(p0);
    QED_TRY(dev_alloc(&p1, (size_t)D0));
    guard.p.push_back(p1);
    QED_TRY(dev_alloc(&flag, (size_t)D0));
    guard.p.push_back(flag);
    QED_TRY(dev_alloc(&idx, (size_t)D0));
    guard.p.push_back(idx);
    QED_CUDA_TRY(cudaMemcpyAsync(rho, rho0, (size_t)(D0 * D0) * 16, cudaMemcpyDeviceToDevice, s));
    std::vector<int64_t> global((size_t)D0);
    for (int64_t k = 0; k < D0; ++k) global[(size_t)k] = k;
    std::vector<int32_t> hflag((size_t)D0);
    const double inv_T = 1.0 / ((double)steps_per_round * m->dt);
    for (int32_t r = 0; r < n_rounds; ++r) {
        const int64_t D = cur->D;
        // solve, then the growth speed of every probability over the round
        diag_f64(s, D, rho, p0);
        QED_TRY(qed_evolve(cur, rho, steps_per_round, 0, 0, 0, nullptr, nullptr, stream));
        QED_TRY(qed_sync_status(cur, stream));
        diag_f64(s, D, rho, p1);
        select_states_flags(s, D, p0, p1, inv_T, eps, flag);
        QED_CUDA_TRY(cudaMemcpyAsync(hflag.data(), flag, (size_t)D * 4, cudaMemcpyDeviceToHost, s));
        QED_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<int64_t> local;
        for (int64_t k = 0; k < D; ++k)
            if (hflag[(size_t)k]) local.push_back(k);
        if (local.empty()) {
            set_error("qed_select_states: every state fell below eps");
            return QED_ENUMERIC;
        }
        const int64_t n = (int64_t)local.size();
        if (sizes) sizes[r] = n;
        if (n < D || (r == n_rounds - 1 && !owned)) {
            // the remaining states: rho restricted to them, and the model on them (P H P, P A_j P)
            QED_CUDA_TRY(cudaMemcpyAsync(idx, local.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
            gather_submatrix(s, D, rho, n, idx, rho_next);
            std::swap(rho, rho_next);
            Owned next(new qed_model(), release);
            std::string err;
            if (!restrict_host_model(cur->host, local, next->host, err)) return einval(err);
            QED_TRY(build_device(next.get(), cur->dt, cur->prec, s));
            next->renorm_every = cur->renorm_every;
            if (cur->scheme != QED_SCHEME_LIE) QED_TRY(qed_set_scheme(next.get(), cur->scheme));
            std::vector<int64_t> g2((size_t)n);
            for (int64_t a = 0; a < n; ++a) g2[(size_t)a] = global[(size_t)local[(size_t)a]];
            global.swap(g2);
            owned = std::move(next);
            cur = owned.get();
        }
        // normalise (and symmetrise) the density matrix of the remaining states
        renormalise(s, n, rho, cur->scalars, cur->err);
        QED_TRY(qed_sync_status(cur, stream));
    }
    const int64_t n = cur->D;
    QED_CUDA_TRY(cudaMemcpyAsync(rho_out, rho, (size_t)(n * n) * 16, cudaMemcpyDeviceToDevice, s));
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    std::copy(global.begin(), global.end(), keep);
    *n_keep = n;
    *out_model = owned.release();
    return QED_OK;
}

qed_status qed_profile_replay(qed_model *m, void *rho_v, int32_t reps, double *ms, int32_t n_kernels, char *names,
                              int32_t name_cap, qed_stream stream) {
    if (!m || !rho_v || !ms || reps <= 0) return einval("bad argument");
    if (m->prec == QED_FP64) {
        set_error("qed_profile_replay: split-precision models only");
        return QED_EUNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    QED_TRY(split_begin(m, (const double2 *)rho_v, s));
    std::vector<double> acc;
    std::string label;
    QED_TRY(split_profile_replay(m, s, reps, acc, label));
    for (int c = 0; c < n_kernels; ++c) ms[c] = c < (int)acc.size() ? acc[(size_t)c] : 0.0;
    if (names && name_cap > 0) {
        std::strncpy(names, label.c_str(), (size_t)name_cap - 1);
        names[name_cap - 1] = 0;
    }
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    return QED_OK;
}

qed_status qed_profile(qed_model *m, void *rho_v, int64_t n_steps, double *ms, int32_t n_kernels, char *names,
                       int32_t name_cap, qed_stream stream) {
    if (!m || !rho_v || !ms || n_steps <= 0) return einval("bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    double2 *rho = (double2 *)rho_v;
    std::vector<double> acc(8, 0.0);
    std::string label;
    int classes = 0;
    if (m->prec != QED_FP64) QED_TRY(split_begin(m, rho, s));
    for (int64_t i = 0; i < n_steps; ++i) {
        if (m->prec == QED_FP64) {
            classes = step_f64(m, rho, s, m->ev, &label);
        } else {
            classes = split_step_timed(m, s, label);
        }
        QED_CUDA_TRY(cudaEventSynchronize(m->ev[classes]));
        for (int c = 0; c < classes; ++c) {
            float t = 0.f;
            cudaEventElapsedTime(&t, m->ev[c], m->ev[c + 1]);
            acc[(size_t)c] += t;
        }
    }
    if (m->prec != QED_FP64) split_end(m, rho, s);
    for (int c = 0; c < n_kernels; ++c) ms[c] = c < classes ? acc[(size_t)c] / (double)n_steps : 0.0;
    if (names && name_cap > 0) {
        std::strncpy(names, label.c_str(), (size_t)name_cap - 1);
        names[name_cap - 1] = 0;
    }
    QED_CUDA_TRY(cudaStreamSynchronize(s));
    return QED_OK;
}

}  // extern "C"
