// Device-resident model: operators, propagator, work space and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "builder.h"
#include "qed.h"

struct qed_model;

namespace qed {

// A named range on the host timeline (NVTX) around a phase of the library's work: shown by
// timeline profilers, a no-op unless one is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

void set_error(const std::string &msg);

// Every device allocation of the library goes through here (cudaMalloc), so that the
// allocation-failure hook (qed_set_alloc_budget) can make it fail like an exhausted device.
cudaError_t device_malloc(void **p, size_t bytes);

#define QED_CUDA_TRY(call)                                                        \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            ::qed::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return QED_ECUDA;                                                     \
        }                                                                         \
    } while (0)

// Device error word bits (written by kernels, read by qed_sync_status).
enum : uint32_t {
    kErrNonFinite = 1u,
    kErrSingular = 2u,
    kErrTimeout = 4u,
    kErrNotDensity = 8u,   // split precision given a rho that is not Hermitian with unit trace
    kErrBounds = 16u,      // a device bounds check of the QED_CHECKS build failed
};

// Tolerances of that check (absolute): max |rho_mn - conj(rho_nm)| and |tr rho - 1|.
constexpr double kDensityHermTol = 1e-8;
constexpr double kDensityTraceTol = 1e-6;

// State of the split-precision (increment form) path; defined in split.cu.
struct SplitState;
// Tables of the adjoint (gradients); defined in adjoint.cu.
struct AdjointState;
void adjoint_release(qed_model *m);

}  // namespace qed

struct qed_model {
    qed::HostModel host;
    int64_t D = 0;
    double dt = 0.0;
    qed_precision prec = QED_FP64;
    int32_t renorm_every = 100;
    int32_t scheme = QED_SCHEME_LIE;

    // device operators (FP64, complex interleaved)
    double2 *U = nullptr;        // D x D
    double2 *work1 = nullptr;    // D x D
    double2 *work2 = nullptr;    // D x D
    double2 *work3 = nullptr;    // D x D stage buffer of the Strang step (FP64 path, on demand)
    double2 *phase = nullptr;    // D: P_k = exp(-i H_kk dt)
    double *anti = nullptr;      // D: d_k = sum_j gamma_j (A_j^+A_j)_kk
    double *anti_zero = nullptr; // D zeros: the damping table of the effective-Hamiltonian step
    // incoming jump lists per row m, sorted by jump id: entries [in_ptr[m], in_ptr[m+1])
    int32_t *in_ptr = nullptr;   // D + 1
    int32_t *in_jump = nullptr;
    int32_t *in_src = nullptr;
    double *in_coef = nullptr;   // coefficient * sqrt(gamma_j)
    int64_t n_in = 0;
    int32_t max_in = 0;
    // observables: named weights [n_named x D]
    double *obs_w = nullptr;
    int32_t n_named = 0;
    int32_t *obs_ids_dev = nullptr;   // scratch for the ids of one call
    int32_t obs_ids_cap = 0;
    double *scalars = nullptr;        // device scratch: trace etc.
    uint32_t *err = nullptr;          // device error word
    uint32_t *err_host = nullptr;     // pinned mirror
    // wait-gate test hook (qed_set_wait_gate): while armed, the split step's tensor-core
    // kernels wait up to gate_budget cycles for *gate to become 0, which nothing does
    uint32_t *gate = nullptr;
    bool gate_armed = false;
    int64_t gate_budget = 0;

    qed::SplitState *sp = nullptr;
    qed::AdjointState *adj = nullptr;
    cudaEvent_t ev[16] = {};

    // step loop as CUDA graphs: graph[0] runs 1 step, graph[1] runs kGraphSteps steps
    double2 *rho_int = nullptr;       // FP64 path: the state the graphs step in place
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
    bool graphs_off = false;          // set if capture is unavailable (direct launches)
};
