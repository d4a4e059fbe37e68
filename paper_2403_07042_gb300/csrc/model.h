// Device-resident model: operators, propagator, work space and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "builder.h"
#include "qed.h"

namespace qed {

void set_error(const std::string &msg);

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
};

// Operand planes of the split-precision (increment form) path.
struct SplitPlanes {
    int64_t Dp = 0;            // padded dimension (multiple of 128)
    // static operands, FP16 [2 (hi, lo)][2Dp][2Dp]
    void *a1 = nullptr;        // [[Dre, Dim], [Dim, -Dre]]      (GEMM1 A, rows k / k+Dp)
    void *b2 = nullptr;        // [[Dre, Dim], [-Dim, Dre]]      (GEMM2 B, rows l / l+Dp)
    // dynamic operands
    void *rho_pl = nullptr;    // FP16 [2][Dp][2Dp]   rows l: [rho_re | rho_im]
    void *w_pl = nullptr;      // FP16 [2][Dp][2Dp]   rows k: [W_re | W_im]
    float *w32 = nullptr;      // FP32 [2][Dp][Dp]    W = Delta rho (re plane, im plane)
    float *x32 = nullptr;      // FP32 [Dp][2Dp]      X = W Delta^+ (cols re | im)
    float *partial = nullptr;  // split-K partial sums
    int64_t partial_elems = 0;
    double scale_delta = 1.0;  // power-of-two scales applied before the FP16 split
    double scale_rho = 1.0;
    double scale_w = 1.0;
    void *tmaps = nullptr;     // device copy of the TMA descriptors (CUtensorMap[4])
    std::vector<unsigned char> tmap_host;
};

}  // namespace qed

struct qed_model {
    qed::HostModel host;
    int64_t D = 0;
    double dt = 0.0;
    qed_precision prec = QED_FP64;
    int32_t renorm_every = 100;

    // device operators (FP64, complex interleaved)
    double2 *U = nullptr;        // D x D
    double2 *work1 = nullptr;    // D x D
    double2 *work2 = nullptr;    // D x D
    double2 *phase = nullptr;    // D: P_k = exp(-i H_kk dt)
    double *anti = nullptr;      // D: d_k = sum_j gamma_j (A_j^+A_j)_kk
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

    qed::SplitPlanes sp;
    cudaEvent_t ev[16] = {};
};
