// Split-precision (increment form) step: U = P (I + Delta) with P = diag(exp(-i H_kk dt)),
// so U rho U^+ = P (rho + W + W^+ + X) P^+ with W = Delta rho and X = W Delta^+; the two
// products run on the tensor cores with FP16 hi/lo operands and FP32 accumulation.
#pragma once

#include <string>

#include "model.h"

namespace qed {

qed_status split_prepare(qed_model *m, cudaStream_t s);      // Delta planes, buffers, TMA maps
qed_status split_begin(qed_model *m, double2 *rho, cudaStream_t s);  // rho -> FP16 planes
void split_step(qed_model *m, double2 *rho, cudaStream_t s);
void split_renorm(qed_model *m, double2 *rho, cudaStream_t s);
void split_sync_rho(qed_model *m, double2 *rho, cudaStream_t s);   // nothing pending after a step
int split_step_timed(qed_model *m, double2 *rho, cudaStream_t s, std::string &label);
void split_release(qed_model *m);

}  // namespace qed
