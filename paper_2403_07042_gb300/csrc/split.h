// Split-precision (increment form) step: U = P (I + Delta) with P = diag(exp(-i H_kk dt)),
// so U rho U^+ = P (rho + W + W^+ + X) P^+ with W = Delta rho and X = W Delta^+; the two
// products run on the tensor cores with FP16 pieces and FP32 accumulation, and the
// master rho is kept as a double-float (two FP32 words) inside the library.
#pragma once

#include <string>

#include "model.h"

namespace qed {

qed_status split_prepare(qed_model *m, cudaStream_t s);                 // Delta planes, buffers, TMA maps
qed_status split_begin(qed_model *m, const double2 *rho, cudaStream_t s);  // caller rho -> internal state
// Sets kErrNotDensity in m->err unless rho (caller layout) is Hermitian with unit trace
// within kDensityHermTol / kDensityTraceTol: the increment form relies on both.
void split_check_density(qed_model *m, const double2 *rho, cudaStream_t s);
void split_step(qed_model *m, cudaStream_t s);
void split_set_scheme(qed_model *m, int scheme);  // QED_SCHEME_LIE or QED_SCHEME_STRANG
// Rebuilds the model's step tables (after a change of its wait-gate hook); synchronises `s`.
qed_status split_rebuild(qed_model *m, cudaStream_t s);
// Times whole steps over the tile widths and split-K factors of both products and keeps
// the fastest; `choice` describes it.
qed_status split_autotune(qed_model *m, cudaStream_t s, int steps, std::string &choice);
void split_renorm(qed_model *m, cudaStream_t s);
void split_observables(qed_model *m, const int32_t *ids, int32_t n_obs, double *out, cudaStream_t s);
void split_end(qed_model *m, double2 *rho, cudaStream_t s);              // internal state -> caller rho
int split_step_timed(qed_model *m, cudaStream_t s, std::string &label);
void split_populations(qed_model *m, double *out, cudaStream_t s);      // out[k] = rho_kk

// Access for the adjoint: the double-float state and V buffer (D x D float4), the Lindblad
// pass alone (V buffer -> state + planes), the planes recomputed from the state.
float4 *split_state(qed_model *m);
float4 *split_vbuf(qed_model *m);
void split_dissipate_only(qed_model *m, cudaStream_t s);
// The pieces of a step, for the adjoint of the Strang step: one Lindblad stage
// out = B + f dt L(X) on the model's buffers (0 state, 1 V buffer, 2 stage buffer; planes:
// also write the state's FP16 planes), out = dt L(X) for any double-float D x D buffer X,
// the two products V = U X U^+ of the state X (planes already written), the stage buffer.
void split_lindblad_stage(qed_model *m, int xsel, int bsel, int osel, float f, int planes, cudaStream_t s);
void split_apply_lindblad(qed_model *m, const float4 *X, float4 *out, cudaStream_t s);
void split_products(qed_model *m, cudaStream_t s);
float4 *split_ybuf(qed_model *m);
void split_refresh_planes(qed_model *m, cudaStream_t s);

// Many split-precision models stepped together: one grouped launch per phase.
struct Batch;
qed_status split_batch_create(qed_model *const *ms, int n, Batch **out);
void split_batch_step(const Batch *b, uint32_t *err, cudaStream_t s);
void split_batch_destroy(Batch *b);
// Times the grouped launches' tile widths on whole batched steps; keeps the fastest in the
// models (used by the next split_batch_create of models that all carry it).
qed_status split_autotune_batched(qed_model *const *ms, int n, cudaStream_t s, int steps, std::string &choice);
// Sets the tile plan of the model's products (what the tuners choose) and rebuilds its step
// tables; the grouped launches take the two widths.
qed_status split_set_plan(qed_model *m, int bn1, int splits1, int bn2, int splits2, cudaStream_t s);
// Per-kernel durations of the Lie step with each kernel replayed back to back from a graph.
qed_status split_profile_replay(qed_model *m, cudaStream_t s, int reps, std::vector<double> &ms, std::string &label);
void split_release(qed_model *m);

}  // namespace qed
