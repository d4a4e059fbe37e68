// Launchers of the device kernels (all enqueue on the given stream, no synchronisation).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qed.h"

namespace qed {

// Number of kernels this library has launched (all launchers add to it).
void count_launches(int64_t n);
int64_t launches();

// C = alpha * A * op(B) + beta * C for complex128 row-major matrices; op(B) = B (conj_b
// false, B is K x N) or B^+ (conj_b true, B is N x K).  FP64 FMA, 32 x 32 tiles.
void zgemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha, const double2 *A,
           int64_t lda, const double2 *B, int64_t ldb, bool conj_b, double beta, double2 *C,
           int64_t ldc);

// C = alpha * op(A) * op(B) + beta * C with op(A) = A (M x K) or A^+ (A is K x M).
void zgemm_ex(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha, const double2 *A, int64_t lda,
              bool conj_a, const double2 *B, int64_t ldb, bool conj_b, double beta, double2 *C, int64_t ldc);

// Y = c0 A + c1 B + c2 C + c3 I + c4 Y (real coefficients; any of A, B, C may be null).
void zlincomb(cudaStream_t s, int64_t D, double c0, const double2 *A, double c1, const double2 *B,
              double c2, const double2 *C, double c3, double c4, double2 *Y);

// X = -i * theta * H
void scale_minus_i(cudaStream_t s, int64_t D, double theta, const double2 *H, double2 *X);

// aug (D x 2D) = [V - U | V + U]
void pade_augment(cudaStream_t s, int64_t D, const double2 *Up, const double2 *Vp, double2 *aug);

// Gauss-Jordan elimination with partial pivoting on aug = [Q | P]; afterwards the right
// half holds Q^-1 P.  Sets kErrSingular in *err if a pivot is exactly zero.
void gauss_jordan(cudaStream_t s, int64_t D, double2 *aug, uint32_t *err);

// The same on a D x W matrix [Q | B_1 | B_2 | ...]: afterwards columns D.. hold Q^-1 B_i.
void gauss_jordan_w(cudaStream_t s, int64_t D, int64_t W, double2 *aug, uint32_t *err);

// aug (D x 4D) = [V - U | V + U | dV + dU | dV - dU]
void frechet_augment(cudaStream_t s, int64_t D, const double2 *Up, const double2 *Vp, const double2 *dUp,
                     const double2 *dVp, double2 *aug);

// out (D x D) = columns [c0, c0 + D) of the D x W matrix aug
void take_block(cudaStream_t s, int64_t D, int64_t W, int64_t c0, const double2 *aug, double2 *out);

// Copy the right half of aug (D x 2D) into R (D x D).
void take_right_half(cudaStream_t s, int64_t D, const double2 *aug, double2 *R);

// rho = V (1 - dt/2 (d_m + d_n)) + dt sum_j c_j(m) c_j(n) V[src_j(m), src_j(n)]
void dissipate_f64(cudaStream_t s, int64_t D, const double2 *V, double2 *rho, const double *anti,
                   const int32_t *in_ptr, const int32_t *in_jump, const int32_t *in_src,
                   const double *in_coef, double dt);

// out = B + tau [ -(d_m + d_n)/2 X_mn + sum_j c_j(m) c_j(n) X[src_j(m), src_j(n)] ] (out may be
// B, not X): a stage of the explicit midpoint rule for the Lindblad term.
void lindblad_axpy_f64(cudaStream_t s, int64_t D, const double2 *X, const double2 *B, double2 *out,
                       const double *anti, const int32_t *in_ptr, const int32_t *in_jump, const int32_t *in_src,
                       const double *in_coef, double tau);

// State space selection (Sec. 3.2): p = Re diag(rho); keep[k] = (|p1 - p0|_k / T >= eps or
// p1_k >= eps); out = rho[idx][:, idx] (n x n).
void diag_f64(cudaStream_t s, int64_t D, const double2 *rho, double *p);
void select_states_flags(cudaStream_t s, int64_t D, const double *p0, const double *p1, double inv_T, double eps,
                         int32_t *keep);
void gather_submatrix(cudaStream_t s, int64_t D, const double2 *rho, int64_t n, const int64_t *idx, double2 *out);

// out[o] = rho_kk (id < D), or sum_k w[id-D][k] rho_kk; deterministic block reduction.
void observables(cudaStream_t s, int64_t D, const double2 *rho, const double *weights,
                 const int32_t *ids, int32_t n_obs, double *out);

// U = exp(-i dt H) (H Hermitian, device) and R = exp(X) (general X with 1-norm xnorm):
// Pade-13 scaling and squaring; allocate their own work space; synchronise `s`.
qed_status propagator(cudaStream_t s, int64_t D, double dt, const double2 *H, double h_norm1, double2 *U,
                      uint32_t *err);
qed_status expm_pade13(cudaStream_t s, int64_t D, const double2 *X, double xnorm, double2 *R, uint32_t *err);
// R = exp(X) and L = L_exp(X, E), the Frechet derivative of exp at X in the direction E
// (general complex X with 1-norm xnorm, any E); same Pade-13 scaling and squaring.
qed_status expm_frechet_pade13(cudaStream_t s, int64_t D, const double2 *X, const double2 *E, double xnorm,
                               double2 *R, double2 *L, uint32_t *err);

// rho <- (rho + rho^+) / (2 tr rho); flags non-finite traces in *err.
void renormalise(cudaStream_t s, int64_t D, double2 *rho, double *scratch, uint32_t *err);

}  // namespace qed
