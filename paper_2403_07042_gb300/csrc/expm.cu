// The propagator stage ("Taylor approximation" in Sec. 4.2, Table 3): U = exp(X) in FP64
// by scaling and squaring with the degree-13 Pade approximant (Higham, SIAM J. Matrix
// Anal. Appl. 26(4), 2005), the linear solve by Gauss-Jordan elimination on the device.
#include <cmath>
#include <string>

#include "kernels.h"
#include "model.h"

namespace qed {

namespace {

qed_status alloc_work(double2 **p, size_t count) {
    if (cudaMalloc((void **)p, count * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed for the propagator work space");
        return QED_ENOMEM;
    }
    return QED_OK;
}

}  // namespace

// Pade-13 coefficients b_j = (2m-j)! m! / ((2m)! j! (m-j)!), m = 13, scaled so b_13 = 1
// (Higham, SIAM J. Matrix Anal. Appl. 26(4), 2005): b_j = (26-j)! / (j! (13-j)!).
void pade13_coefficients(double b[14]) {
    for (int j = 0; j <= 13; ++j) {
        long double v = 1.0L;
        for (int q = 14 - j; q <= 26 - j; ++q) v *= q;  // (26-j)! / (13-j)!
        for (int q = 2; q <= j; ++q) v /= q;            // / j!
        b[j] = (double)v;
    }
}

// theta_13 of the Pade-13 scaling-and-squaring method (Higham 2005, Table 2.3): the
// largest 1-norm of X for which the degree-13 approximant is accurate to unit roundoff.
constexpr double kTheta13 = 5.371920351148152;

// R = exp(X0) for a general complex X0 (device, D x D) with 1-norm xnorm.  Allocates
// and frees its own work space; synchronises `s`.
qed_status expm_pade13(cudaStream_t s, int64_t D, const double2 *X0, double xnorm, double2 *U, uint32_t *err) {
    double b[14];
    pade13_coefficients(b);
    int sq = 0;
    if (xnorm > kTheta13) sq = (int)std::ceil(std::log2(xnorm / kTheta13));
    const size_t DD = (size_t)(D * D);
    double2 *buf = nullptr;
    qed_status st = alloc_work(&buf, DD * 9);
    if (st != QED_OK) return st;
    double2 *X = buf, *X2 = buf + DD, *X4 = buf + 2 * DD, *X6 = buf + 3 * DD, *T = buf + 4 * DD,
            *Up = buf + 5 * DD, *Vp = buf + 6 * DD, *aug = buf + 7 * DD;  // aug takes 2 DD
    zlincomb(s, D, std::ldexp(1.0, -sq), X0, 0.0, nullptr, 0.0, nullptr, 0.0, 0.0, X);
    zgemm(s, D, D, D, 1.0, X, D, X, D, false, 0.0, X2, D);
    zgemm(s, D, D, D, 1.0, X2, D, X2, D, false, 0.0, X4, D);
    zgemm(s, D, D, D, 1.0, X4, D, X2, D, false, 0.0, X6, D);
    // U_p = X [X6 (b13 X6 + b11 X4 + b9 X2) + b7 X6 + b5 X4 + b3 X2 + b1 I]
    zlincomb(s, D, b[13], X6, b[11], X4, b[9], X2, 0.0, 0.0, T);
    zgemm(s, D, D, D, 1.0, X6, D, T, D, false, 0.0, Vp, D);
    zlincomb(s, D, b[7], X6, b[5], X4, b[3], X2, b[1], 1.0, Vp);
    zgemm(s, D, D, D, 1.0, X, D, Vp, D, false, 0.0, Up, D);
    // V_p = X6 (b12 X6 + b10 X4 + b8 X2) + b6 X6 + b4 X4 + b2 X2 + b0 I
    zlincomb(s, D, b[12], X6, b[10], X4, b[8], X2, 0.0, 0.0, T);
    zgemm(s, D, D, D, 1.0, X6, D, T, D, false, 0.0, Vp, D);
    zlincomb(s, D, b[6], X6, b[4], X4, b[2], X2, b[0], 1.0, Vp);
    // solve (V_p - U_p) R = V_p + U_p
    pade_augment(s, D, Up, Vp, aug);
    gauss_jordan(s, D, aug, err);
    take_right_half(s, D, aug, U);
    // undo the scaling: R^(2^sq)
    for (int q = 0; q < sq; ++q) {
        zgemm(s, D, D, D, 1.0, U, D, U, D, false, 0.0, T, D);
        cudaMemcpyAsync(U, T, DD * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_error(std::string("propagator: ") + cudaGetErrorString(e));
        return QED_ECUDA;
    }
    return QED_OK;
}


qed_status propagator(cudaStream_t s, int64_t D, double dt, const double2 *H, double h_norm1, double2 *U,
                      uint32_t *err) {
    double2 *X = nullptr;
    qed_status st = alloc_work(&X, (size_t)(D * D));
    if (st != QED_OK) return st;
    scale_minus_i(s, D, dt, H, X);
    st = expm_pade13(s, D, X, dt * h_norm1, U, err);
    cudaFree(X);
    return st;
}

}  // namespace qed
