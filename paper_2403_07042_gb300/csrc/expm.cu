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
    if (device_malloc((void **)p, count * sizeof(double2)) != cudaSuccess) {
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


// R = exp(X0) and L = L_exp(X0, E0).  Every step of the Pade-13 evaluation above is applied
// to the block upper-triangular matrix [[X, E], [0, X]], whose powers and polynomials keep
// the form [[p(X), dp], [0, p(X)]] with dp the directional derivative of p at X along E
// (Al-Mohy and Higham, SIAM J. Matrix Anal. Appl. 30(4), 2009): a product of two such blocks
// costs three D x D products instead of eight for the dense 2D x 2D matrix.  With
// r = Q^-1 P, dr = Q^-1 (dP - dQ r); squaring maps (R, L) to (R R, R L + L R).  The scaling
// depends on ||X|| alone, since L is linear in E.
qed_status expm_frechet_pade13(cudaStream_t s, int64_t D, const double2 *X0, const double2 *E0, double xnorm,
                               double2 *R, double2 *L, uint32_t *err) {
    double b[14];
    pade13_coefficients(b);
    int sq = 0;
    if (xnorm > kTheta13) sq = (int)std::ceil(std::log2(xnorm / kTheta13));
    const size_t DD = (size_t)(D * D);
    double2 *buf = nullptr;
    qed_status st = alloc_work(&buf, DD * 20);
    if (st != QED_OK) return st;
    double2 *X = buf, *E = buf + DD, *X2 = buf + 2 * DD, *M2 = buf + 3 * DD, *X4 = buf + 4 * DD,
            *M4 = buf + 5 * DD, *X6 = buf + 6 * DD, *M6 = buf + 7 * DD, *T1 = buf + 8 * DD, *T2 = buf + 9 * DD,
            *Up = buf + 10 * DD, *dUp = buf + 11 * DD, *Vp = buf + 12 * DD, *dVp = buf + 13 * DD,
            *W = buf + 14 * DD, *dW = buf + 15 * DD, *aug = buf + 16 * DD;  // aug takes 4 DD
    const double sc = std::ldexp(1.0, -sq);
    zlincomb(s, D, sc, X0, 0.0, nullptr, 0.0, nullptr, 0.0, 0.0, X);
    zlincomb(s, D, sc, E0, 0.0, nullptr, 0.0, nullptr, 0.0, 0.0, E);
    // powers: X2k and their derivatives M2k
    zgemm(s, D, D, D, 1.0, X, D, X, D, false, 0.0, X2, D);
    zgemm(s, D, D, D, 1.0, X, D, E, D, false, 0.0, M2, D);
    zgemm(s, D, D, D, 1.0, E, D, X, D, false, 1.0, M2, D);
    zgemm(s, D, D, D, 1.0, X2, D, X2, D, false, 0.0, X4, D);
    zgemm(s, D, D, D, 1.0, X2, D, M2, D, false, 0.0, M4, D);
    zgemm(s, D, D, D, 1.0, M2, D, X2, D, false, 1.0, M4, D);
    zgemm(s, D, D, D, 1.0, X4, D, X2, D, false, 0.0, X6, D);
    zgemm(s, D, D, D, 1.0, X4, D, M2, D, false, 0.0, M6, D);
    zgemm(s, D, D, D, 1.0, M4, D, X2, D, false, 1.0, M6, D);
    // odd part: W = X6 (b13 X6 + b11 X4 + b9 X2) + b7 X6 + b5 X4 + b3 X2 + b1 I, U = X W
    zlincomb(s, D, b[13], X6, b[11], X4, b[9], X2, 0.0, 0.0, T1);
    zlincomb(s, D, b[13], M6, b[11], M4, b[9], M2, 0.0, 0.0, T2);
    zgemm(s, D, D, D, 1.0, X6, D, T1, D, false, 0.0, W, D);
    zgemm(s, D, D, D, 1.0, X6, D, T2, D, false, 0.0, dW, D);
    zgemm(s, D, D, D, 1.0, M6, D, T1, D, false, 1.0, dW, D);
    zlincomb(s, D, b[7], X6, b[5], X4, b[3], X2, b[1], 1.0, W);
    zlincomb(s, D, b[7], M6, b[5], M4, b[3], M2, 0.0, 1.0, dW);
    zgemm(s, D, D, D, 1.0, X, D, W, D, false, 0.0, Up, D);
    zgemm(s, D, D, D, 1.0, X, D, dW, D, false, 0.0, dUp, D);
    zgemm(s, D, D, D, 1.0, E, D, W, D, false, 1.0, dUp, D);
    // even part: V = X6 (b12 X6 + b10 X4 + b8 X2) + b6 X6 + b4 X4 + b2 X2 + b0 I
    zlincomb(s, D, b[12], X6, b[10], X4, b[8], X2, 0.0, 0.0, T1);
    zlincomb(s, D, b[12], M6, b[10], M4, b[8], M2, 0.0, 0.0, T2);
    zgemm(s, D, D, D, 1.0, X6, D, T1, D, false, 0.0, Vp, D);
    zgemm(s, D, D, D, 1.0, X6, D, T2, D, false, 0.0, dVp, D);
    zgemm(s, D, D, D, 1.0, M6, D, T1, D, false, 1.0, dVp, D);
    zlincomb(s, D, b[6], X6, b[4], X4, b[2], X2, b[0], 1.0, Vp);
    zlincomb(s, D, b[6], M6, b[4], M4, b[2], M2, 0.0, 1.0, dVp);
    // Q = V - U, P = V + U: one elimination gives Q^-1 P, Q^-1 dP and Q^-1 dQ
    frechet_augment(s, D, Up, Vp, dUp, dVp, aug);
    gauss_jordan_w(s, D, 4 * D, aug, err);
    take_block(s, D, 4 * D, D, aug, R);
    take_block(s, D, 4 * D, 2 * D, aug, L);
    take_block(s, D, 4 * D, 3 * D, aug, T1);
    zgemm(s, D, D, D, -1.0, T1, D, R, D, false, 1.0, L, D);
    // undo the scaling
    for (int q = 0; q < sq; ++q) {
        zgemm(s, D, D, D, 1.0, R, D, L, D, false, 0.0, T1, D);
        zgemm(s, D, D, D, 1.0, L, D, R, D, false, 1.0, T1, D);
        zgemm(s, D, D, D, 1.0, R, D, R, D, false, 0.0, T2, D);
        cudaMemcpyAsync(L, T1, DD * sizeof(double2), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(R, T2, DD * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_error(std::string("expm_frechet_pade13: ") + cudaGetErrorString(e));
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
