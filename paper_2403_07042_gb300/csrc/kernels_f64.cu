// FP64 kernels: complex GEMM, the Pade pieces of the propagator, the Lindblad update
// of Eq. (3) on a stored V, observables and renormalisation.
#include <atomic>

#include "kernels.h"
#include "model.h"

namespace qed {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

namespace {

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // c + a b
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}

constexpr int TM = 32, TN = 32, TK = 16;

// 64 threads; thread (ty, tx) in 8 x 8 owns rows ty + 8i and columns tx + 8j.
template <bool CONJ_A, bool CONJ_B>
__global__ void __launch_bounds__(64) zgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                   const double2 *__restrict__ A, int64_t lda,
                                                   const double2 *__restrict__ B, int64_t ldb,
                                                   double beta, double2 *__restrict__ C, int64_t ldc) {
    __shared__ double2 As[TK][TM + 1];
    __shared__ double2 Bs[TK][TN + 1];
    const int t = threadIdx.x;
    const int tx = t & 7, ty = t >> 3;
    const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

    for (int64_t k0 = 0; k0 < K; k0 += TK) {
        if (!CONJ_A) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {  // A tile: 32 rows x 16 k, coalesced along k
                int mm = (t >> 4) + 4 * r, kk = t & 15;
                int64_t gm = m0 + mm, gk = k0 + kk;
                As[kk][mm] = (gm < M && gk < K) ? A[gm * lda + gk] : make_double2(0.0, 0.0);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) {  // op(A)[m][k] = conj(A[k][m]), coalesced along m
                int mm = t & 31, kk = (t >> 5) + 2 * r;
                int64_t gm = m0 + mm, gk = k0 + kk;
                double2 v = (gm < M && gk < K) ? A[gk * lda + gm] : make_double2(0.0, 0.0);
                As[kk][mm] = make_double2(v.x, -v.y);
            }
        }
        if (!CONJ_B) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {  // B tile: 16 k x 32 n, coalesced along n
                int nn = t & 31, kk = (t >> 5) + 2 * r;
                int64_t gk = k0 + kk, gn = n0 + nn;
                Bs[kk][nn] = (gk < K && gn < N) ? B[gk * ldb + gn] : make_double2(0.0, 0.0);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) {  // op(B)[k][n] = conj(B[n][k]), coalesced along k
                int kk = t & 15, nn = (t >> 4) + 4 * r;
                int64_t gk = k0 + kk, gn = n0 + nn;
                double2 v = (gk < K && gn < N) ? B[gn * ldb + gk] : make_double2(0.0, 0.0);
                Bs[kk][nn] = make_double2(v.x, -v.y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            double2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 8 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 8 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t gm = m0 + ty + 8 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gn = n0 + tx + 8 * j;
            if (gn >= N) continue;
            double2 v = make_double2(alpha * acc[i][j].x, alpha * acc[i][j].y);
            if (beta != 0.0) {
                double2 c = C[gm * ldc + gn];
                v.x = fma(beta, c.x, v.x);
                v.y = fma(beta, c.y, v.y);
            }
            C[gm * ldc + gn] = v;
        }
    }
}

// Small products (fewer 32 x 32 tiles than SMs): FP64 issue is a few DFMA per clock per SM,
// so the work is spread over as many SMs as possible instead of reused through shared
// memory.  One warp per CTA computes 8 consecutive outputs of the row-major M x N result;
// the 4 lanes of an output take every 4th k and are summed by shuffles.
template <bool CONJ_A, bool CONJ_B>
__global__ void __launch_bounds__(32) zgemm_small_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                         const double2 *__restrict__ A, int64_t lda,
                                                         const double2 *__restrict__ B, int64_t ldb, double beta,
                                                         double2 *__restrict__ C, int64_t ldc) {
    const int lane = threadIdx.x, q = lane & 3;
    const int64_t idx = (int64_t)blockIdx.x * 8 + (lane >> 2);
    const bool valid = idx < M * N;
    const int64_t m = valid ? idx / N : 0, n = valid ? idx % N : 0;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t k = q; k < K; k += 4) {
        double2 a = CONJ_A ? A[k * lda + m] : A[m * lda + k];
        double2 b = CONJ_B ? B[n * ldb + k] : B[k * ldb + n];
        if (CONJ_A) a.y = -a.y;
        if (CONJ_B) b.y = -b.y;
        acc = cfma(a, b, acc);
    }
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (!valid || q != 0) return;
    double2 v = make_double2(alpha * acc.x, alpha * acc.y);
    if (beta != 0.0) {
        const double2 c = C[m * ldc + n];
        v.x = fma(beta, c.x, v.x);
        v.y = fma(beta, c.y, v.y);
    }
    C[m * ldc + n] = v;
}

__global__ void lincomb_kernel(int64_t D, double c0, const double2 *A, double c1, const double2 *B,
                               double c2, const double2 *C, double c3, double c4, double2 *Y) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    double2 y = make_double2(0.0, 0.0);
    if (c4 != 0.0) { y = Y[idx]; y.x *= c4; y.y *= c4; }
    if (A) { y.x = fma(c0, A[idx].x, y.x); y.y = fma(c0, A[idx].y, y.y); }
    if (B) { y.x = fma(c1, B[idx].x, y.x); y.y = fma(c1, B[idx].y, y.y); }
    if (C) { y.x = fma(c2, C[idx].x, y.x); y.y = fma(c2, C[idx].y, y.y); }
    if (idx / D == idx % D) y.x += c3;
    Y[idx] = y;
}

__global__ void scale_minus_i_kernel(int64_t D, double theta, const double2 *H, double2 *X) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    double2 h = H[idx];
    X[idx] = make_double2(theta * h.y, -theta * h.x);  // -i theta (hr + i hi)
}

__global__ void pade_augment_kernel(int64_t D, const double2 *Up, const double2 *Vp, double2 *aug) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    int64_t r = idx / D, c = idx % D;
    double2 u = Up[idx], v = Vp[idx];
    aug[r * 2 * D + c] = make_double2(v.x - u.x, v.y - u.y);
    aug[r * 2 * D + D + c] = make_double2(v.x + u.x, v.y + u.y);
}

// aug (D x 4D) = [V - U | V + U | dV + dU | dV - dU]
__global__ void frechet_augment_kernel(int64_t D, const double2 *Up, const double2 *Vp, const double2 *dUp,
                                       const double2 *dVp, double2 *aug) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    int64_t r = idx / D, c = idx % D;
    const double2 u = Up[idx], v = Vp[idx], du = dUp[idx], dv = dVp[idx];
    double2 *row = aug + r * 4 * D;
    row[c] = make_double2(v.x - u.x, v.y - u.y);
    row[D + c] = make_double2(v.x + u.x, v.y + u.y);
    row[2 * D + c] = make_double2(dv.x + du.x, dv.y + du.y);
    row[3 * D + c] = make_double2(dv.x - du.x, dv.y - du.y);
}

// out (D x D) = columns [c0, c0 + D) of the D x W matrix aug
__global__ void take_block_kernel(int64_t D, int64_t W, int64_t c0, const double2 *aug, double2 *out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    out[idx] = aug[(idx / D) * W + c0 + idx % D];
}

// One block: pivot search in column k (rows >= k), row swap, scaling of row k.
__global__ void __launch_bounds__(1024) gj_pivot_kernel(int64_t D, int64_t W, int64_t k, double2 *aug,
                                                        uint32_t *err) {
    __shared__ double best[1024];
    __shared__ int64_t arg[1024];
    const int t = threadIdx.x;
    double b = -1.0;
    int64_t a = k;
    for (int64_t i = k + t; i < D; i += blockDim.x) {
        double2 v = aug[i * W + k];
        double m = v.x * v.x + v.y * v.y;
        if (m > b) { b = m; a = i; }
    }
    best[t] = b;
    arg[t] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) {
            if (best[t + s] > best[t] || (best[t + s] == best[t] && arg[t + s] < arg[t])) {
                best[t] = best[t + s];
                arg[t] = arg[t + s];
            }
        }
        __syncthreads();
    }
    const int64_t p = arg[0];
    if (!(best[0] > 0.0)) {
        if (t == 0) atomicOr(err, kErrSingular);
        return;
    }
    if (p != k) {
        for (int64_t j = k + t; j < W; j += blockDim.x) {
            double2 x = aug[k * W + j];
            aug[k * W + j] = aug[p * W + j];
            aug[p * W + j] = x;
        }
    }
    __syncthreads();
    double2 piv = aug[k * W + k];
    double den = piv.x * piv.x + piv.y * piv.y;
    double2 inv = make_double2(piv.x / den, -piv.y / den);
    __syncthreads();
    for (int64_t j = k + 1 + t; j < W; j += blockDim.x) {
        double2 x = aug[k * W + j];
        aug[k * W + j] = make_double2(x.x * inv.x - x.y * inv.y, x.x * inv.y + x.y * inv.x);
    }
    if (t == 0) aug[k * W + k] = make_double2(1.0, 0.0);
}

// rows i != k: row_i -= aug[i][k] * row_k, for columns j > k.
__global__ void gj_eliminate_kernel(int64_t D, int64_t W, int64_t k, double2 *aug, const uint32_t *err) {
    if (*err & kErrSingular) return;
    const int64_t i = blockIdx.y;
    const int64_t j = k + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == k || j >= W) return;
    double2 f = aug[i * W + k];
    double2 r = aug[k * W + j];
    double2 x = aug[i * W + j];
    x.x -= f.x * r.x - f.y * r.y;
    x.y -= f.x * r.y + f.y * r.x;
    aug[i * W + j] = x;
}

__global__ void take_right_half_kernel(int64_t D, const double2 *aug, double2 *R) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    R[idx] = aug[(idx / D) * 2 * D + D + idx % D];
}

// Pairs of long incoming lists (many jumps into one state, e.g. every leak into the
// vacuum): the whole warp (blockDim.x == 32, every lane present) merges each such pair.
// Lanes take every 32nd entry of the shorter list and find its jump in the longer one by
// bisection; the owner lane of the pair gets scale * sum c_p c_q X[src_p, src_q] added to
// acc.  Returns whether this lane's own pair was handled here.
constexpr int kLongMergeF64 = 32;

__device__ bool long_merge_f64(int64_t D, const double2 *X, const int32_t *in_jump, const int32_t *in_src,
                               const double *in_coef, int p, int pe, int q, int qe, double scale, double2 &acc) {
    const bool is_long = pe > p && qe > q && (pe - p) + (qe - q) > kLongMergeF64;
    unsigned longs = __ballot_sync(0xffffffffu, is_long);
    const int lane = threadIdx.x;
    while (longs) {
        const int owner = __ffs(longs) - 1;
        longs &= longs - 1;
        const int op = __shfl_sync(0xffffffffu, p, owner), ope = __shfl_sync(0xffffffffu, pe, owner);
        const int oq = __shfl_sync(0xffffffffu, q, owner), oqe = __shfl_sync(0xffffffffu, qe, owner);
        const bool m_short = ope - op <= oqe - oq;
        const int s0 = m_short ? op : oq, s1 = m_short ? ope : oqe;
        const int l0 = m_short ? oq : op, l1 = m_short ? oqe : ope;
        double sx = 0.0, sy = 0.0;
        for (int e = s0 + lane; e < s1; e += 32) {
            const int j = in_jump[e];
            int lo = l0, hi = l1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (in_jump[mid] < j)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            if (lo < l1 && in_jump[lo] == j) {
                const int ep = m_short ? e : lo, eq = m_short ? lo : e;
                const double c = scale * in_coef[ep] * in_coef[eq];
                const double2 g = X[(int64_t)in_src[ep] * D + in_src[eq]];
                sx = fma(c, g.x, sx);
                sy = fma(c, g.y, sy);
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, off);
            sy += __shfl_xor_sync(0xffffffffu, sy, off);
        }
        if (lane == owner) {
            acc.x += sx;
            acc.y += sy;
        }
    }
    return is_long;
}

// out = B + tau [ -(d_m + d_n)/2 X_mn + sum_j c_j(m) c_j(n) X[src_j(m), src_j(n)] ]: a stage
// of the explicit midpoint rule for the Lindblad term (Eq. 3).  out may be B (each
// element reads only its own B entry), never X.
__global__ void lindblad_axpy_f64_kernel(int64_t D, const double2 *__restrict__ X, const double2 *B, double2 *out,
                                         const double *__restrict__ anti, const int32_t *__restrict__ in_ptr,
                                         const int32_t *__restrict__ in_jump, const int32_t *__restrict__ in_src,
                                         const double *__restrict__ in_coef, double tau) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const bool inside = m < D && n < D;  // outside lanes stay for the warp-shared merge
    const int64_t mc = inside ? m : 0, nc = inside ? n : 0;
    const double2 x = X[mc * D + nc];
    const double h = -0.5 * (anti[mc] + anti[nc]);
    double2 l = make_double2(h * x.x, h * x.y);
    int a = inside ? in_ptr[m] : 0, ae = inside ? in_ptr[m + 1] : 0;
    int b = inside ? in_ptr[n] : 0, be = inside ? in_ptr[n + 1] : 0;
    if (long_merge_f64(D, X, in_jump, in_src, in_coef, a, ae, b, be, 1.0, l)) ae = a;
    while (a < ae && b < be) {  // jumps present in both incoming lists
        const int ja = in_jump[a], jb = in_jump[b];
        if (ja < jb) {
            ++a;
        } else if (ja > jb) {
            ++b;
        } else {
            const double c = in_coef[a] * in_coef[b];
            const double2 g = X[(int64_t)in_src[a] * D + in_src[b]];
            l.x = fma(c, g.x, l.x);
            l.y = fma(c, g.y, l.y);
            ++a;
            ++b;
        }
    }
    if (!inside) return;
    const double2 base = B[m * D + n];
    out[m * D + n] = make_double2(fma(tau, l.x, base.x), fma(tau, l.y, base.y));
}

// p[k] = Re rho_kk
__global__ void diag_kernel(int64_t D, const double2 *rho, double *p) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < D) p[k] = rho[k * D + k].x;
}

// keep[k] = 1 if the probability's growth speed |p1 - p0| / T or the probability itself
// is at least eps (state space selection, Sec. 3.2)
__global__ void select_kernel(int64_t D, const double *p0, const double *p1, double inv_T, double eps,
                              int32_t *keep) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    const double growth = fabs(p1[k] - p0[k]) * inv_T;
    keep[k] = (growth >= eps || p1[k] >= eps) ? 1 : 0;
}

// out[a][b] = rho[idx[a]][idx[b]] (n x n from D x D)
__global__ void gather_kernel(int64_t D, const double2 *rho, int64_t n, const int64_t *idx, double2 *out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t a = e / n, b = e % n;
    out[e] = rho[idx[a] * D + idx[b]];
}

__global__ void dissipate_f64_kernel(int64_t D, const double2 *__restrict__ V, double2 *__restrict__ rho,
                                     const double *__restrict__ anti, const int32_t *__restrict__ in_ptr,
                                     const int32_t *__restrict__ in_jump, const int32_t *__restrict__ in_src,
                                     const double *__restrict__ in_coef, double dt) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const bool inside = m < D && n < D;  // outside lanes stay for the warp-shared merge
    const int64_t mc = inside ? m : 0, nc = inside ? n : 0;
    double2 v = V[mc * D + nc];
    double f = 1.0 - 0.5 * dt * (anti[mc] + anti[nc]);
    double2 out = make_double2(v.x * f, v.y * f);
    int a = inside ? in_ptr[m] : 0, ae = inside ? in_ptr[m + 1] : 0;
    int b = inside ? in_ptr[n] : 0, be = inside ? in_ptr[n + 1] : 0;
    if (long_merge_f64(D, V, in_jump, in_src, in_coef, a, ae, b, be, dt, out)) ae = a;
    while (a < ae && b < be) {  // jumps present in both incoming lists
        int ja = in_jump[a], jb = in_jump[b];
        if (ja < jb) {
            ++a;
        } else if (ja > jb) {
            ++b;
        } else {
            double c = dt * in_coef[a] * in_coef[b];
            double2 g = V[(int64_t)in_src[a] * D + in_src[b]];
            out.x = fma(c, g.x, out.x);
            out.y = fma(c, g.y, out.y);
            ++a;
            ++b;
        }
    }
    if (!inside) return;
    rho[m * D + n] = out;
}

__global__ void __launch_bounds__(256) observables_kernel(int64_t D, const double2 *rho, const double *w,
                                                          const int32_t *ids, double *out) {
    __shared__ double part[256];
    const int o = blockIdx.x;
    const int id = ids[o];
    const int t = threadIdx.x;
    double s = 0.0;
    if (id < D) {
        if (t == 0) s = rho[(int64_t)id * D + id].x;
    } else {
        const double *wr = w + (int64_t)(id - D) * D;
        for (int64_t k = t; k < D; k += blockDim.x) s += wr[k] * rho[k * D + k].x;
    }
    part[t] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (t < st) part[t] += part[t + st];
        __syncthreads();
    }
    if (t == 0) out[o] = part[0];
}

__global__ void __launch_bounds__(1024) trace_kernel(int64_t D, const double2 *rho, double *tr, uint32_t *err) {
    __shared__ double part[1024];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t k = t; k < D; k += blockDim.x) s += rho[k * D + k].x;
    part[t] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (t < st) part[t] += part[t + st];
        __syncthreads();
    }
    if (t == 0) {
        *tr = part[0];
        if (!isfinite(part[0]) || !(part[0] > 0.0)) atomicOr(err, kErrNonFinite);
    }
}

__global__ void symmetrise_kernel(int64_t D, double2 *rho, const double *tr, const uint32_t *err) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= D || j >= D || j < i) return;
    if (*err & kErrNonFinite) return;
    const double inv = 1.0 / *tr;
    double2 a = rho[i * D + j], b = rho[j * D + i];
    double2 s = make_double2(0.5 * (a.x + b.x) * inv, 0.5 * (a.y - b.y) * inv);
    if (i == j) s.y = 0.0;
    rho[i * D + j] = s;
    rho[j * D + i] = make_double2(s.x, -s.y);
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void zgemm_ex(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha, const double2 *A, int64_t lda,
              bool conj_a, const double2 *B, int64_t ldb, bool conj_b, double beta, double2 *C, int64_t ldc) {
    count_launches(1);
    dim3 grid(blocks_for(N, TN), blocks_for(M, TM));
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 148;
    if ((int64_t)grid.x * grid.y < sms) {
        const unsigned nb = blocks_for(M * N, 8);
        if (conj_a) {
            if (conj_b)
                zgemm_small_kernel<true, true><<<nb, 32, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
            else
                zgemm_small_kernel<true, false><<<nb, 32, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
        } else {
            if (conj_b)
                zgemm_small_kernel<false, true><<<nb, 32, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
            else
                zgemm_small_kernel<false, false><<<nb, 32, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
        }
        return;
    }
    if (conj_a) {
        if (conj_b)
            zgemm_kernel<true, true><<<grid, 64, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
        else
            zgemm_kernel<true, false><<<grid, 64, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    } else {
        if (conj_b)
            zgemm_kernel<false, true><<<grid, 64, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
        else
            zgemm_kernel<false, false><<<grid, 64, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    }
}

void zgemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha, const double2 *A, int64_t lda,
           const double2 *B, int64_t ldb, bool conj_b, double beta, double2 *C, int64_t ldc) {
    zgemm_ex(s, M, N, K, alpha, A, lda, false, B, ldb, conj_b, beta, C, ldc);
}

void zlincomb(cudaStream_t s, int64_t D, double c0, const double2 *A, double c1, const double2 *B, double c2,
              const double2 *C, double c3, double c4, double2 *Y) {
    count_launches(1);
    lincomb_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, c0, A, c1, B, c2, C, c3, c4, Y);
}

void scale_minus_i(cudaStream_t s, int64_t D, double theta, const double2 *H, double2 *X) {
    count_launches(1);
    scale_minus_i_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, theta, H, X);
}

void pade_augment(cudaStream_t s, int64_t D, const double2 *Up, const double2 *Vp, double2 *aug) {
    count_launches(1);
    pade_augment_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, Up, Vp, aug);
}

void gauss_jordan(cudaStream_t s, int64_t D, double2 *aug, uint32_t *err) { gauss_jordan_w(s, D, 2 * D, aug, err); }

void gauss_jordan_w(cudaStream_t s, int64_t D, int64_t W, double2 *aug, uint32_t *err) {
    count_launches(2 * D);
    for (int64_t k = 0; k < D; ++k) {
        gj_pivot_kernel<<<1, 1024, 0, s>>>(D, W, k, aug, err);
        int64_t cols = W - k - 1;
        if (cols > 0) {
            dim3 grid(blocks_for(cols, 256), (unsigned)D);
            gj_eliminate_kernel<<<grid, 256, 0, s>>>(D, W, k, aug, err);
        }
    }
}

void frechet_augment(cudaStream_t s, int64_t D, const double2 *Up, const double2 *Vp, const double2 *dUp,
                     const double2 *dVp, double2 *aug) {
    count_launches(1);
    frechet_augment_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, Up, Vp, dUp, dVp, aug);
}

void take_block(cudaStream_t s, int64_t D, int64_t W, int64_t c0, const double2 *aug, double2 *out) {
    count_launches(1);
    take_block_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, W, c0, aug, out);
}

void take_right_half(cudaStream_t s, int64_t D, const double2 *aug, double2 *R) {
    count_launches(1);
    take_right_half_kernel<<<blocks_for(D * D, 256), 256, 0, s>>>(D, aug, R);
}

void dissipate_f64(cudaStream_t s, int64_t D, const double2 *V, double2 *rho, const double *anti,
                   const int32_t *in_ptr, const int32_t *in_jump, const int32_t *in_src, const double *in_coef,
                   double dt) {
    count_launches(1);
    dim3 block(32, 8);
    dim3 grid(blocks_for(D, 32), blocks_for(D, 8));
    dissipate_f64_kernel<<<grid, block, 0, s>>>(D, V, rho, anti, in_ptr, in_jump, in_src, in_coef, dt);
}

void lindblad_axpy_f64(cudaStream_t s, int64_t D, const double2 *X, const double2 *B, double2 *out,
                       const double *anti, const int32_t *in_ptr, const int32_t *in_jump, const int32_t *in_src,
                       const double *in_coef, double tau) {
    count_launches(1);
    dim3 block(32, 8);
    dim3 grid(blocks_for(D, 32), blocks_for(D, 8));
    lindblad_axpy_f64_kernel<<<grid, block, 0, s>>>(D, X, B, out, anti, in_ptr, in_jump, in_src, in_coef, tau);
}

void diag_f64(cudaStream_t s, int64_t D, const double2 *rho, double *p) {
    count_launches(1);
    diag_kernel<<<blocks_for(D, 256), 256, 0, s>>>(D, rho, p);
}

void select_states_flags(cudaStream_t s, int64_t D, const double *p0, const double *p1, double inv_T, double eps,
                         int32_t *keep) {
    count_launches(1);
    select_kernel<<<blocks_for(D, 256), 256, 0, s>>>(D, p0, p1, inv_T, eps, keep);
}

void gather_submatrix(cudaStream_t s, int64_t D, const double2 *rho, int64_t n, const int64_t *idx, double2 *out) {
    count_launches(1);
    gather_kernel<<<blocks_for(n * n, 256), 256, 0, s>>>(D, rho, n, idx, out);
}

void observables(cudaStream_t s, int64_t D, const double2 *rho, const double *weights, const int32_t *ids,
                 int32_t n_obs, double *out) {
    if (n_obs <= 0) return;
    count_launches(1);
    observables_kernel<<<n_obs, 256, 0, s>>>(D, rho, weights, ids, out);
}

void renormalise(cudaStream_t s, int64_t D, double2 *rho, double *scratch, uint32_t *err) {
    count_launches(2);
    trace_kernel<<<1, 1024, 0, s>>>(D, rho, scratch, err);
    dim3 block(32, 8);
    dim3 grid(blocks_for(D, 32), blocks_for(D, 8));
    symmetrise_kernel<<<grid, block, 0, s>>>(D, rho, scratch, err);
}

}  // namespace qed
