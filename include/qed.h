/*
 * qed.h — C ABI of libqed, a single-GPU (GB300, sm_103a) integrator of the quantum
 * master equation (QME) of finite-dimensional cavity QED models.
 *
 * The method (Li, Miao, Ozhigov, "Supercomputer model of finite-dimensional quantum
 * electrodynamics applications"):
 *   - Sec. 2, first point: basis states are strings of digits (photon numbers of the
 *     cavity modes, atom bits, further two-level degrees of freedom); H is the energy
 *     operator on that basis (Eqs. 6-12 give the JC/TC/JCH terms used here).
 *   - Sec. 2, second point: the QME i hbar rho' = [H, rho] + i L(rho) (Eq. 2) with the
 *     Lindblad term L(rho) = sum_j gamma_j (A_j rho A_j^+ - 1/2 {A_j^+ A_j, rho}) (Eq. 3).
 *   - Sec. 4.2, Table 3: the two stages "Taylor approximation" (the propagator
 *     U = exp(-i H dt), here by scaling-and-squaring Pade in FP64 on the GPU) and
 *     "unitary evolution" (rho -> U rho U^+ per step, followed here by one explicit
 *     Euler step of the Lindblad term).
 *
 * Units: hbar = 1; every frequency, coupling and rate is an angular frequency.
 *
 * Memory: every rho / records / gradient buffer is owned by the caller (device memory
 * unless stated otherwise).  Operators, propagators and work space are owned by the
 * model and released by qed_free.  All device work is enqueued on the caller's stream;
 * only qed_build and qed_sync_status synchronise.  Errors are returned as codes (never
 * abort/exit/trap); qed_last_error() gives a thread-local message for the last failure.
 *
 * Density matrices are complex128, row-major, D x D, interleaved (re, im) — the layout
 * of a contiguous torch.complex128 tensor.  Rows and columns follow the basis order
 * returned by qed_basis_labels.
 */
#ifndef QED_H
#define QED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st *qed_stream;

typedef enum {
    QED_OK = 0,
    QED_EINVAL = 1,        /* bad argument or model specification              */
    QED_ENOMEM = 2,        /* device or host allocation failed                 */
    QED_ECUDA = 3,         /* a CUDA runtime/driver call failed                */
    QED_ETIMEOUT = 4,      /* a bounded device wait ran out                    */
    QED_ENUMERIC = 5,      /* non-finite values or a singular Pade denominator */
    QED_EUNSUPPORTED = 6   /* valid request the library does not implement     */
} qed_status;

typedef enum {
    QED_FP64 = 0,          /* U rho U^+ as two FP64 complex GEMMs                          */
    QED_SPLIT_FP16x2 = 1,  /* increment form on tcgen05: FP16 hi+lo operands, FP32 accumulate */
    QED_SPLIT_BF16x3 = 2,  /* reserved                                                    */
    QED_SPLIT_TF32x3 = 3   /* reserved                                                    */
} qed_precision;

/* Time-stepping schemes for the two stages of Table 3 (the unitary evolution of Eq. 2 and
 * the Lindblad term of Eq. 3; the paper does not state how they are combined). */
enum {
    QED_SCHEME_LIE = 0,    /* rho <- E(dt) U rho U^+, E(t) one explicit Euler step: first order */
    QED_SCHEME_STRANG = 1, /* rho <- E2(dt/2) U E2(dt/2)(rho) U^+, E2(t) X = X + t L(X + t/2 L(X))
                              (explicit midpoint rule): second order in dt                   */
    QED_SCHEME_EFFECTIVE = 2 /* Eq. 3 regrouped: V = U_eff rho U_eff^+ with
                              U_eff = exp(-i dt (H - i/2 sum_j gamma_j A_j^+ A_j)) (the
                              anticommutator inside the propagator), then
                              rho <- V + dt sum_j gamma_j A_j V A_j^+: first order, completely
                              positive, trace kept to O(dt^2) per step                       */
};

/* Basis kinds (Sec. 4.2, Eqs. 10-11 restrict the 2^Area product space to one photon). */
enum {
    QED_BASIS_FULL = 0,        /* full product space, mixed-radix order (first digit slowest) */
    QED_BASIS_CAP = 1,         /* states with <= excitation_cap excitations, mixed-radix order */
    QED_BASIS_SINGLE_G = 2,    /* vacuum, then per cavity: its photon, then its atoms          */
    QED_BASIS_FIRST_D = 3,     /* first dim_cap states ordered by (excitations, mixed radix)  */
    QED_BASIS_SECTOR = 4       /* exactly excitation_cap excitations, mixed-radix order       */
};

/* Jump operator kinds for Eq. (3). */
enum {
    QED_JUMP_A = 0,        /* a_c: photon loss from cavity `site`                               */
    QED_JUMP_SIGMA = 1,    /* sigma_a: decay of atom `site` (atoms numbered cavity by cavity)   */
    QED_JUMP_DEPHASE = 2,  /* sigma_z = |1><1| - |0><0| on extra two-level digit `site`         */
    QED_JUMP_LEAK = 3      /* |G><photon_c|: the one-photon state of cavity `site` -> vacuum    */
};

/*
 * Model specification (Sec. 2, first two points).  Digits of a basis state: for each
 * cavity c its photon number 0..n_max[c] followed by one bit per atom in that cavity,
 * then one bit per extra two-level degree of freedom.  An excitation is a photon or an
 * excited atom (extra digits are not counted).
 *
 * H = sum_c omega_c a_c^+ a_c + sum_a omega_a s_a^+ s_a            (Eqs. 8b-8d, 12)
 *   + sum_a g[a] (a_c(a)^+ s_a + a_c(a) s_a^+)                     (JC / TC coupling, Eq. 8b)
 *   + sum_b zeta[b] (a_i^+ a_j + a_i a_j^+),  (i, j) = bond_ij[2b..2b+1]   (hopping, Eq. 12)
 *   + sum_x extra_tunnel[x] sigma_x(x)                              (two-site tunnelling, Eq. 4)
 * projected on the chosen basis.  All arrays are caller-owned and copied by the callee.
 */
typedef struct {
    int32_t n_cavities;
    const int32_t *atoms_per_cavity;   /* [n_cavities] */
    const int32_t *n_max;              /* [n_cavities] photon truncation */
    int32_t n_extra;
    int32_t basis_kind;                /* QED_BASIS_* */
    int32_t excitation_cap;
    int64_t dim_cap;
    double omega_c, omega_a;
    const double *g;                   /* [total atoms] */
    int32_t n_bonds;
    const int32_t *bond_ij;            /* [2 * n_bonds] cavity pairs */
    const double *zeta;                /* [n_bonds] */
    const double *extra_tunnel;        /* [n_extra] */
    int32_t n_jumps;
    const int32_t *jump_kind;          /* [n_jumps] QED_JUMP_* */
    const int32_t *jump_site;          /* [n_jumps] */
    const double *gamma;               /* [n_jumps] rates, >= 0 */
} qed_spec;

typedef struct qed_model qed_model;   /* opaque, library-owned */

/* ---------------------------------------------------------------- host-only queries
 * These run the host-side model builder only (no GPU needed).                         */

/* Basis dimension and digit count of a specification.  EINVAL on a malformed spec. */
qed_status qed_spec_dim(const qed_spec *spec, int64_t *dim, int32_t *n_digits);

/* Basis states as digits, host int32 [dim x n_digits] (capacity in elements). */
qed_status qed_spec_basis(const qed_spec *spec, int32_t *digits, int64_t capacity);

/* Dense projected H, host complex128 [dim x dim] interleaved (capacity in complex). */
qed_status qed_spec_hamiltonian(const qed_spec *spec, double *H, int64_t capacity);

/* Dense projected A_j (not scaled by gamma), host complex128 [dim x dim]. */
qed_status qed_spec_jump(const qed_spec *spec, int32_t j, double *A, int64_t capacity);

/* The operators of the model restricted to the basis states keep[0..n-1] (increasing
 * indices into the spec's basis), as qed_select_states builds them (Sec. 3.2): j = -1 gives
 * P H P, j >= 0 gives P A_j P (not scaled by gamma), host complex128 [n x n]; d (host FP64
 * [n], or NULL) receives d_k = sum_j gamma_j (P A_j^+ P A_j P)_kk.  EINVAL for an empty or
 * unsorted list or a small buffer. */
qed_status qed_spec_restricted(const qed_spec *spec, const int64_t *keep, int64_t n, int32_t j, double *out,
                               int64_t capacity, double *d);

/* ---------------------------------------------------------------- model lifetime */

/* Build basis, H, jump tables and observables on the host, upload them, and compute
 * U = exp(-i H dt) on the device in FP64 (Pade-13 scaling and squaring; the
 * "Taylor approximation" stage of Sec. 4.2).  In split precision also prepares the
 * diagonal phase P = diag(exp(-i H_kk dt)), Delta = P^-1 U - I and its FP16 hi/lo
 * operand planes.  Synchronises `stream`.  EINVAL on a bad spec, ENOMEM, ECUDA,
 * ENUMERIC (singular Pade denominator), EUNSUPPORTED for reserved precisions. */
qed_status qed_build(const qed_spec *spec, double dt, qed_precision prec, qed_stream stream,
                     qed_model **out);

qed_status qed_free(qed_model *m);

qed_status qed_dim(const qed_model *m, int64_t *dim);

/* Digits of every basis state, host int32 [dim x n_digits]; n_digits from qed_spec_dim. */
qed_status qed_basis_labels(const qed_model *m, int32_t *digits);

/* Index of the basis state with the given digits (host int32 [n_digits]); EINVAL and
 * *index = -1 if it is not in the basis. */
qed_status qed_basis_index(const qed_model *m, const int32_t *digits, int64_t *index);

/* Number of observable ids: ids 0..dim-1 are populations rho_kk; id dim is the trace;
 * then <n_c> per cavity, <s_a^+ s_a> per atom, and the extra digits' <1|.|1>. */
qed_status qed_n_observables(const qed_model *m, int32_t *n);

/* Steps between trace renormalisation + Hermitian symmetrisation in split precision
 * (0 = never; default 100).  Ignored in FP64. */
qed_status qed_set_renorm_every(qed_model *m, int32_t every);

/* The time-stepping scheme (QED_SCHEME_LIE, the default, QED_SCHEME_STRANG or
 * QED_SCHEME_EFFECTIVE) that qed_evolve and qed_evolve_batched use from now on; the Strang
 * scheme runs four Lindblad stages per step instead of one.  Switching to or from the
 * effective scheme recomputes the propagator (U_eff = exp(X), X = -i dt H - (dt/2) diag(d),
 * d_k = sum_j gamma_j (A_j^+ A_j)_kk, by Pade-13 scaling and squaring; every jump operator
 * here is a monomial, so A_j^+ A_j is diagonal) and, in split precision, the increment form
 * with the damped phases P_k = exp(-i H_kk dt - d_k dt/2); under that scheme the split
 * path's periodic pass symmetrises rho without dividing by its trace (the scheme's own
 * trace drift is part of its result).  EINVAL for an unknown scheme; ENOMEM if a buffer
 * cannot be allocated; ENUMERIC for a singular Pade denominator.  Synchronises the device.
 * qed_adjoint differentiates the Lie and Strang steps on both paths, not the effective
 * step (EUNSUPPORTED). */
qed_status qed_set_scheme(qed_model *m, int32_t scheme);

/* Tile autotuner (the paper has no counterpart: it concerns only how this library maps the
 * step's products onto the GPU) for a split-precision model stepped on its own: times
 * `steps` whole steps for each candidate tile width (128 or 256 columns) and split-K
 * factor (1, 2, 4) of the step's two tensor-core products, GEMM1's candidates first, then
 * GEMM2's with the best GEMM1, and keeps the fastest.  (The batched path plans its own
 * grouped launches.)  Writes a description of the choice into `choice` (size choice_cap;
 * may be NULL).  Uses the model's internal state as scratch (the next qed_evolve imports
 * rho again) and drops the captured step graphs; synchronises the device.  FP64 models
 * have nothing to tune (OK).  EINVAL for steps <= 0. */
qed_status qed_autotune(qed_model *m, int32_t steps, char *choice, int32_t choice_cap, qed_stream stream);

/* Sets the tile plan that qed_autotune would otherwise choose (no counterpart in the paper):
 * the tile width (128 or 256 columns) and split-K factor (CTAs per cluster, a power of two:
 * GEMM1 up to 8, GEMM2 up to 4) of the step's two tensor-core products.  qed_evolve_batched
 * takes the two widths for its grouped launches (unsplit) when every model of the batch
 * carries the same ones.  Drops the captured step graphs; synchronises the device.  EINVAL
 * for other values or for more slices than the product has 64-wide K blocks for (two per
 * slice), EUNSUPPORTED for FP64 models. */
qed_status qed_set_plan(qed_model *m, int32_t gemm1_bn, int32_t gemm1_splits, int32_t gemm2_bn, int32_t gemm2_splits,
                        qed_stream stream);

/* The batched counterpart (no counterpart in the paper either): the grouped launches of
 * qed_evolve_batched share one tile plan, so this times `steps` whole batched steps of the
 * n split-precision models `ms` for each pair of tile widths of the two products (GEMM1 256
 * or 128 columns, GEMM2 128 or 256; both unsplit) and stores the fastest in every model; a
 * later qed_evolve_batched uses it when all its models carry the same pair (else 256/256).  The
 * models' internal states are zeroed and used as scratch (qed_evolve_batched imports rho
 * again); synchronises the stream.  Writes the choice and the timings into `choice` (size
 * choice_cap; may be NULL).  EINVAL for n <= 0, steps <= 0, a NULL, repeated or FP64 model. */
qed_status qed_autotune_batched(int32_t n, qed_model *const *ms, int32_t steps, char *choice, int32_t choice_cap,
                                qed_stream stream);

/* ---------------------------------------------------------------- hot path */

/*
 * Advance rho (device complex128 D x D, in/out) by n_steps steps of
 *     V = U rho U^+                          ("unitary evolution", Sec. 4.2, Eq. 2)
 *     rho <- V + dt sum_j gamma_j (A_j V A_j^+ - 1/2 {A_j^+ A_j, V})      (Eq. 3)
 * (the Lie scheme; under QED_SCHEME_STRANG the symmetric step of qed_set_scheme).
 * Records observables obs_ids (host int32 [n_obs]) into records (device FP64,
 * row-major [n_rec x n_obs]) at every local step i in 0..n_steps (before step i+1)
 * with (step_offset + i) % record_every == 0; records may be NULL when n_obs == 0.
 * n_rec = number of such i.  Asynchronous on `stream`: device-side errors (non-finite
 * trace at a renormalisation) surface through qed_sync_status.
 *
 * Split precision (QED_SPLIT_FP16x2) accepts only a density matrix: rho Hermitian and of
 * unit trace (|rho_mn - conj(rho_nm)| <= 1e-8 and |tr rho - 1| <= 1e-6; under
 * QED_SCHEME_EFFECTIVE, whose own steps move the trace, 0 < tr rho <= 1 + 1e-6).  Its first product
 * reads the row-major rho as rho^T = conj(rho), the second forms the Hermitian X = W Delta^+,
 * the FP16 scale assumes |rho_mn| <= 1 and the renormalisation divides by tr rho; any other
 * input would give a silently different answer.  A device check at the start of the call
 * flags a violation, which qed_sync_status returns as EINVAL (the evolved rho is then
 * meaningless).  The FP64 path takes any complex D x D matrix.
 */
qed_status qed_evolve(qed_model *m, void *rho, int64_t n_steps, int64_t step_offset,
                      int32_t record_every, int32_t n_obs, const int32_t *obs_ids,
                      double *records, qed_stream stream);

/*
 * Gradients of the loss L = tr(diag(obs_diag) rho_N) after n_steps steps from rho0 (device
 * complex128 D x D, not modified), by the discrete adjoint of the step qed_evolve takes
 * with the Lie scheme (Eq. 2 and Eq. 3, unitary part then one Euler step of the Lindblad
 * term):
 *   lambda_N = diag(obs_diag);  kappa = J^+(lambda_{n+1});  lambda_n = U^+ kappa U;
 *   dL/dgamma_j = dt sum_n tr(lambda_{n+1} D_j(V_n));
 *   dL/dtheta   = 2 dt Im tr(G dH/dtheta),  G = L_exp(-i dt H, sum_n rho_n U^+ kappa_{n+1}),
 * the Frechet derivative taken once (the Pade-13 approximant and its derivative, i.e. the
 * upper-right block of exp([[X, M], [0, X]]) evaluated on D x D blocks).  rho is
 * checkpointed every `checkpoint_every` steps; every segment but the last is recomputed
 * during the backward pass (the forward pass stores the last one, so checkpoint_every >=
 * n_steps recomputes nothing at the cost of 2 n_steps D^2 x 16 bytes).  Outputs are
 * device FP64: *loss; grad_g[total atoms], grad_zeta[n_bonds], grad_gamma[n_jumps] in the
 * order of the spec (each may be NULL only if its count is 0).  FP64 models use FP64
 * kernels throughout; split-precision models run the forward steps, the co-state steps
 * (as a backward model with U^+ and the outgoing jump lists) and the products
 * rho_n lambda_n in split precision, accumulating M in FP64.  Under QED_SCHEME_STRANG the
 * adjoint of the symmetric step, on both paths: kappa_n = E^+(lambda_{n+1}),
 * mu_n = U^+ kappa_n U, lambda_n = E^+(mu_n) with E the midpoint half step,
 * M = sum_n E(rho_n) U^+ kappa_n, and the rate gradients of both half steps (in split
 * precision the backward model runs the same stages; the forward pass keeps rho_n, E(rho_n)
 * and V_n of a segment).  QED_SCHEME_EFFECTIVE is not differentiated (EUNSUPPORTED).  In split precision rho0 must be Hermitian with unit trace (EINVAL otherwise, as
 * in qed_evolve).  Allocates its work space per call; synchronises `stream`.
 */
qed_status qed_adjoint(qed_model *m, const void *rho0, int64_t n_steps, int32_t checkpoint_every,
                       const double *obs_diag, double *loss, double *grad_g, double *grad_zeta,
                       double *grad_gamma, qed_stream stream);

/*
 * Evolve n independent models together, each by n_steps steps of qed_evolve's step:
 * rhos[i] (device complex128 D_i x D_i, in/out) belongs to ms[i].  For split-precision
 * models every phase of a step is one grouped launch over all instances (the tcgen05
 * GEMM's work items are the 128 x 128 tiles of every instance, largest first; the element
 * kernels' blocks tile every instance), and the step loop is captured in CUDA graphs.
 * FP64 models run one after another.  All models must share one precision and appear
 * once.  records (host array of n device pointers, or NULL): records[i] (device FP64, or
 * NULL) receives the populations rho_kk of instance i, row-major [n_rec x D_i], at steps
 * 0, r, 2r, ... <= n_steps (r = record_every).  Each model's renormalisation setting
 * applies.  Split precision requires each rho to be Hermitian with unit trace (as in
 * qed_evolve); a violation, like any device-side error of an instance, is returned by this
 * call (EINVAL, ETIMEOUT, ENUMERIC) after the final synchronisation.  Synchronises `stream`
 * before returning (it frees the batch's tables).
 */
qed_status qed_evolve_batched(int32_t n, qed_model *const *ms, void *const *rhos, int64_t n_steps,
                              int32_t record_every, double *const *records, qed_stream stream);

/*
 * State space selection (Sec. 3.2, "State space selection algorithm"; Table 1): starting
 * from rho0 (device complex128 D x D of model m, not modified), n_rounds rounds of
 *   solve:      qed_evolve for steps_per_round steps with the current model;
 *   growth:     g_k = |p_k(t + T) - p_k(t)| / T of each state's probability p_k = rho_kk,
 *               T = steps_per_round * dt;
 *   comparison: delete every state with g_k < eps (a state whose probability is at least
 *               eps is kept: a stationary populated state is not what the paper deletes);
 *   normalise:  rho <- the remaining states' block, (rho + rho^+) / (2 tr rho);
 * the model of the remaining states is H and every A_j projected onto them (P H P,
 * P A_j P), with m's dt, precision, scheme and renormalisation interval.  Outputs:
 * *out_model, a new model on the kept states (caller frees it with qed_free; m is left as
 * it was); rho_out (device complex128, capacity D x D) the final n x n density matrix;
 * keep (host int64 [D]) the kept states' indices in m's basis, increasing, first *n_keep
 * valid; sizes (host int64 [n_rounds], or NULL) the dimension after each round.
 * EINVAL for bad arguments, ENUMERIC if every state falls below eps or a trace is not
 * finite.  Allocates its work space; synchronises `stream`.
 */
qed_status qed_select_states(qed_model *m, const void *rho0, int64_t steps_per_round, int32_t n_rounds, double eps,
                             qed_model **out_model, void *rho_out, int64_t *keep, int64_t *n_keep, int64_t *sizes,
                             qed_stream stream);

/* Observables of one rho (device) into out (device FP64 [n_obs]). */
qed_status qed_observables(const qed_model *m, const void *rho, int32_t n_obs,
                           const int32_t *obs_ids, double *out, qed_stream stream);

/* Synchronise `stream` and report device-side errors raised since the last call. */
qed_status qed_sync_status(qed_model *m, qed_stream stream);

/* ---------------------------------------------------------------- test and measurement hooks */

/* Replace U by a caller-provided propagator (device complex128 D x D), e.g. the
 * oracle's, so the step can be compared without the expm's own rounding.  Recomputes
 * Delta and its planes in split precision.  Synchronises `stream`. */
qed_status qed_set_U(qed_model *m, const void *U, qed_stream stream);

/* Copy the model's U (device complex128 D x D) into caller memory (device). */
qed_status qed_get_U(const qed_model *m, void *U, qed_stream stream);

/*
 * Wait-gate test hook (the paper has no counterpart: it exercises this library's own error
 * path).  With closed != 0 the tensor-core kernels of m's split-precision step first wait,
 * for at most budget_cycles SM clock cycles, for a device flag to clear - a flag that nothing
 * clears - before they issue any load or product.  When that wait runs out a kernel records
 * the timeout and skips its work (the step's result is then meaningless) and the next
 * qed_sync_status returns QED_ETIMEOUT; the model stays usable.  closed = 0 removes the
 * wait.  Drops the captured step graphs; synchronises `stream`.  EINVAL for a negative
 * budget, EUNSUPPORTED for FP64 models (that path has no bounded waits).
 */
qed_status qed_set_wait_gate(qed_model *m, int32_t closed, int64_t budget_cycles, qed_stream stream);

/*
 * Allocation-failure test hook (process-wide; the paper has no counterpart): from now on the
 * library's device allocations fail as on an exhausted device (the call that needed them
 * returns QED_ENOMEM and frees what it had allocated) once they would exceed `bytes` bytes
 * in total; bytes < 0 removes the limit.
 */
qed_status qed_set_alloc_budget(int64_t bytes);

/*
 * Run n_steps steps like qed_evolve (no records), timing each kernel class with CUDA
 * events on `stream`; writes the mean duration in milliseconds per step of each class
 * into ms[0..n_kernels-1] and the class names (comma separated) into names (size
 * name_cap).  Synchronises.  For measurement only: it perturbs the pipelining.
 */
qed_status qed_profile(qed_model *m, void *rho, int64_t n_steps, double *ms, int32_t n_kernels,
                       char *names, int32_t name_cap, qed_stream stream);

/*
 * The kernels of a split-precision model's Lie step timed one at a time in steady state:
 * imports rho (not modified), runs one step, then replays each kernel (GEMM1, GEMM2, the
 * Lindblad update) `reps` times back to back from a CUDA graph, as the step loop runs
 * them (each launch's set-up overlapping the previous one's tail), and writes the mean
 * milliseconds per launch into ms[0..n_kernels-1] and the names (comma separated) into
 * names (size name_cap).  Each kernel repeats identical work: it reads only what the
 * others write.  Synchronises.  EUNSUPPORTED for FP64 models and the other schemes.
 */
qed_status qed_profile_replay(qed_model *m, void *rho, int32_t reps, double *ms, int32_t n_kernels, char *names,
                              int32_t name_cap, qed_stream stream);

/*
 * The tensor-core product of the split-precision step, exposed for testing:
 *     out[s] = sum over the K-slices of slice s of  sum_q A_{pa(q)} B_{pb(q)}^T
 * with A = a_planes (device FP16 [planes_a][M][K], K contiguous), B = b_planes (device
 * FP16 [planes_b][N][K]) and the n_seg (<= 6) plane pairs seg_pairs = {pa(0), pb(0), ...}
 * (host int32), e.g. {0,0, 0,1, 1,0} for hi*hi + hi*lo + lo*hi.  out is device FP32
 * [splits][M][N] (split-K partial sums; their sum is the product).  M and N multiples of
 * 128, K of 64, planes 16-byte aligned.  tcgen05.mma (kind::f16, FP32 accumulation in
 * tensor memory) fed by TMA.  Synchronises `stream`.  EINVAL on bad shapes or plane
 * indices, ETIMEOUT if a bounded wait ran out.
 */
qed_status qed_tc_gemm(const void *a_planes, int32_t planes_a, const void *b_planes, int32_t planes_b,
                       int32_t M, int32_t N, int32_t K, int32_t n_seg, const int32_t *seg_pairs,
                       int32_t splits, float *out, qed_stream stream);

/*
 * The same product as qed_tc_gemm, for callers that cannot allocate device memory (code
 * that runs inside another framework's fixed memory pool, or whose allocations are all
 * made up front): it calls no cudaMalloc, cudaFree or allocating library routine.  The
 * split-K partial sums live in a file-scope device array of 4 Mi floats (16 MiB) that
 * every GPU loading the library holds until exit, plus a device error word; out is
 * device FP32 [M][N], the summed product (not the partials).  The paper has no
 * counterpart: this is a deployment variant of the library's own GEMM.
 *   - EINVAL when splits * M * N exceeds 4 Mi floats, or on the shape rules of qed_tc_gemm.
 *   - The first call on a device looks up the array's device address (with that device
 *     current); make that first call before any stream capture.
 *   - Every call shares the array, which keeps the last call's partials; calls whose work
 *     overlaps on the GPU (two streams, two host threads) race on it.
 * Synchronises `stream` to report ETIMEOUT from a bounded device wait.
 */
qed_status qed_tc_gemm_static(const void *a_planes, int32_t planes_a, const void *b_planes, int32_t planes_b,
                              int32_t M, int32_t N, int32_t K, int32_t n_seg, const int32_t *seg_pairs,
                              int32_t splits, float *out, qed_stream stream);

/* Total number of kernels this library has launched in this process (all models). */
qed_status qed_launch_count(int64_t *count);

const char *qed_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QED_H */
