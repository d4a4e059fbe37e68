"""Plain FP64 CPU oracle of the cavity-QED quantum master equation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module: only
the tests, the smoke check and the bench's CPU-baseline / reference leg use it.  It
shares no code with the CUDA library; the two meet only through the seeded model
dictionaries of `qed_workloads`.

What it computes (Li, Miao, Ozhigov, "Supercomputer model of finite-dimensional
quantum electrodynamics applications"):

* the QME of Eq. (2), i hbar drho/dt = [H, rho] + i L(rho), with hbar = 1, i.e.
  drho/dt = -i [H, rho] + L(rho);
* the Lindblad term of Eq. (3), L(rho) = sum_j gamma_j (A_j rho A_j^+ - 1/2 {A_j^+ A_j, rho})
  (the printed anticommutator lacks its second argument; it is read as {A^+A, rho});
* the two stages the paper times (Sec. 4.2, Table 3): the propagator U = exp(-i H dt)
  ("Taylor approximation" stage; here by eigendecomposition, a different method from
  the GPU's Pade), then the "unitary evolution" V = U rho U^+ followed by one explicit
  Euler step of the Lindblad term on V (Lie splitting, unitary first):

      rho_{n+1} = V + dt * sum_j gamma_j (A_j V A_j^+ - 1/2 (A_j^+A_j V + V A_j^+A_j)).

* basis states as digit strings (Sec. 2, first point; Eqs. 6, 9, 10, 11): per cavity a
  photon number 0..n_max and one bit per atom, then the extra two-level digits; the
  mixed-radix order puts the first digit most significant.
* the Hamiltonian terms of Eqs. (8b)-(8d) (omega a^+a + omega sigma^+sigma +
  g (a sigma^+ + a^+ sigma)), the hopping term of Eq. (12) (zeta (a_i^+ a_j + a_i a_j^+) on
  each nearest-neighbour pair once) and a transverse term zeta sigma_x on extra
  two-level digits (the tunnelling of Eq. 4 written in its eigenbasis-free form).
* two further step schemes built from the same two stages: the symmetric (Strang) step,
  and the effective-Hamiltonian form of Eq. (3) regrouped (U_eff = exp(-i dt (H - i/2
  sum gamma A^+A)) carries the anticommutator, one Euler step adds the jump terms).
* discrete adjoint gradients of tr(O rho_N) with respect to g, zeta and gamma.

Every function below is pinned by tests that do not re-derive it: closed forms (Rabi
oscillation, tight-binding lattice, discrete photon decay), the dimensions the paper
prints, brute force on the vectorised superoperator, a Kronecker-product construction
of the same operators, invariants, and central finite differences.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

JUMP_A = 0        # a_c, photon loss from cavity c
JUMP_SIGMA = 1    # sigma_a, atom a decays
JUMP_DEPHASE = 2  # sigma_z on extra two-level digit x
JUMP_LEAK = 3     # |G><photon_c|, a photon in cavity c leaks to the vacuum state


# --------------------------------------------------------------------------- basis
class Basis:
    """Basis states as rows of digits, plus the digit layout and a reverse index."""

    def __init__(self, model, digits):
        self.model = model
        self.digits = np.asarray(digits, dtype=np.int64)
        self.layout = digit_layout(model)
        self.dim = self.digits.shape[0]
        self.index = {row.tobytes(): k for k, row in enumerate(self.digits)}

    def find(self, digits):
        """Index of the state with these digits, or -1 if it is outside the basis."""
        return self.index.get(np.asarray(digits, dtype=np.int64).tobytes(), -1)

    def photon_digit(self, c):
        return self.layout["photon_digit"][c]

    def atom_digit(self, a):
        return self.layout["atom_digit"][a]

    def extra_digit(self, x):
        return self.layout["extra_digit"][x]


def digit_layout(model):
    """Digit order: for each cavity its photon number then its atom bits, then extras."""
    radix, counted, kind = [], [], []
    photon_digit, atom_digit, atom_cavity, extra_digit = [], [], [], []
    for c in range(model["n_cavities"]):
        photon_digit.append(len(radix))
        radix.append(model["n_max"][c] + 1)
        counted.append(True)
        kind.append("photon")
        for _ in range(model["atoms_per_cavity"][c]):
            atom_digit.append(len(radix))
            atom_cavity.append(c)
            radix.append(2)
            counted.append(True)
            kind.append("atom")
    for _ in range(model["n_extra"]):
        extra_digit.append(len(radix))
        radix.append(2)
        counted.append(False)
        kind.append("extra")
    return dict(radix=radix, counted=counted, kind=kind, photon_digit=photon_digit,
                atom_digit=atom_digit, atom_cavity=atom_cavity, extra_digit=extra_digit)


def _sort_lex(rows):
    """Sort digit rows in mixed-radix order (first digit most significant)."""
    if len(rows) == 0:
        return rows
    keys = tuple(rows[:, i] for i in reversed(range(rows.shape[1])))
    return rows[np.lexsort(keys)]


def _sector(layout, e):
    """All states with exactly e excitations (photons + atom bits), any extra digits."""
    radix, counted = layout["radix"], layout["counted"]
    n = len(radix)
    pos = [i for i in range(n) if counted[i] and radix[i] > 1]
    extras = [i for i in range(n) if not counted[i]]
    rows = []
    for combo in itertools.combinations_with_replacement(pos, e):
        d = np.zeros(n, dtype=np.int64)
        for p in combo:
            d[p] += 1
        if any(d[p] >= radix[p] for p in combo):
            continue
        for ex in itertools.product(*[range(radix[i]) for i in extras]):
            r = d.copy()
            r[extras] = ex
            rows.append(r)
    return _sort_lex(np.array(rows, dtype=np.int64).reshape(-1, n))


def _max_excitations(layout):
    return sum(r - 1 for r, c in zip(layout["radix"], layout["counted"]) if c)


def enumerate_basis(model):
    """The basis of the model as a `Basis` (five kinds, see qed_workloads)."""
    lay = digit_layout(model)
    radix = lay["radix"]
    kind = model["basis_kind"]
    n = len(radix)
    if kind == 0:
        rows = np.array(list(itertools.product(*[range(r) for r in radix])),
                        dtype=np.int64).reshape(-1, n)
    elif kind == 1:
        cap = model["excitation_cap"]
        rows = _sort_lex(np.concatenate([_sector(lay, e) for e in range(cap + 1)]))
    elif kind == 2:
        if model["n_extra"]:
            raise ValueError("ground + single-excitation basis takes no extra digits")
        rows = [np.zeros(n, dtype=np.int64)]
        atom = 0
        for c in range(model["n_cavities"]):
            if model["n_max"][c] >= 1:
                r = np.zeros(n, dtype=np.int64)
                r[lay["photon_digit"][c]] = 1
                rows.append(r)
            for _ in range(model["atoms_per_cavity"][c]):
                r = np.zeros(n, dtype=np.int64)
                r[lay["atom_digit"][atom]] = 1
                rows.append(r)
                atom += 1
        rows = np.array(rows)
    elif kind == 3:
        need = model["dim_cap"]
        parts, have = [], 0
        for e in range(_max_excitations(lay) + 1):
            s = _sector(lay, e)
            parts.append(s)
            have += len(s)
            if have >= need:
                break
        rows = np.concatenate(parts)
        if len(rows) < need:
            raise ValueError("dim_cap exceeds the product space")
        rows = rows[:need]
    elif kind == 4:
        rows = _sector(lay, model["excitation_cap"])
    else:
        raise ValueError(f"unknown basis kind {kind}")
    return Basis(model, rows)


def initial_index(model, basis):
    """Index of the pure initial basis state described by model['init']."""
    d = np.zeros(len(basis.layout["radix"]), dtype=np.int64)
    for c, v in model["init"].get("photons", {}).items():
        d[basis.photon_digit(int(c))] = v
    for a, v in model["init"].get("atoms", {}).items():
        d[basis.atom_digit(int(a))] = v
    for x, v in model["init"].get("extra", {}).items():
        d[basis.extra_digit(int(x))] = v
    k = basis.find(d)
    if k < 0:
        raise ValueError("initial state outside the basis")
    return k


def initial_density(model, basis):
    k = initial_index(model, basis)
    rho = np.zeros((basis.dim, basis.dim), dtype=np.complex128)
    rho[k, k] = 1.0
    return rho


# ------------------------------------------------------------------ operators
def _apply_terms(m, basis, digits):
    """Yield (target_digits, unit_amplitude, coefficient, param) for the terms of H
    applied to one basis state; the matrix element is coefficient * unit_amplitude.

    param is None for the diagonal, ('g', a) for an atom coupling, ('zeta', b) for a
    hop and ('tunnel', x) for an extra-digit flip (so dH/dparam is unit_amplitude)."""
    lay = basis.layout
    energy = 0.0
    for c in range(m["n_cavities"]):
        energy += m["omega_c"] * digits[lay["photon_digit"][c]]
    for a in range(len(lay["atom_digit"])):
        energy += m["omega_a"] * digits[lay["atom_digit"][a]]
    yield digits.copy(), energy, 1.0, None
    for a, g in enumerate(m["g"]):
        pa = lay["photon_digit"][lay["atom_cavity"][a]]
        sa = lay["atom_digit"][a]
        n = digits[pa]
        nmax = lay["radix"][pa] - 1
        if digits[sa] == 1 and n < nmax:          # a^+ sigma: atom emits into cavity
            t = digits.copy(); t[sa] = 0; t[pa] = n + 1
            yield t, np.sqrt(n + 1.0), g, ("g", a)
        if digits[sa] == 0 and n >= 1:            # a sigma^+: atom absorbs a photon
            t = digits.copy(); t[sa] = 1; t[pa] = n - 1
            yield t, np.sqrt(float(n)), g, ("g", a)
    for b, ((i, j), z) in enumerate(zip(m["bonds"], m["zeta"])):
        pi, pj = lay["photon_digit"][i], lay["photon_digit"][j]
        ni, nj = digits[pi], digits[pj]
        if nj >= 1 and ni < lay["radix"][pi] - 1:   # a_i^+ a_j
            t = digits.copy(); t[pi] = ni + 1; t[pj] = nj - 1
            yield t, np.sqrt((ni + 1.0) * nj), z, ("zeta", b)
        if ni >= 1 and nj < lay["radix"][pj] - 1:   # a_i a_j^+
            t = digits.copy(); t[pi] = ni - 1; t[pj] = nj + 1
            yield t, np.sqrt(ni * (nj + 1.0)), z, ("zeta", b)
    for x, t_x in enumerate(m["extra_tunnel"]):
        px = lay["extra_digit"][x]
        t = digits.copy(); t[px] = 1 - digits[px]
        yield t, 1.0, t_x, ("tunnel", x)


def hamiltonian(model, basis=None, param=None):
    """Dense H projected on the basis (complex128).  With param=('g', a), ('zeta', b)
    or ('tunnel', x) returns dH/dparam instead."""
    basis = basis or enumerate_basis(model)
    D = basis.dim
    H = np.zeros((D, D), dtype=np.complex128)
    for k in range(D):
        for t, unit, coef, p in _apply_terms(model, basis, basis.digits[k]):
            if param is not None and p != param:
                continue
            j = basis.find(t)
            if j >= 0:
                H[j, k] += unit if param is not None else coef * unit
    return H


def hamiltonian_derivative_entries(model, basis=None):
    """{param: [(row, col, unit_amplitude), ...]}: the entries of dH/dparam for every
    parameter at once (the same terms as hamiltonian(model, basis, param), collected in one
    pass over the basis)."""
    basis = basis or enumerate_basis(model)
    ent = {}
    for k in range(basis.dim):
        for t, unit, coef, p in _apply_terms(model, basis, basis.digits[k]):
            if p is None:
                continue
            j = basis.find(t)
            if j >= 0:
                ent.setdefault(p, []).append((j, k, unit))
    return ent


def jump_operator(model, basis, kind, site):
    """A_j projected on the basis (PAP) as a scipy.sparse CSR matrix."""
    lay = basis.layout
    D = basis.dim
    rows, cols, vals = [], [], []

    def put(target, k, v):
        j = basis.find(target)
        if j >= 0:
            rows.append(j); cols.append(k); vals.append(v)

    for k in range(D):
        d = basis.digits[k]
        if kind == JUMP_A:
            p = lay["photon_digit"][site]
            if d[p] >= 1:
                t = d.copy(); t[p] -= 1
                put(t, k, np.sqrt(float(d[p])))
        elif kind == JUMP_SIGMA:
            p = lay["atom_digit"][site]
            if d[p] == 1:
                t = d.copy(); t[p] = 0
                put(t, k, 1.0)
        elif kind == JUMP_DEPHASE:
            p = lay["extra_digit"][site]
            rows.append(k); cols.append(k); vals.append(1.0 if d[p] == 1 else -1.0)
        elif kind == JUMP_LEAK:
            p = lay["photon_digit"][site]
            if d[p] == 1 and int(np.sum(d)) == 1:
                put(np.zeros_like(d), k, 1.0)
        else:
            raise ValueError(f"unknown jump kind {kind}")
    return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(D, D))


def jump_operators(model, basis):
    """[(gamma_j, A_j)] with A_j as a scipy.sparse CSR matrix (products with dense rho
    are then plain sparse-dense matrix products)."""
    return [(float(g), jump_operator(model, basis, int(k), int(s))) for k, s, g in model["jumps"]]


def _dense(A):
    return A.toarray() if sp.issparse(A) else np.asarray(A)


# ------------------------------------------------------------------ dynamics
def propagator(H, dt):
    """U = exp(-i H dt) by the eigendecomposition of the Hermitian H."""
    lam, Q = np.linalg.eigh(H)
    return (Q * np.exp(-1j * lam * dt)) @ Q.conj().T


def _add_sandwich(out, gamma, A, X):
    """out += gamma A X A^+ for a sparse A, computed on the rows where A has entries."""
    rows = np.flatnonzero(np.diff(A.indptr))
    if len(rows) == 0:
        return
    Ar = A[rows, :]
    T = Ar @ X                                    # (A X) restricted to those rows
    out[np.ix_(rows, rows)] += gamma * (Ar @ T.conj().T).conj().T


def lindblad(V, jumps):
    """Eq. (3): sum_j gamma_j (A_j V A_j^+ - 1/2 (A_j^+A_j V + V A_j^+A_j)); the
    anticommutator terms are summed as K = sum_j gamma_j A_j^+A_j (linearity)."""
    out = np.zeros_like(V)
    K = None
    for gamma, A in jumps:
        _add_sandwich(out, gamma, A, V)
        AdA = gamma * (A.conj().T @ A)
        K = AdA if K is None else K + AdA
    if K is not None:
        KV = K @ V
        out -= 0.5 * (KV + KV.conj().T) if _is_hermitian(V) else 0.5 * (KV + (K @ V.conj().T).conj().T)
    return out


def _is_hermitian(X):
    return X.shape[0] == X.shape[1] and np.array_equal(X, X.conj().T)


def lindblad_adjoint(X, jumps):
    """Hilbert-Schmidt adjoint of Eq. (3): sum_j gamma_j (A^+ X A - 1/2 {A^+A, X})."""
    out = np.zeros_like(X)
    K = None
    for gamma, A in jumps:
        Ad = sp.csr_matrix(A.conj().T)
        _add_sandwich(out, gamma, Ad, X)
        AdA = gamma * (A.conj().T @ A)
        K = AdA if K is None else K + AdA
    if K is not None:
        out -= 0.5 * (K @ X + (K @ X.conj().T).conj().T)
    return out


def step(rho, U, jumps, dt):
    """One step: unitary evolution, then one Euler step of the Lindblad term."""
    V = U @ rho @ U.conj().T
    return V + dt * lindblad(V, jumps)


def lindblad_midpoint(X, jumps, tau):
    """tau of the Lindblad flow dX/dt = L(X) (Eq. 3) by the explicit midpoint rule,
    X + tau L(X + tau/2 L(X)); for the linear L this is X + tau L X + tau^2/2 L^2 X."""
    return X + tau * lindblad(X + 0.5 * tau * lindblad(X, jumps), jumps)


def step_strang(rho, U, jumps, dt):
    """One symmetric step of the two stages (Lindblad term, unitary evolution): half a
    Lindblad step, U . U^+, half a Lindblad step, the halves by the explicit midpoint
    rule.  Second order in dt."""
    X = lindblad_midpoint(rho, jumps, 0.5 * dt)
    V = U @ X @ U.conj().T
    return lindblad_midpoint(V, jumps, 0.5 * dt)


def effective_propagator(H, jumps, dt):
    """U_eff = exp(-i dt H_eff), H_eff = H - (i/2) sum_j gamma_j A_j^+ A_j: the anticommutator
    of Eq. (3) folded into a non-Hermitian generator together with the commutator of Eq. (2).
    H_eff is not Hermitian, so the exponential is scipy's expm (not an eigendecomposition)."""
    K = np.zeros_like(H, dtype=np.complex128)
    for gamma, A in jumps:
        K += gamma * _dense(A.conj().T @ A)
    return sla.expm(-1j * dt * (np.asarray(H, dtype=np.complex128) - 0.5j * K))


def step_effective(rho, U, jumps, dt):
    """One step of Eq. (3) regrouped: V = U_eff rho U_eff^+ carries the Hamiltonian and the
    anticommutator part exactly (U is the effective propagator), then one Euler step of the
    jump terms, V + dt sum_j gamma_j A_j V A_j^+.  First order in dt, completely positive,
    trace kept to O(dt^2) per step."""
    V = U @ rho @ U.conj().T
    out = V.copy()
    for gamma, A in jumps:
        _add_sandwich(out, dt * gamma, A, V)
    return out


STEPS = {"lie": step, "strang": step_strang, "effective": step_effective}


def observable_weights(model, basis):
    """Diagonal observables: trace, photon number per cavity, atom excitation per atom,
    extra digit per extra DOF (in that order)."""
    lay = basis.layout
    D = basis.dim
    w = [np.ones(D)]
    w += [basis.digits[:, p].astype(float) for p in lay["photon_digit"]]
    w += [basis.digits[:, p].astype(float) for p in lay["atom_digit"]]
    w += [basis.digits[:, p].astype(float) for p in lay["extra_digit"]]
    return np.array(w).reshape(-1, D)


def observables(rho, weights, obs_ids):
    """Population rho_kk for id < D, else tr(W_{id-D} rho) for the diagonal weights."""
    D = rho.shape[0]
    p = np.real(np.diag(rho))
    out = []
    for i in obs_ids:
        out.append(p[i] if i < D else float(weights[i - D] @ p))
    return np.array(out)


def evolve(model, rho0=None, n_steps=None, record_every=None, obs_ids=None, U=None,
           basis=None, return_records=True, scheme="lie"):
    """Integrate n_steps with the step of `scheme` ('lie', 'strang' or 'effective', whose U
    is the effective propagator); record observables at steps 0, r, 2r, ... (<= n_steps)."""
    advance = STEPS[scheme]
    basis = basis or enumerate_basis(model)
    H = hamiltonian(model, basis)
    dt = model["dt"]
    jumps = jump_operators(model, basis)
    if U is None:
        U = effective_propagator(H, jumps, dt) if scheme == "effective" else propagator(H, dt)
    rho = initial_density(model, basis) if rho0 is None else np.array(rho0, dtype=np.complex128)
    n_steps = model["n_steps"] if n_steps is None else n_steps
    r = record_every or model["record_every"]
    obs_ids = list(range(basis.dim)) if obs_ids is None else list(obs_ids)
    W = observable_weights(model, basis)
    records = []
    for n in range(n_steps + 1):
        if n % r == 0:
            records.append(observables(rho, W, obs_ids))
        if n < n_steps:
            rho = advance(rho, U, jumps, dt)
    if return_records:
        return rho, np.array(records)
    return rho


# ------------------------------------------------------------------ state selection
def select_states(model, eps, steps_per_round, n_rounds, rho0=None, basis=None, scheme="lie"):
    """The state space selection of Sec. 3.2: rounds of {solve the QME for T =
    steps_per_round * dt; growth speed of each state's probability,
    |p_k(t + T) - p_k(t)| / T; delete every state whose growth speed is below eps;
    normalise the density matrix of the remaining states}.  H and the A_j of the remaining
    states are the projections P H P and P A_j P onto them.

    Reading: taken literally a populated state whose probability happens to stay constant
    would be deleted; a state whose probability is at least eps is kept.

    Returns (kept indices into the original basis, final rho on them, sizes after each
    round)."""
    basis = basis or enumerate_basis(model)
    dt = model["dt"]
    H = hamiltonian(model, basis)
    jumps = jump_operators(model, basis)
    advance = STEPS[scheme]
    keep = np.arange(basis.dim)
    rho = initial_density(model, basis) if rho0 is None else np.array(rho0, dtype=np.complex128)
    T = steps_per_round * dt
    sizes = []
    for _ in range(n_rounds):
        Hs = H[np.ix_(keep, keep)]
        Us = propagator(Hs, dt)
        js = [(g, sp.csr_matrix(A[keep][:, keep])) for g, A in jumps]
        p0 = np.real(np.diag(rho)).copy()
        for _ in range(steps_per_round):
            rho = advance(rho, Us, js, dt)
        p1 = np.real(np.diag(rho))
        growth = np.abs(p1 - p0) / T
        local = np.flatnonzero((growth >= eps) | (p1 >= eps))
        if len(local) == 0:
            raise ValueError("every state fell below eps")
        rho = rho[np.ix_(local, local)]
        rho = 0.5 * (rho + rho.conj().T) / np.trace(rho).real
        keep = keep[local]
        sizes.append(len(keep))
    return keep, rho, sizes


# ------------------------------------------------------------------ brute force# ------------------------------------------------------------------ brute force
def vec(X):
    """Column-stacking vectorisation."""
    return np.asarray(X).reshape(-1, order="F")


def unvec(v, D):
    return np.asarray(v).reshape(D, D, order="F")


def liouvillian(H, jumps):
    """Superoperator of Eq. (2) with Eq. (3), using vec(A X B) = (B^T kron A) vec X."""
    D = H.shape[0]
    I = np.eye(D)
    L = -1j * (np.kron(I, H) - np.kron(H.T, I))
    for gamma, A in jumps:
        A = _dense(A)
        AdA = A.conj().T @ A
        L = L + gamma * (np.kron(A.conj(), A) - 0.5 * np.kron(I, AdA) - 0.5 * np.kron(AdA.T, I))
    return L


def discrete_superoperator(U, jumps, dt):
    """S = (I + dt * D)(conj(U) kron U), the one-step map of `step` in Liouville space."""
    D = U.shape[0]
    I = np.eye(D)
    Dis = np.zeros((D * D, D * D), dtype=np.complex128)
    for gamma, A in jumps:
        A = _dense(A)
        AdA = A.conj().T @ A
        Dis += gamma * (np.kron(A.conj(), A) - 0.5 * np.kron(I, AdA) - 0.5 * np.kron(AdA.T, I))
    return (np.eye(D * D) + dt * Dis) @ np.kron(U.conj(), U)


def matrix_power_by_squaring(S, n):
    result = np.eye(S.shape[0], dtype=S.dtype)
    base = S.copy()
    while n:
        if n & 1:
            result = result @ base
        base = base @ base
        n >>= 1
    return result


def continuum(model, t, rho0=None, basis=None):
    """rho(t) = exp(L t) rho0 for the continuous QME (dense expm of the Liouvillian)."""
    basis = basis or enumerate_basis(model)
    H = hamiltonian(model, basis)
    jumps = jump_operators(model, basis)
    rho0 = initial_density(model, basis) if rho0 is None else rho0
    L = liouvillian(H, jumps)
    return unvec(sla.expm(L * t) @ vec(rho0), basis.dim)


# ------------------------------------------------------------------ Kronecker form
def kron_operators(model):
    """H and A_j on the FULL product space from Kronecker products of single-digit
    operators (a textbook construction kept apart from `hamiltonian`); for tests."""
    lay = digit_layout(model)
    radix = lay["radix"]

    def embed(ops):
        out = np.ones((1, 1), dtype=np.complex128)
        for i, r in enumerate(radix):
            out = np.kron(out, ops.get(i, np.eye(r)))
        return out

    def lower(r):
        return np.diag(np.sqrt(np.arange(1, r, dtype=float)), k=1).astype(np.complex128)

    full = int(np.prod(radix))
    H = np.zeros((full, full), dtype=np.complex128)
    for c in range(model["n_cavities"]):
        p = lay["photon_digit"][c]
        a = lower(radix[p])
        H += model["omega_c"] * embed({p: a.conj().T @ a})
    for at in range(len(lay["atom_digit"])):
        s = lay["atom_digit"][at]
        sm = lower(2)
        H += model["omega_a"] * embed({s: sm.conj().T @ sm})
        p = lay["photon_digit"][lay["atom_cavity"][at]]
        a = lower(radix[p])
        term = embed({p: a.conj().T, s: sm})
        H += model["g"][at] * (term + term.conj().T)
    for (i, j), z in zip(model["bonds"], model["zeta"]):
        pi, pj = lay["photon_digit"][i], lay["photon_digit"][j]
        term = embed({pi: lower(radix[pi]).conj().T, pj: lower(radix[pj])})
        H += z * (term + term.conj().T)
    for x, t in enumerate(model["extra_tunnel"]):
        px = lay["extra_digit"][x]
        H += t * embed({px: np.array([[0, 1], [1, 0]], dtype=np.complex128)})
    jumps = []
    for kind, site, gamma in model["jumps"]:
        if kind == JUMP_A:
            p = lay["photon_digit"][site]
            A = embed({p: lower(radix[p])})
        elif kind == JUMP_SIGMA:
            A = embed({lay["atom_digit"][site]: lower(2)})
        elif kind == JUMP_DEPHASE:
            A = embed({lay["extra_digit"][site]: np.diag([-1.0, 1.0]).astype(np.complex128)})
        elif kind == JUMP_LEAK:
            vac = np.zeros(full); vac[0] = 1.0
            one = np.zeros(full)
            idx = [0] * len(radix)
            idx[lay["photon_digit"][site]] = 1
            one[np.ravel_multi_index(idx, radix)] = 1.0
            A = np.outer(vac, one).astype(np.complex128)
        jumps.append((gamma, A))
    return H, jumps


def full_product_rows(model):
    """Flat product-space index of each basis row (mixed radix, first digit slowest)."""
    basis = enumerate_basis(model)
    radix = basis.layout["radix"]
    return np.ravel_multi_index(tuple(basis.digits.T), radix), basis


# ------------------------------------------------------------------ gradients
def _trace_dissipator(lam, V, A):
    """tr(lam D_A(V)) with D_A(V) = A V A^+ - 1/2 (A^+A V + V A^+A) (Eq. 3, one jump, unit
    rate), for a sparse A without forming D x D intermediates:
      tr(lam A V A^+) = sum over k, l in R of lam[l, k] (A V A^+)[k, l], R the rows where A
      has entries (A V A^+ vanishes outside R x R);
      tr(lam (K V + V K)) = sum over the entries K[m, j] of K[m, j] ((V lam)[j, m] +
      (lam V)[j, m]), K = A^+A."""
    rows = np.flatnonzero(np.diff(A.indptr))
    if len(rows) == 0:
        return 0.0
    Ar = A[rows, :]
    S = (Ar @ (Ar @ V).conj().T).conj().T          # (A V A^+) on R x R
    sandwich = np.sum(lam[np.ix_(rows, rows)].T * S)
    K = (A.conj().T @ A).tocoo()
    vl = np.einsum("ei,ie->e", V[K.col, :], lam[:, K.row])
    lv = np.einsum("ei,ie->e", lam[K.col, :], V[:, K.row])
    return sandwich - 0.5 * np.sum(K.data * (vl + lv))


def _lindblad_midpoint_adjoint(Lam, jumps, tau):
    """The Hilbert-Schmidt adjoint of lindblad_midpoint: Lam + tau L^+(T) with the stage
    T = Lam + tau/2 L^+(Lam); returns (result, T)."""
    T = Lam + 0.5 * tau * lindblad_adjoint(Lam, jumps)
    return Lam + tau * lindblad_adjoint(T, jumps), T


def _midpoint_rate_traces(Lam, T, Y, jumps, tau):
    """d/dgamma_j of tr(Lam E(Y)) for the midpoint step E(Y) = Y + tau L Y + tau^2/2 L^2 Y,
    L = sum_j gamma_j D_j: tr(Lam (tau D_j Y + tau^2/2 (D_j L Y + L D_j Y)))
    = tau tr(T D_j(Y)) + tau^2/2 tr(Lam D_j(L Y)), T = Lam + tau/2 L^+(Lam)."""
    LY = lindblad(Y, jumps)
    return np.array([np.real(tau * _trace_dissipator(T, Y, A) + 0.5 * tau * tau * _trace_dissipator(Lam, LY, A))
                     for _, A in jumps])


def adjoint_gradients(model, obs_diag, n_steps=None, rho0=None, basis=None, scheme="lie"):
    """Discrete adjoint of L = tr(diag(obs) rho_N) through the map of `step`.

    lambda_N = O; lambda'_{n+1} = J^+(lambda_{n+1}) with J(V) = V + dt L(V);
    lambda_n = U^+ lambda'_{n+1} U.
    dL/dgamma_j = dt * sum_n tr(lambda_{n+1} D_j(V_n)),
    dL/dtheta   = 2 Re sum_n tr(lambda'_{n+1} (dU/dtheta) rho_n U^+), with dU/dtheta from
    the Daleckii-Krein divided differences of exp(-i lambda dt) in H's eigenbasis.

    scheme="strang": the map of step_strang, X_n = E(rho_n), V_n = U X_n U^+,
    rho_{n+1} = E(V_n) with the midpoint half step E (tau = dt/2): kappa_n = E^+(lambda_{n+1}),
    mu_n = U^+ kappa_n U, lambda_n = E^+(mu_n); M = sum_n X_n U^+ kappa_n; the rate gradients
    differentiate both half steps (_midpoint_rate_traces).
    Returns (loss, grad_g, grad_zeta, grad_gamma)."""
    if scheme == "strang":
        return _adjoint_gradients_strang(model, obs_diag, n_steps, rho0, basis)
    basis = basis or enumerate_basis(model)
    H = hamiltonian(model, basis)
    dt = model["dt"]
    n_steps = model["n_steps"] if n_steps is None else n_steps
    lam, Q = np.linalg.eigh(H)
    f = np.exp(-1j * lam * dt)
    U = (Q * f) @ Q.conj().T
    jumps = jump_operators(model, basis)
    rho = initial_density(model, basis) if rho0 is None else np.array(rho0, dtype=np.complex128)
    rhos = [rho]
    for _ in range(n_steps):
        rho = step(rho, U, jumps, dt)
        rhos.append(rho)
    O = np.diag(np.asarray(obs_diag, dtype=float)).astype(np.complex128)
    loss = float(np.real(np.trace(O @ rhos[-1])))
    lam_next = O
    M = np.zeros_like(H)
    grad_gamma = np.zeros(len(jumps))
    for n in reversed(range(n_steps)):
        V = U @ rhos[n] @ U.conj().T
        for j, (gamma, A) in enumerate(jumps):
            grad_gamma[j] += dt * np.real(_trace_dissipator(lam_next, V, A))
        lam_prime = lam_next + dt * lindblad_adjoint(lam_next, jumps)
        M += rhos[n] @ U.conj().T @ lam_prime
        lam_next = U.conj().T @ lam_prime @ U
    grad_g, grad_zeta = _hamiltonian_gradients(model, basis, lam, Q, f, dt, M)
    return loss, grad_g, grad_zeta, grad_gamma


def _hamiltonian_gradients(model, basis, lam, Q, f, dt, M):
    """dL/dtheta = 2 Re tr(dU/dtheta M) for every g and zeta, dU/dtheta by the
    Daleckii-Krein divided differences of f(x) = exp(-i x dt) at H's eigenvalues lam
    (eigenvectors Q, f = f(lam))."""
    # divided differences F_kl of f(x) = exp(-i x dt) at the eigenvalues
    dl = lam[:, None] - lam[None, :]
    same = np.abs(dl) < 1e-13 * max(1.0, float(np.max(np.abs(lam))))
    F = np.where(same, -1j * dt * f[:, None], (f[:, None] - f[None, :]) / np.where(same, 1.0, dl))
    Mt = Q.conj().T @ M @ Q
    K = Q @ (F.T * Mt) @ Q.conj().T   # tr(dU M) = tr(dH K)
    # tr(dH/dtheta K) = sum over the entries (j, k, u) of dH/dtheta of u K[k, j]
    ent = hamiltonian_derivative_entries(model, basis)

    def contract(p):
        return 2.0 * np.real(sum(u * K[k, j] for j, k, u in ent.get(p, [])))

    grad_g = np.array([contract(("g", a)) for a in range(len(model["g"]))])
    grad_zeta = np.array([contract(("zeta", b)) for b in range(len(model["zeta"]))])
    return grad_g, grad_zeta


def _adjoint_gradients_strang(model, obs_diag, n_steps, rho0, basis):
    basis = basis or enumerate_basis(model)
    H = hamiltonian(model, basis)
    dt = model["dt"]
    tau = 0.5 * dt
    n_steps = model["n_steps"] if n_steps is None else n_steps
    lam, Q = np.linalg.eigh(H)
    f = np.exp(-1j * lam * dt)
    U = (Q * f) @ Q.conj().T
    jumps = jump_operators(model, basis)
    rho = initial_density(model, basis) if rho0 is None else np.array(rho0, dtype=np.complex128)
    rhos = [rho]
    for _ in range(n_steps):
        rho = step_strang(rho, U, jumps, dt)
        rhos.append(rho)
    O = np.diag(np.asarray(obs_diag, dtype=float)).astype(np.complex128)
    loss = float(np.real(np.trace(O @ rhos[-1])))
    lam_next = O
    M = np.zeros_like(H)
    grad_gamma = np.zeros(len(jumps))
    for n in reversed(range(n_steps)):
        X = lindblad_midpoint(rhos[n], jumps, tau)
        V = U @ X @ U.conj().T
        kappa, T1 = _lindblad_midpoint_adjoint(lam_next, jumps, tau)
        grad_gamma += _midpoint_rate_traces(lam_next, T1, V, jumps, tau)
        M += X @ U.conj().T @ kappa
        mu = U.conj().T @ kappa @ U
        lam_next, T2 = _lindblad_midpoint_adjoint(mu, jumps, tau)
        grad_gamma += _midpoint_rate_traces(mu, T2, rhos[n], jumps, tau)
    grad_g, grad_zeta = _hamiltonian_gradients(model, basis, lam, Q, f, dt, M)
    return loss, grad_g, grad_zeta, grad_gamma


def loss_diag(model, basis, photons=(), atoms=()):
    """Diagonal loss weights: population of the listed single photons / atoms."""
    w = np.zeros(basis.dim)
    for c in photons:
        d = np.zeros(len(basis.layout["radix"]), dtype=np.int64)
        d[basis.photon_digit(c)] = 1
        k = basis.find(d)
        if k >= 0:
            w[k] = 1.0
    for a in atoms:
        d = np.zeros(len(basis.layout["radix"]), dtype=np.int64)
        d[basis.atom_digit(a)] = 1
        k = basis.find(d)
        if k >= 0:
            w[k] = 1.0
    return w


def loss_value(model, obs_diag, params=None, n_steps=None, basis=None, scheme="lie"):
    """tr(diag(obs) rho_N) with some parameters overridden: used by finite differences."""
    m = dict(model)
    if params:
        for (name, i), v in params.items():
            key = {"g": "g", "zeta": "zeta"}[name]
            arr = list(m[key])
            arr[i] = v
            m[key] = arr
    rho = evolve(m, n_steps=n_steps, basis=basis, return_records=False, scheme=scheme)
    return float(np.real(np.sum(np.asarray(obs_diag) * np.diag(rho))))
