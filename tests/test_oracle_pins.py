"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares it with a closed form, a
number the paper prints, a differently built operator (Kronecker products), brute force
in Liouville space, an invariant, or finite differences.
"""
import json
import os

import numpy as np
import pytest

import oracle
import qed_workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_model(spec):
    if "lattice" in spec:
        L, Wd = spec["lattice"]
        m = W.lattice(L, Wd, gamma=0.0, atoms=spec.get("atoms", True),
                      basis_kind=spec["basis_kind"], start=(0, 0))
        m["excitation_cap"] = spec.get("excitation_cap", 0)
        return m
    m = W._model(**spec)
    n_atoms = sum(m["atoms_per_cavity"])
    m["g"] = [0.01] * n_atoms
    m["extra_tunnel"] = [0.0] * m["n_extra"]
    return m


# ---------------------------------------------------------------- dimensions / basis
def test_paper_dimensions():
    """Dimensions printed in the paper (Eq. 6, Eq. 9, Table 1, Sec. 4.2, Eqs. 10-11)."""
    with open(os.path.join(GOLDEN, "paper_dimensions.json")) as f:
        entries = json.load(f)["entries"]
    for e in entries:
        b = oracle.enumerate_basis(_golden_model(e["model"]))
        assert b.dim == e["dim"], e["what"]


def test_workload_dimensions():
    """The workload sizes: 36, (4*4)^2*2 = 512, 2*1024+1 = 2049, 2*576+1 = 1153."""
    assert oracle.enumerate_basis(W.jch_two_cavities()).dim == 36
    assert oracle.enumerate_basis(W.hb_shaped()).dim == 512
    assert oracle.enumerate_basis(W.lattice()).dim == 2049
    assert oracle.enumerate_basis(W.adjoint_lattice()).dim == 1153


def test_basis_order_mixed_radix():
    """Full product order: index = ((n1*2+s1)*3+n2)*2+s2 for two cavities, one atom each."""
    b = oracle.enumerate_basis(W.jch_two_cavities())
    for k, (n1, s1, n2, s2) in enumerate(b.digits):
        assert k == ((n1 * 2 + s1) * 3 + n2) * 2 + s2


def test_sector_bases_against_filtering():
    """Kinds 1, 3 and 4 equal a filter / stable sort of the full product basis."""
    m = W.chain_instance(np.random.default_rng(3), 32, 200)
    m.update(n_cavities=3, atoms_per_cavity=[2, 1, 2], n_max=[2, 1, 3], g=[0.01] * 5,
             bonds=[(0, 1), (1, 2)], zeta=[0.004, 0.006], jumps=[])
    full = m | {"basis_kind": 0}
    fb = oracle.enumerate_basis(full)
    exc = fb.digits.sum(axis=1)
    # kind 1: excitations <= cap, mixed-radix order
    b1 = oracle.enumerate_basis(m | {"basis_kind": 1, "excitation_cap": 3})
    assert np.array_equal(b1.digits, fb.digits[exc <= 3])
    # kind 4: exactly cap
    b4 = oracle.enumerate_basis(m | {"basis_kind": 4, "excitation_cap": 2})
    assert np.array_equal(b4.digits, fb.digits[exc == 2])
    # kind 3: first D after a stable sort by excitation number
    order = np.argsort(exc, kind="stable")
    for D in (1, 7, 40, 111):
        b3 = oracle.enumerate_basis(m | {"basis_kind": 3, "dim_cap": D})
        assert np.array_equal(b3.digits, fb.digits[order[:D]])


def test_single_excitation_layout():
    """Kind 2: index 0 is the vacuum, 1 + 2c the photon in cavity c, 2 + 2c its atom."""
    m = W.lattice(4, 3, gamma=0.0)
    b = oracle.enumerate_basis(m)
    assert b.dim == 25
    assert b.digits[0].sum() == 0
    for c in range(12):
        assert b.digits[1 + 2 * c][b.photon_digit(c)] == 1 and b.digits[1 + 2 * c].sum() == 1
        assert b.digits[2 + 2 * c][b.atom_digit(c)] == 1 and b.digits[2 + 2 * c].sum() == 1


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("make", [
    lambda: W.jch_two_cavities(),
    lambda: W.hb_shaped(),
    lambda: W.lattice(2, 2, gamma=1e-3, seed=1),
    lambda: W._model(n_cavities=3, atoms_per_cavity=[2, 1, 2], n_max=[1, 2, 1], basis_kind=3,
                     dim_cap=60, g=[0.011, 0.012, 0.013, 0.014, 0.015], bonds=[(0, 1), (1, 2)],
                     zeta=[0.004, 0.006], jumps=[(0, 0, 1e-3), (0, 2, 2e-3), (1, 3, 3e-3)]),
])
def test_operators_equal_kronecker_construction(make):
    """H and every A_j equal P^T (Kronecker-product operator) P for the basis rows P."""
    m = make()
    rows, b = oracle.full_product_rows(m)
    Hk, jk = oracle.kron_operators(m)
    H = oracle.hamiltonian(m, b)
    Hp = Hk[np.ix_(rows, rows)]
    assert np.abs(H - Hp).max() < 1e-15
    for (g1, A1), (g2, A2) in zip(oracle.jump_operators(m, b), jk):
        assert g1 == g2
        assert np.abs(A1.toarray() - A2[np.ix_(rows, rows)]).max() < 1e-15


def test_hamiltonian_hermitian_and_real_couplings():
    for m in (W.jch_two_cavities(), W.hb_shaped(), W.lattice(5, 5, seed=2)):
        H = oracle.hamiltonian(m)
        assert np.abs(H - H.conj().T).max() == 0.0


def test_jch_single_excitation_spectrum():
    """Two cavities (hopping zeta), one resonant atom each (g): in the one-excitation
    sector the eigenvalues are omega +- zeta/2 +- sqrt(zeta^2/4 + g^2)."""
    g, z, w = 0.01, 0.005, 1.0
    m = W.jch_two_cavities(gamma=0.0, g=g, zeta=z)
    b = oracle.enumerate_basis(m)
    H = oracle.hamiltonian(m, b)
    one = np.where(b.digits.sum(axis=1) == 1)[0]
    ev = np.sort(np.linalg.eigvalsh(H[np.ix_(one, one)]))
    r = np.sqrt(z * z / 4 + g * g)
    want = np.sort([w + z / 2 + r, w + z / 2 - r, w - z / 2 + r, w - z / 2 - r])
    assert np.abs(ev - want).max() < 1e-15


def test_uniform_lattice_modes():
    """Lattice with uniform g: eigenvalues are those of [[omega + eps_k, g], [g, omega]]
    for the open-boundary tight-binding energies eps_k = 2 zeta (cos k_m + cos k_n)."""
    L, Wd, g, z = 4, 3, 0.01, 0.01
    m = W.lattice(L, Wd, g=g, zeta=z, gamma=0.0)
    b = oracle.enumerate_basis(m)
    H = oracle.hamiltonian(m, b)
    ev = np.sort(np.linalg.eigvalsh(H))
    eps = [2 * z * (np.cos(np.pi * p / (L + 1)) + np.cos(np.pi * q / (Wd + 1)))
           for p in range(1, L + 1) for q in range(1, Wd + 1)]
    want = [0.0]
    for e in eps:
        want += list(np.linalg.eigvalsh(np.array([[1.0 + e, g], [g, 1.0]])))
    assert np.abs(ev - np.sort(want)).max() < 1e-14


# ---------------------------------------------------------------- closed-form dynamics
@pytest.mark.parametrize("n", [0, 1, 2])
def test_rabi_oscillation(n):
    """Resonant JC from |e, n>: P_e(t) = cos^2(g sqrt(n+1) t) (frequency 2 g sqrt(n+1))."""
    g, dt, steps = 0.05, 0.1, 400
    m = W.jc_single(n_max=3, g=g, dt=dt, n_steps=steps, init_photons=n)
    b = oracle.enumerate_basis(m)
    atom_obs = b.dim + 1 + 1   # trace, photon number, then atom excitation
    _, rec = oracle.evolve(m, obs_ids=[atom_obs], basis=b)
    t = dt * np.arange(steps + 1)
    assert np.abs(rec[:, 0] - np.cos(g * np.sqrt(n + 1) * t) ** 2).max() < 1e-12


def test_tight_binding_closed_form():
    """g = 0 lattice: psi(i, j, t) = psi1(i, t) psi1(j, t) with open-boundary modes
    phi_m(i) = sqrt(2/(L+1)) sin(k_m (i+1)), k_m = pi m/(L+1), energy omega/2 + 2 zeta cos k_m
    per axis (the two halves of omega add up)."""
    L, Wd, z, dt, steps = 5, 4, 0.05, 0.1, 300
    i0, j0 = 1, 2
    m = W.lattice(L, Wd, g=0.0, zeta=z, gamma=0.0, dt=dt, n_steps=steps, start=(i0, j0))
    b = oracle.enumerate_basis(m)
    rho, _ = oracle.evolve(m, basis=b, obs_ids=[0])

    def psi1(n, x0, t):
        k = np.pi * np.arange(1, n + 1) / (n + 1)
        phi = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(np.arange(n) + 1, k))
        return phi @ (phi[x0] * np.exp(-1j * (0.5 + 2 * z * np.cos(k)) * t))

    t = dt * steps
    psi = np.outer(psi1(L, i0, t), psi1(Wd, j0, t)).reshape(-1)
    idx = [1 + 2 * c for c in range(L * Wd)]
    want = np.outer(psi, psi.conj())
    assert np.abs(rho[np.ix_(idx, idx)] - want).max() < 1e-12


def test_lattice_closed_form_with_atoms():
    """Uniform-g lattice, one excitation: each open-boundary hopping mode is a 2 x 2 JC
    block, giving the state in closed form (tests/closed_forms.py)."""
    from closed_forms import lattice_single_excitation_state
    m = W.lattice(5, 4, g=0.02, zeta=0.03, gamma=0.0, dt=0.1, n_steps=150, start=(1, 2))
    rho = oracle.evolve(m, return_records=False)
    psi = lattice_single_excitation_state(5, 4, 1.0, 0.02, 0.03, 15.0, (1, 2))
    assert np.abs(rho - np.outer(psi, psi.conj())).max() < 1e-12


def test_discrete_photon_decay():
    """H = omega a^+a, A = a: <n>_k = (1 - gamma dt)^k <n>_0 exactly for the scheme,
    because a^+ (a^+ a) a = n(n - 1) and the anticommutator removes 2n^2 gamma dt / 2."""
    gamma, dt, steps = 0.02, 0.1, 500
    m = W._model(n_cavities=1, atoms_per_cavity=[0], n_max=[6], jumps=[(0, 0, gamma)],
                 dt=dt, n_steps=steps, init={"photons": {0: 4}})
    b = oracle.enumerate_basis(m)
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    psi /= np.linalg.norm(psi)
    rho0 = np.outer(psi, psi.conj())
    _, rec = oracle.evolve(m, rho0=rho0, basis=b, obs_ids=[b.dim + 1])
    n0 = float(np.real(np.sum(np.arange(7) * np.diag(rho0))))
    want = n0 * (1 - gamma * dt) ** np.arange(steps + 1)
    assert np.abs(rec[:, 0] - want).max() < 1e-13
    # and the continuum exp(-gamma t) is within gamma^2 dt t / 2 (first-order scheme)
    t = dt * steps
    assert abs(rec[-1, 0] - n0 * np.exp(-gamma * t)) <= n0 * gamma ** 2 * dt * t


def test_atom_decay_and_dephasing_closed_forms():
    """sigma jump: P_e decays as (1 - gamma dt)^k; sigma_z dephasing: the coherence of the
    extra digit shrinks by (1 - 2 gamma dt) per step, populations unchanged."""
    ga, gp, dt, steps = 0.03, 0.05, 0.1, 200
    m = W._model(n_cavities=1, atoms_per_cavity=[1], n_max=[0], g=[0.0], n_extra=1,
                 extra_tunnel=[0.0], jumps=[(1, 0, ga), (2, 0, gp)], dt=dt, n_steps=steps,
                 omega_a=0.7, init={"atoms": {0: 1}})
    b = oracle.enumerate_basis(m)
    assert b.dim == 4
    psi_x = np.array([0.6, 0.8])
    psi = np.kron(np.array([0.0, 1.0]), psi_x)   # atom excited, extra digit in superposition
    rho0 = np.outer(psi, psi).astype(complex)
    rho, rec = oracle.evolve(m, rho0=rho0, basis=b, obs_ids=[b.dim + 2, b.dim + 3])
    k = np.arange(steps + 1)
    assert np.abs(rec[:, 0] - (1 - ga * dt) ** k).max() < 1e-14
    assert np.abs(rec[:, 1] - 0.64).max() < 1e-14
    # extra-digit coherence, summed over the atom states (partial trace)
    coh = rho[0, 1] + rho[2, 3]
    assert abs(abs(coh) - 0.48 * (1 - 2 * gp * dt) ** steps) < 1e-14


def test_leak_moves_population_to_vacuum():
    """|G><photon_c| leaks: with g = zeta = 0, the photon population decays as
    (1 - gamma dt)^k and the vacuum gains exactly what it loses."""
    m = W.lattice(2, 2, g=0.0, zeta=0.0, gamma=0.05, dt=0.1, n_steps=100, start=(1, 0))
    b = oracle.enumerate_basis(m)
    c0 = 1 * 2 + 0
    _, rec = oracle.evolve(m, basis=b, obs_ids=[0, 1 + 2 * c0], record_every=1)
    k = np.arange(101)
    assert np.abs(rec[:, 1] - (1 - 0.005) ** k).max() < 1e-14
    assert np.abs(rec[:, 0] + rec[:, 1] - 1.0).max() < 1e-14


# ---------------------------------------------------------------- brute force
def test_superoperator_power_matches_step_loop():
    """vec rho_n = S^n vec rho_0 with S = (I + dt D)(conj(U) kron U), built from
    Kronecker products, equals the matrix-form step loop (D = 36, n = 2000)."""
    m = W.jch_two_cavities(n_steps=2000, gamma=0.01)
    b = oracle.enumerate_basis(m)
    H = oracle.hamiltonian(m, b)
    U = oracle.propagator(H, m["dt"])
    jumps = oracle.jump_operators(m, b)
    rho0 = W.random_density(36, seed=1)
    rho_loop = oracle.evolve(m, rho0=rho0, basis=b, return_records=False)
    S = oracle.discrete_superoperator(U, jumps, m["dt"])
    rho_sup = oracle.unvec(oracle.matrix_power_by_squaring(S, 2000) @ oracle.vec(rho0), 36)
    assert np.abs(rho_loop - rho_sup).max() < 1e-12


def test_propagator_matches_expm_and_is_unitary():
    import scipy.linalg as sla
    for m in (W.jch_two_cavities(), W.hb_shaped()):
        H = oracle.hamiltonian(m)
        U = oracle.propagator(H, m["dt"])
        assert np.abs(U - sla.expm(-1j * H * m["dt"])).max() < 1e-14
        assert np.abs(U.conj().T @ U - np.eye(len(U))).max() < 1e-13


def test_first_order_convergence_to_continuum():
    """The split scheme converges to exp(L t) rho_0 at first order in dt."""
    m = W.jch_two_cavities(gamma=0.05)
    b = oracle.enumerate_basis(m)
    t = 20.0
    exact = oracle.continuum(m, t, basis=b)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        mm = dict(m, dt=dt, n_steps=int(round(t / dt)))
        rho = oracle.evolve(mm, basis=b, return_records=False)
        errs.append(np.abs(rho - exact).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.8 <= e1 / e2 <= 2.2


def test_liouvillian_generates_trace_and_hermiticity():
    m = W.hb_shaped()
    m.update(n_cavities=1, atoms_per_cavity=[2], n_max=[2], g=m["g"][:2], jumps=[(0, 0, 0.01), (2, 0, 0.02)])
    b = oracle.enumerate_basis(m)
    L = oracle.liouvillian(oracle.hamiltonian(m, b), oracle.jump_operators(m, b))
    D = b.dim
    # tr(L rho) = 0 for every rho: the row vec(I)^T L vanishes
    assert np.abs(oracle.vec(np.eye(D)) @ L).max() < 1e-14


# ---------------------------------------------------------------- invariants
def test_invariants_along_trajectory():
    m = W.hb_shaped(n_steps=300, record_every=50)
    b = oracle.enumerate_basis(m)
    H = oracle.hamiltonian(m, b)
    U = oracle.propagator(H, m["dt"])
    jumps = oracle.jump_operators(m, b)
    # The Euler step is rho' = (I - dt K/2) V (I - dt K/2) + dt sum gamma A V A^+ - dt^2/4 K V K
    # with K = sum gamma A^+A: only the last term can push a zero eigenvalue below zero.
    K = sum(g * (A.conj().T @ A).toarray() for g, A in jumps)
    neg = (m["dt"] * np.abs(np.linalg.eigvalsh(K)).max()) ** 2 / 4
    rho = W.random_density(b.dim, seed=2, rank=3)
    for k in range(101):
        rho = oracle.step(rho, U, jumps, m["dt"])
        if k % 25 == 0:
            assert abs(np.trace(rho).real - 1.0) < 1e-12
            assert np.abs(rho - rho.conj().T).max() < 1e-15
            assert np.linalg.eigvalsh(rho).min() > -(k + 1) * neg - 1e-15


def test_photon_number_conserved_when_closed():
    """Without jumps the excitation number (photons + atoms) is conserved (Sec. 4.2)."""
    m = W.jch_two_cavities(gamma=0.0, n_steps=500, record_every=100)
    b = oracle.enumerate_basis(m)
    ids = [b.dim + 1, b.dim + 2, b.dim + 3, b.dim + 4]
    _, rec = oracle.evolve(m, basis=b, obs_ids=ids)
    assert np.abs(rec.sum(axis=1) - 1.0).max() < 1e-13


def test_mirror_symmetry_of_symmetric_start():
    """Started on the mirror axis, P(i, j) = P(L-1-i, j) for all t (Sec. 4.2)."""
    L, Wd = 7, 4
    m = W.lattice(L, Wd, gamma=1e-3, n_steps=200, start=(3, 0))
    b = oracle.enumerate_basis(m)
    rho = oracle.evolve(m, basis=b, return_records=False)
    p = np.real(np.diag(rho))[1::2].reshape(L, Wd)
    assert np.abs(p - p[::-1, :]).max() < 1e-14
    # the asymmetric start breaks it
    m2 = W.lattice(L, Wd, gamma=1e-3, n_steps=200, start=(1, 0))
    p2 = np.real(np.diag(oracle.evolve(m2, basis=b, return_records=False)))[1::2].reshape(L, Wd)
    assert np.abs(p2 - p2[::-1, :]).max() > 1e-3


def test_separable_model_stays_a_product_state():
    """With no jumps the hydrogen-bond-shaped model is H_1 + H_2 + H_pos on separate
    digits, so rho_n is the Kronecker product of the separately evolved factors."""
    m = W.hb_shaped(gamma=0.0, gamma_pos=0.0, n_steps=50)
    b = oracle.enumerate_basis(m)
    rho = oracle.evolve(m, basis=b, return_records=False)
    c1 = W._model(n_cavities=1, atoms_per_cavity=[2], n_max=[3], g=m["g"][:2], dt=m["dt"],
                  n_steps=50, init={"atoms": {0: 1}})
    c2 = W._model(n_cavities=1, atoms_per_cavity=[2], n_max=[3], g=m["g"][2:], dt=m["dt"],
                  n_steps=50)
    px = W._model(n_cavities=0, atoms_per_cavity=[], n_max=[], n_extra=1,
                  extra_tunnel=m["extra_tunnel"], dt=m["dt"], n_steps=50)
    r1 = oracle.evolve(c1, return_records=False)
    r2 = oracle.evolve(c2, return_records=False)
    r3 = oracle.evolve(px, return_records=False)
    assert np.abs(rho - np.kron(np.kron(r1, r2), r3)).max() < 1e-13


# ---------------------------------------------------------------- gradients
def test_rabi_gradient_closed_form():
    """d/dg cos^2(g sqrt(n+1) t) = -sqrt(n+1) t sin(2 g sqrt(n+1) t)."""
    g, dt, steps, n = 0.05, 0.1, 300, 1
    m = W.jc_single(n_max=3, g=g, dt=dt, n_steps=steps, init_photons=n)
    b = oracle.enumerate_basis(m)
    w = (b.digits[:, b.atom_digit(0)] == 1).astype(float)
    loss, gg, gz, gga = oracle.adjoint_gradients(m, w, basis=b)
    t = dt * steps
    s = np.sqrt(n + 1)
    assert abs(loss - np.cos(g * s * t) ** 2) < 1e-12
    assert abs(gg[0] - (-s * t * np.sin(2 * g * s * t))) < 1e-10


def test_adjoint_matches_central_differences():
    """Adjoint gradients against the fourth-order central stencil (h = 1e-3), whose
    truncation and rounding errors are both below 1e-10 here."""
    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=60, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    loss, gg, gz, gga = oracle.adjoint_gradients(m, w, basis=b)
    h = 1e-3

    def stencil(f):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    for name, i, grad in (("g", 0, gg[0]), ("g", 4, gg[4]), ("zeta", 0, gz[0]), ("zeta", 5, gz[5])):
        base = m[name][i]
        fd = stencil(lambda d: oracle.loss_value(m, w, {(name, i): base + d}, basis=b))
        assert abs(grad - fd) <= 1e-6 * abs(fd) + 1e-10
    j = 3

    def with_rate(d):
        jumps = [(k, s, g + (d if q == j else 0.0)) for q, (k, s, g) in enumerate(m["jumps"])]
        return oracle.loss_value(dict(m, jumps=jumps), w, basis=b)

    fd = stencil(with_rate)
    assert abs(gga[j] - fd) <= 1e-6 * abs(fd) + 1e-10


def test_rate_gradients_all_jump_kinds_match_central_differences():
    """dL/dgamma_j for photon loss, atom decay and dephasing of an extra two-level degree of
    freedom, from a random mixed state, against the fourth-order central stencil."""
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    m["jumps"] = list(m["jumps"]) + [(1, 0, 0.01)]
    b = oracle.enumerate_basis(m)
    kinds = sorted({int(k) for k, _, _ in m["jumps"]})
    assert kinds == [0, 1, 2]
    rho0 = W.random_density(b.dim, seed=5)
    w = np.random.default_rng(3).uniform(-1, 1, b.dim)
    _, _, _, gga = oracle.adjoint_gradients(m, w, n_steps=30, rho0=rho0, basis=b)
    h = 1e-3

    def loss(jumps):
        rho = oracle.evolve(dict(m, jumps=jumps), n_steps=30, rho0=rho0, basis=b, return_records=False)
        return float(np.sum(w * np.real(np.diag(rho))))

    for j in range(len(m["jumps"])):
        def f(d):
            return loss([(k, s, g + (d if q == j else 0.0)) for q, (k, s, g) in enumerate(m["jumps"])])
        fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
        assert abs(gga[j] - fd) <= 1e-6 * abs(fd) + 1e-10, (j, gga[j], fd)


# ---------------------------------------------------------------- Strang scheme
def test_strang_second_order_convergence_to_continuum():
    """The symmetric scheme (midpoint half Lindblad steps around U) converges to exp(L t)
    rho_0 at second order in dt: halving dt divides the error by ~4."""
    m = W.jch_two_cavities(gamma=0.05)
    b = oracle.enumerate_basis(m)
    t = 20.0
    exact = oracle.continuum(m, t, basis=b)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        mm = dict(m, dt=dt, n_steps=int(round(t / dt)))
        rho = oracle.evolve(mm, basis=b, return_records=False, scheme="strang")
        errs.append(np.abs(rho - exact).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.6 <= e1 / e2 <= 4.4, errs
    # and it is far closer to the continuum than the first-order step at the same dt
    lie = oracle.evolve(dict(m, dt=0.1, n_steps=200), basis=b, return_records=False)
    assert errs[1] < 0.05 * np.abs(lie - exact).max()


def test_strang_discrete_photon_decay():
    """H = omega a^+a, A = a: L^+(a^+a) = -gamma a^+a, so each midpoint half step multiplies
    <n> by 1 - gamma dt/2 + (gamma dt/2)^2/2 and U keeps it: <n>_k = that factor^(2k) <n>_0."""
    gamma, dt, steps = 0.02, 0.1, 500
    m = W._model(n_cavities=1, atoms_per_cavity=[0], n_max=[6], jumps=[(0, 0, gamma)],
                 dt=dt, n_steps=steps, init={"photons": {0: 4}})
    b = oracle.enumerate_basis(m)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    psi /= np.linalg.norm(psi)
    rho0 = np.outer(psi, psi.conj())
    _, rec = oracle.evolve(m, rho0=rho0, basis=b, obs_ids=[b.dim + 1], scheme="strang")
    n0 = float(np.real(np.sum(np.arange(7) * np.diag(rho0))))
    h = 0.5 * gamma * dt
    want = n0 * (1 - h + 0.5 * h * h) ** (2 * np.arange(steps + 1))
    assert np.abs(rec[:, 0] - want).max() < 1e-13
    # second order: within (gamma dt)^2 gamma t / 24 of exp(-gamma t) (plus rounding)
    t = dt * steps
    assert abs(rec[-1, 0] - n0 * np.exp(-gamma * t)) <= n0 * (gamma * dt) ** 2 * gamma * t / 20


def test_strang_trace_and_unitary_limit():
    """Trace is kept exactly (tr L(X) = 0 in both stages); with no jumps the step is U rho U^+."""
    m = W.hb_shaped(n_steps=100, record_every=50)
    m.update(n_cavities=1, atoms_per_cavity=[2], n_max=[2], g=m["g"][:2], jumps=[(0, 0, 0.01), (2, 0, 0.02)])
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=7)
    rho = oracle.evolve(m, rho0=rho0, basis=b, return_records=False, scheme="strang")
    assert abs(np.trace(rho) - 1.0) < 1e-13
    m0 = dict(m, jumps=[])
    U = oracle.propagator(oracle.hamiltonian(m0, b), m0["dt"])
    rho_u = oracle.evolve(m0, rho0=rho0, basis=b, return_records=False, scheme="strang")
    Un = np.linalg.matrix_power(U, 100)
    assert np.abs(rho_u - Un @ rho0 @ Un.conj().T).max() < 1e-12


# ---------------------------------------------------------------- effective-Hamiltonian scheme
def _photon_cavity(gamma, dt, steps, n_max=2, n0=2):
    return W._model(n_cavities=1, atoms_per_cavity=[0], n_max=[n_max], jumps=[(0, 0, gamma)], dt=dt,
                    n_steps=steps, init={"photons": {0: n0}})


def test_effective_propagator_closed_form():
    """H = omega a^+a, A = a: H_eff = (omega - i gamma/2) a^+a is diagonal, so
    U_eff = diag(exp(-i omega k dt - gamma k dt / 2))."""
    gamma, dt = 0.03, 0.1
    m = _photon_cavity(gamma, dt, 1, n_max=4)
    b = oracle.enumerate_basis(m)
    U = oracle.effective_propagator(oracle.hamiltonian(m, b), oracle.jump_operators(m, b), dt)
    k = np.arange(5)
    assert np.abs(U - np.diag(np.exp(-1j * 1.0 * k * dt - 0.5 * gamma * k * dt))).max() < 1e-15


def test_effective_discrete_photon_decay():
    """Two photons, H = omega a^+a, A = a.  V_kk = exp(-gamma k dt) p_k, and the jump term
    adds dt gamma (k+1) V_{k+1,k+1} to p_k, so the populations follow
        p2' = e^{-2 gamma dt} p2,   p1' = e^{-gamma dt} p1 + 2 gamma dt e^{-2 gamma dt} p2,
        p0' = p0 + gamma dt e^{-gamma dt} p1;
    in particular p2 decays exactly as exp(-2 gamma t)."""
    gamma, dt, steps = 0.02, 0.1, 400
    m = _photon_cavity(gamma, dt, steps)
    b = oracle.enumerate_basis(m)
    _, rec = oracle.evolve(m, basis=b, obs_ids=[0, 1, 2], scheme="effective", record_every=1)
    p = np.array([0.0, 0.0, 1.0])
    want = [p.copy()]
    a1, a2 = np.exp(-gamma * dt), np.exp(-2 * gamma * dt)
    for _ in range(steps):
        p = np.array([p[0] + gamma * dt * a1 * p[1], a1 * p[1] + 2 * gamma * dt * a2 * p[2], a2 * p[2]])
        want.append(p.copy())
    # rounding only: a few units of 2^-53 per step over 400 steps
    assert np.abs(rec - np.array(want)).max() < 400 * 8 * 2.0 ** -53
    assert abs(rec[-1, 2] - np.exp(-2 * gamma * dt * steps)) < 400 * 8 * 2.0 ** -53


def test_effective_first_order_convergence_to_continuum():
    """The scheme converges to exp(L t) rho_0 at first order: halving dt halves the error."""
    m = W.jch_two_cavities(gamma=0.05)
    b = oracle.enumerate_basis(m)
    t = 20.0
    exact = oracle.continuum(m, t, basis=b)
    errs = []
    for dt in (0.2, 0.1, 0.05):
        mm = dict(m, dt=dt, n_steps=int(round(t / dt)))
        rho = oracle.evolve(mm, basis=b, return_records=False, scheme="effective")
        errs.append(np.abs(rho - exact).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.8 <= e1 / e2 <= 2.2, errs


def test_effective_positivity_trace_and_unitary_limit():
    """Each step is a sum of completely positive maps (U_eff . U_eff^+ and the jump
    sandwiches), so rho stays positive; the trace drifts by O(dt^2) per step (halving dt over
    a fixed time halves the drift); without jumps the step is U rho U^+."""
    m = W.hb_shaped(n_steps=200, record_every=50)
    m.update(n_cavities=1, atoms_per_cavity=[2], n_max=[2], g=m["g"][:2], jumps=[(0, 0, 0.05), (2, 0, 0.02)])
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=8)
    drift = []
    for dt, n in ((0.1, 200), (0.05, 400)):
        rho = oracle.evolve(dict(m, dt=dt), rho0=rho0, n_steps=n, basis=b, return_records=False, scheme="effective")
        assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -1e-13
        drift.append(abs(np.trace(rho).real - 1.0))
    assert 1.8 <= drift[0] / drift[1] <= 2.2, drift
    m0 = dict(m, jumps=[])
    U = oracle.propagator(oracle.hamiltonian(m0, b), m0["dt"])
    rho_u = oracle.evolve(m0, rho0=rho0, n_steps=100, basis=b, return_records=False, scheme="effective")
    Un = np.linalg.matrix_power(U, 100)
    assert np.abs(rho_u - Un @ rho0 @ Un.conj().T).max() < 1e-12


# ---------------------------------------------------------------- state selection (Sec. 3.2)
def test_selection_with_eps_zero_keeps_every_state_and_the_trajectory():
    """eps = 0 deletes nothing: the rounds reproduce the plain trajectory (each round's
    normalisation divides by a trace that is 1 to rounding)."""
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=3)
    keep, rho, sizes = oracle.select_states(m, 0.0, 40, 3, rho0=rho0, basis=b)
    assert sizes == [b.dim] * 3 and np.array_equal(keep, np.arange(b.dim))
    ref = oracle.evolve(m, rho0=rho0, n_steps=120, basis=b, return_records=False)
    assert np.abs(rho - ref).max() < 1e-13


def _reachable(H, start):
    """States connected to `start` through nonzero entries of H (breadth-first search)."""
    seen, front = {start}, [start]
    while front:
        nxt = []
        for k in front:
            for j in np.flatnonzero(H[:, k]):
                if j not in seen:
                    seen.add(int(j))
                    nxt.append(int(j))
        front = nxt
    return np.array(sorted(seen))


def test_selection_keeps_exactly_the_reachable_states_of_a_closed_model():
    """Without jumps the dynamics stays in the subspace H connects to the initial state;
    every other state has probability exactly zero and is deleted at any eps > 0, and the
    reduced trajectory equals the full one restricted to the kept states."""
    m = W.jch_two_cavities(gamma=0.0)
    m["jumps"] = []
    b = oracle.enumerate_basis(m)
    H = oracle.hamiltonian(m, b)
    k0 = oracle.initial_index(m, b)
    keep, rho, sizes = oracle.select_states(m, 1e-35, 50, 2, basis=b)
    assert np.array_equal(keep, _reachable(H, k0))
    assert len(keep) < b.dim
    full = oracle.evolve(m, n_steps=100, basis=b, return_records=False)
    assert np.abs(full[np.ix_(keep, keep)] - rho).max() < 1e-13
    assert np.abs(np.delete(np.diag(full), keep)).max() == 0.0


def test_selection_rounds_normalise_and_shrink():
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    keep, rho, sizes = oracle.select_states(m, 1e-20, 100, 3, basis=b)
    assert all(x >= y for x, y in zip(sizes, sizes[1:])) and sizes[-1] == len(keep) < b.dim
    assert abs(np.trace(rho).real - 1.0) < 1e-14
    assert np.abs(rho - rho.conj().T).max() < 1e-15
    assert oracle.initial_index(m, b) in keep


def test_photon_plane_closed_form():
    """One photon on a 9 x 5 plane without atoms (Sec. 4.2, basis |i>|j>): the oracle's
    trajectory equals the separable open-boundary mode expansion, and the symmetric start
    (4, 0) keeps the mirror symmetry P(i, j) = P(8 - i, j)."""
    from closed_forms import plane_photon_state
    m = W.photon_plane(9, 5, zeta=0.1, dt=0.1, n_steps=300, start=(4, 0))
    b = oracle.enumerate_basis(m)
    assert b.dim == 45
    rho = oracle.evolve(m, basis=b, return_records=False)
    psi = plane_photon_state(9, 5, 1.0, 0.1, 30.0, (4, 0))
    cav = np.array([int(np.flatnonzero(d)[0]) for d in b.digits])   # cavity of each basis state
    amp = psi.reshape(-1)[cav]
    assert np.abs(rho - np.outer(amp, amp.conj())).max() < 1e-12
    P = np.zeros(45)
    P[cav] = np.real(np.diag(rho))
    P = P.reshape(9, 5)
    assert np.abs(P - P[::-1, :]).max() < 1e-13


def test_strang_adjoint_matches_central_differences():
    """The discrete adjoint of the Strang step against the fourth-order central stencil
    (h = 1e-3) for couplings, hoppings and a leak rate of a 3 x 3 lattice, and for photon
    loss, atom decay and dephasing rates of a two-cavity model from a random mixed state."""
    h = 1e-3

    def stencil(f):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=60, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    loss, gg, gz, gga = oracle.adjoint_gradients(m, w, basis=b, scheme="strang")
    assert abs(loss - oracle.loss_value(m, w, basis=b, scheme="strang")) < 1e-14
    for name, i, grad in (("g", 0, gg[0]), ("g", 4, gg[4]), ("zeta", 0, gz[0]), ("zeta", 5, gz[5])):
        base = m[name][i]
        fd = stencil(lambda d: oracle.loss_value(m, w, {(name, i): base + d}, basis=b, scheme="strang"))
        assert abs(grad - fd) <= 1e-6 * abs(fd) + 1e-10, (name, i, grad, fd)
    j = 3

    def with_rate(d):
        jumps = [(k, s, g + (d if q == j else 0.0)) for q, (k, s, g) in enumerate(m["jumps"])]
        return oracle.loss_value(dict(m, jumps=jumps), w, basis=b, scheme="strang")
    fd = stencil(with_rate)
    assert abs(gga[j] - fd) <= 1e-6 * abs(fd) + 1e-10

    m2 = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m2.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
              zeta=[0.006], dt=0.1)
    m2["jumps"] = list(m2["jumps"]) + [(1, 0, 0.01)]
    b2 = oracle.enumerate_basis(m2)
    rho0 = W.random_density(b2.dim, seed=5)
    w2 = np.random.default_rng(3).uniform(-1, 1, b2.dim)
    _, _, _, gga2 = oracle.adjoint_gradients(m2, w2, n_steps=30, rho0=rho0, basis=b2, scheme="strang")

    def loss2(jumps):
        rho = oracle.evolve(dict(m2, jumps=jumps), n_steps=30, rho0=rho0, basis=b2, return_records=False,
                            scheme="strang")
        return float(np.sum(w2 * np.real(np.diag(rho))))

    for j in range(len(m2["jumps"])):
        fd = stencil(lambda d: loss2([(k, s, g + (d if q == j else 0.0)) for q, (k, s, g) in enumerate(m2["jumps"])]))
        assert abs(gga2[j] - fd) <= 1e-6 * abs(fd) + 1e-10, (j, gga2[j], fd)


def test_strang_adjoint_without_jumps_equals_the_lie_adjoint():
    """With no jumps both steps are U rho U^+, so the two adjoints coincide."""
    m = W.jch_two_cavities(gamma=0.0)
    m["jumps"] = []
    b = oracle.enumerate_basis(m)
    w = np.random.default_rng(8).uniform(0, 1, b.dim)
    a = oracle.adjoint_gradients(m, w, n_steps=50, basis=b)
    s = oracle.adjoint_gradients(m, w, n_steps=50, basis=b, scheme="strang")
    assert abs(a[0] - s[0]) < 1e-15
    for x, y in zip(a[1:3], s[1:3]):
        assert np.abs(x - y).max() < 1e-15
