"""The effective-Hamiltonian step (QED_SCHEME_EFFECTIVE: Eq. 3 regrouped, the anticommutator
inside U_eff = exp(-i dt (H - i/2 sum gamma A^+A)), then one Euler step of the jump terms) on
both GPU paths against the oracle's step_effective, whose U_eff comes from scipy's expm."""
import numpy as np
import pytest

import oracle
import qed_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")

RHO_TOL, POP_TOL = 1e-5, 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    build.build()


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _oracle_Ueff(m, b):
    return oracle.effective_propagator(oracle.hamiltonian(m, b), oracle.jump_operators(m, b), m["dt"])


def _photon_cavity(gamma=0.02, dt=0.1, steps=400):
    return W._model(n_cavities=1, atoms_per_cavity=[0], n_max=[2], jumps=[(0, 0, gamma)], dt=dt,
                    n_steps=steps, record_every=1, init={"photons": {0: 2}})


@pytest.mark.parametrize("make", [lambda: W.jch_two_cavities(gamma=0.02), lambda: W.hb_shaped(),
                                  lambda: W.lattice(5, 4, seed=1, gamma=5e-3), _photon_cavity])
def test_effective_propagator_matches_oracle(make):
    m = make()
    b = oracle.enumerate_basis(m)
    gm = qed.Model(m, scheme="effective")
    assert np.abs(gm.get_U().cpu().numpy() - _oracle_Ueff(m, b)).max() <= 1e-14


@pytest.mark.parametrize("make,steps", [(lambda: W.jch_two_cavities(gamma=0.02), 2000),
                                        (lambda: W.hb_shaped(), 300),
                                        (lambda: W.lattice(6, 5, seed=7, gamma=5e-3), 300)])
def test_effective_fp64_step_with_oracle_U(make, steps):
    """The step itself, with the oracle's U_eff injected, to 1e-12 per element."""
    m = make()
    b = oracle.enumerate_basis(m)
    U = _oracle_Ueff(m, b)
    gm = qed.Model(m, precision="fp64", scheme="effective")
    gm.set_U(_cuda(U))
    obs = list(range(b.dim))
    rho = _cuda(oracle.initial_density(m, b))
    rec = gm.evolve(rho, steps, record_every=50, obs_ids=obs)
    gm.sync()
    rho_ref, rec_ref = oracle.evolve(m, n_steps=steps, record_every=50, U=U, basis=b, obs_ids=obs,
                                     scheme="effective")
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= 1e-12
    assert np.abs(rec.cpu().numpy() - rec_ref).max() <= 1e-12


def test_effective_fp64_discrete_photon_decay():
    """Two photons in a damped cavity: with the GPU's own U_eff the top population decays as
    exp(-2 gamma t) exactly (the scheme's closed form), to rounding."""
    m = _photon_cavity()
    gm = qed.Model(m, precision="fp64", scheme="effective")
    b = oracle.enumerate_basis(m)
    rho = _cuda(oracle.initial_density(m, b))
    rec = gm.evolve(rho, 400, record_every=1, obs_ids=[2]).cpu().numpy()[:, 0]
    t = 0.1 * np.arange(401)
    assert np.abs(rec - np.exp(-2 * 0.02 * t)).max() <= 1e-13


@pytest.mark.parametrize("make,steps,rho0", [
    (lambda: W.jch_two_cavities(gamma=0.02), 2000, None),
    (lambda: W.hb_shaped(), 500, None),
    (lambda: W.hb_shaped(), 200, "random"),
    (lambda: W.chain_instance(np.random.default_rng(4), 100, 257), 300, None),
])
def test_effective_split_matches_oracle(make, steps, rho0):
    """Split precision (the increment form with the damped phases P_k = exp(-i H_kk dt -
    d_k dt/2)), the GPU's own U_eff, against the oracle's step with its own U_eff."""
    m = make()
    b = oracle.enumerate_basis(m)
    r0 = W.random_density(b.dim, seed=9) if rho0 == "random" else oracle.initial_density(m, b)
    gm = qed.Model(m, precision="split_fp16x2", scheme="effective")
    obs = list(range(b.dim))
    rho = _cuda(r0)
    rec = gm.evolve(rho, steps, record_every=50, obs_ids=obs)
    gm.sync()
    rho_ref, rec_ref = oracle.evolve(m, rho0=r0, n_steps=steps, record_every=50, basis=b, obs_ids=obs,
                                     scheme="effective")
    err, perr = np.abs(rho.cpu().numpy() - rho_ref).max(), np.abs(rec.cpu().numpy() - rec_ref).max()
    print(f"{m['name']} effective split, {steps} steps: max|drho| {err:.2e}, max|dpop| {perr:.2e}")
    assert err <= RHO_TOL and perr <= POP_TOL


def test_effective_batched_split_matches_oracle():
    specs = W.batched_chains(6, seed=2, dim_lo=32, dim_hi=300, n_steps=200, record_every=50)
    models, rhos = [], []
    for m in specs:
        gm = qed.Model(m, precision="split_fp16x2", scheme="effective")
        b = oracle.enumerate_basis(m)
        models.append(gm)
        rhos.append(_cuda(oracle.initial_density(m, b)))
    recs = qed.evolve_batched(models, rhos, 200, record_every=50)
    torch.cuda.synchronize()
    for m, r, rec in zip(specs, rhos, recs):
        b = oracle.enumerate_basis(m)
        rho_ref, rec_ref = oracle.evolve(m, n_steps=200, record_every=50, basis=b, obs_ids=list(range(b.dim)),
                                         scheme="effective")
        assert np.abs(r.cpu().numpy() - rho_ref).max() <= RHO_TOL
        assert np.abs(rec.cpu().numpy() - rec_ref).max() <= POP_TOL


@pytest.mark.parametrize("precision", ["fp64", "split_fp16x2"])
def test_switching_schemes_restores_the_lie_step(precision):
    """effective -> lie recomputes U = exp(-i H dt), the phases and the damping table: the
    model then steps exactly like a fresh Lie model."""
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    a = qed.Model(m, precision=precision)
    a.set_scheme("effective")
    a.set_scheme("lie")
    fresh = qed.Model(m, precision=precision)
    assert torch.equal(a.get_U(), fresh.get_U())
    ra, rf = _cuda(oracle.initial_density(m, b)), _cuda(oracle.initial_density(m, b))
    a.evolve(ra, 150)
    fresh.evolve(rf, 150)
    a.sync()
    fresh.sync()
    assert torch.equal(ra, rf)


def test_effective_adjoint_is_unsupported():
    m = W.jc_single(gamma=0.01)
    gm = qed.Model(m, precision="fp64", scheme="effective")
    b = oracle.enumerate_basis(m)
    with pytest.raises(qed.QedError) as ei:
        gm.adjoint(_cuda(oracle.initial_density(m, b)), 10, torch.ones(b.dim, dtype=torch.float64, device="cuda"))
    assert ei.value.status == qed.QED_EUNSUPPORTED
