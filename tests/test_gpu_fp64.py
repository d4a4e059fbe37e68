"""GPU parity of the all-FP64 path against the FP64 oracle (max-abs per element)."""
import numpy as np
import pytest

import oracle
import qed_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    build.build()


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _run(model, n_steps, U=None, precision="fp64", rho0=None, record_every=None, obs=None):
    b = oracle.enumerate_basis(model)
    gm = qed.Model(model, precision=precision)
    if U is not None:
        gm.set_U(_cuda(U))
    rho = _cuda(oracle.initial_density(model, b) if rho0 is None else rho0)
    rec = gm.evolve(rho, n_steps, record_every=record_every or 0, obs_ids=obs)
    gm.sync()
    return gm, rho.cpu().numpy(), (rec.cpu().numpy() if rec is not None else None)


@pytest.mark.parametrize("make", [
    lambda: W.jch_two_cavities(),
    lambda: W.hb_shaped(),
    lambda: W.lattice(5, 4, seed=1),
    lambda: W.chain_instance(np.random.default_rng(2), 60, 200),
])
def test_propagator_matches_oracle(make):
    m = make()
    b = oracle.enumerate_basis(m)
    U_ref = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    gm = qed.Model(m)
    U = gm.get_U().cpu().numpy()
    assert np.abs(U - U_ref).max() <= 1e-14
    assert np.abs(U.conj().T @ U - np.eye(len(U))).max() <= 1e-13


def test_propagator_with_squaring():
    """||H dt||_1 above theta_13 exercises the squaring phase."""
    m = W.jch_two_cavities()
    m["dt"] = 3.0
    b = oracle.enumerate_basis(m)
    U_ref = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    U = qed.Model(m).get_U().cpu().numpy()
    assert np.abs(U - U_ref).max() <= 1e-13


def test_jch2_full_length_with_oracle_U():
    """Two coupled JC cavities (dim 36), 20000 steps, populations every 100 steps, with the
    oracle's U injected: the step itself matches to 1e-12 max-abs."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    U = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    obs = list(range(b.dim))
    rho_ref, rec_ref = oracle.evolve(m, U=U, basis=b, obs_ids=obs)
    _, rho, rec = _run(m, m["n_steps"], U=U, record_every=m["record_every"], obs=obs)
    assert rec.shape == rec_ref.shape == (201, 36)
    assert np.abs(rho - rho_ref).max() <= 1e-12
    assert np.abs(rec - rec_ref).max() <= 1e-12


def test_jch2_full_length_own_U():
    """With the GPU's own Pade U the step maps differ by dU = U_gpu - U_oracle; since
    ||U rho U^+ - U' rho U'^+|| <= 2 ||dU||_2 for unit-trace rho and every later step is
    a contraction, the difference after n steps is at most 2 n ||dU||_2."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    U_ref = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    rho_ref = oracle.evolve(m, basis=b, return_records=False)
    gm, rho, _ = _run(m, m["n_steps"])
    dU = np.linalg.norm(gm.get_U().cpu().numpy() - U_ref, 2)
    assert dU <= 1e-14
    err = np.abs(rho - rho_ref).max()
    print(f"own-U max|drho| after {m['n_steps']} steps = {err:.3e} (bound {2 * m['n_steps'] * dU:.3e})")
    assert err <= 2 * m["n_steps"] * dU + 1e-13


@pytest.mark.parametrize("make,steps", [
    (lambda: W.hb_shaped(), 100),
    (lambda: W.lattice(6, 5, seed=7, gamma=5e-3), 200),
    (lambda: W.chain_instance(np.random.default_rng(4), 100, 257), 150),
    (lambda: W.jch_two_cavities(gamma=0.02), 500),
])
def test_fp64_parity_random_state(make, steps):
    """A random mixed initial state (every element nonzero), ragged dimensions."""
    m = make()
    b = oracle.enumerate_basis(m)
    U = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    rho0 = W.random_density(b.dim, seed=5)
    rho_ref = oracle.evolve(m, rho0=rho0, n_steps=steps, U=U, basis=b, return_records=False)
    _, rho, _ = _run(m, steps, U=U, rho0=rho0)
    assert np.abs(rho - rho_ref).max() <= 1e-12


def test_observables_and_offsets():
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    U = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    gm = qed.Model(m)
    gm.set_U(_cuda(U))
    rho = _cuda(oracle.initial_density(m, b))
    n_named = gm.n_observables - b.dim
    ids = [0, 3, b.dim - 1] + [b.dim + k for k in range(n_named)]
    rec1 = gm.evolve(rho, 30, record_every=7, obs_ids=ids)
    rec2 = gm.evolve(rho, 25, record_every=7, obs_ids=ids, step_offset=30)
    gm.sync()
    rho_ref, rec_ref = oracle.evolve(m, n_steps=55, record_every=7, U=U, basis=b, obs_ids=ids)
    got = np.concatenate([rec1.cpu().numpy(), rec2.cpu().numpy()])
    # records at 0, 7, ..., 28 from the first call and 35, 42, 49 from the second
    assert got.shape == rec_ref.shape
    assert np.abs(got - rec_ref).max() <= 1e-12
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= 1e-12
    out = gm.observables(rho, ids).cpu().numpy()
    W_ = oracle.observable_weights(m, b)
    assert np.abs(out - oracle.observables(rho_ref, W_, ids)).max() <= 1e-12


def test_zero_steps_and_argument_errors():
    m = W.jch_two_cavities()
    gm = qed.Model(m)
    rho = torch.zeros((36, 36), dtype=torch.complex128, device="cuda")
    rho[0, 0] = 1
    rec = gm.evolve(rho, 0, record_every=1, obs_ids=[0])
    gm.sync()
    assert rec.shape == (1, 1) and float(rec[0, 0]) == 1.0
    with pytest.raises(qed.QedError):
        gm.evolve(rho, 5, record_every=0, obs_ids=[0], records=torch.zeros(1, 1, device="cuda",
                                                                           dtype=torch.float64))
    with pytest.raises(qed.QedError):
        gm.observables(rho, [10 ** 6])
    with pytest.raises(qed.QedError):
        gm.evolve(rho, -1)


def test_build_errors_are_codes():
    m = W.jch_two_cavities()
    with pytest.raises(qed.QedError) as ei:
        qed.Model(m, dt=-1.0)
    assert ei.value.status == qed.QED_EINVAL
    with pytest.raises(qed.QedError) as ei:
        qed.Model(m, precision="split_tf32x3")
    assert ei.value.status == qed.QED_EUNSUPPORTED
