"""GPU parity of the symmetric (Strang) scheme, qed_set_scheme(QED_SCHEME_STRANG): half
Lindblad steps by the explicit midpoint rule around U rho U^+, on the FP64 path, the
split-precision path (padded jump rows and the list merge), and the batched path, against
the oracle's step_strang."""
import numpy as np
import pytest

import oracle
import qed_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")

RHO_TOL = 1e-5
POP_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    build.build()


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _evolve(model, n_steps, precision, rho0=None, U=None, record_every=0, obs=None):
    b = oracle.enumerate_basis(model)
    gm = qed.Model(model, precision=precision, scheme="strang")
    if U is not None:
        gm.set_U(_cuda(U))
    rho = _cuda(oracle.initial_density(model, b) if rho0 is None else rho0)
    rec = gm.evolve(rho, n_steps, record_every=record_every, obs_ids=obs)
    gm.sync()
    return rho.cpu().numpy(), (None if rec is None else rec.cpu().numpy())


def test_fp64_strang_jch2_full_length_with_oracle_U():
    """Two JC cavities (dim 36), 20000 steps: per element within 1e-12 of the oracle."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    U = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    obs = list(range(b.dim))
    rho_ref, rec_ref = oracle.evolve(m, U=U, basis=b, obs_ids=obs, scheme="strang")
    rho, rec = _evolve(m, m["n_steps"], "fp64", U=U, record_every=m["record_every"], obs=obs)
    assert np.abs(rho - rho_ref).max() <= 1e-12
    assert np.abs(rec - rec_ref).max() <= 1e-12


def test_fp64_strang_mixed_state_many_jumps():
    """Photon loss, atom decay and dephasing from a random mixed state (dim 72)."""
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    m["jumps"] = list(m["jumps"]) + [(1, 0, 0.01)]
    b = oracle.enumerate_basis(m)
    U = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    rho0 = W.random_density(b.dim, seed=13)
    rho_ref = oracle.evolve(m, rho0=rho0, U=U, n_steps=400, basis=b, return_records=False, scheme="strang")
    rho, _ = _evolve(m, 400, "fp64", rho0=rho0, U=U)
    assert np.abs(rho - rho_ref).max() <= 1e-12


@pytest.mark.parametrize("make,steps", [
    (lambda: W.jch_two_cavities(), 20000),                 # padded jump rows, one tile
    (lambda: W.lattice(4, 4, seed=3, gamma=5e-3), 500),     # 16 leaks into the vacuum: list merge
    (lambda: W.hb_shaped(), 200),                           # dim 512, four tiles
])
def test_split_strang_matches_oracle(make, steps):
    m = make()
    b = oracle.enumerate_basis(m)
    obs = list(range(b.dim))
    r = 100 if steps >= 1000 else 50
    rho_ref, rec_ref = oracle.evolve(m, n_steps=steps, record_every=r, basis=b, obs_ids=obs, scheme="strang")
    rho, rec = _evolve(m, steps, "split_fp16x2", record_every=r, obs=obs)
    err, perr = np.abs(rho - rho_ref).max(), np.abs(rec - rec_ref).max()
    print(f"strang {m['name']} D={b.dim} steps={steps}: max|drho|={err:.2e} max|dpop|={perr:.2e}")
    assert err <= RHO_TOL and perr <= POP_TOL


def test_strang_closer_to_continuum_than_lie_on_gpu():
    """At dt = 0.1 the GPU's Strang trajectory is within 3e-7 of exp(L t) rho_0 (the oracle's
    Strang step: 1.5e-7) while the Lie trajectory is off by the first-order error, 2.3e-4
    (dim 36, t = 20)."""
    m = W.jch_two_cavities(gamma=0.05)
    b = oracle.enumerate_basis(m)
    mm = dict(m, dt=0.1, n_steps=200)
    exact = oracle.continuum(mm, 20.0, basis=b)
    rho_s, _ = _evolve(mm, 200, "fp64")
    gm = qed.Model(mm, precision="fp64")
    rho = _cuda(oracle.initial_density(mm, b))
    gm.evolve(rho, 200)
    gm.sync()
    err_s = np.abs(rho_s - exact).max()
    err_l = np.abs(rho.cpu().numpy() - exact).max()
    print(f"vs continuum: strang {err_s:.2e}, lie {err_l:.2e}")
    assert err_s <= 3e-7 and err_s < 0.01 * err_l


def test_batched_strang_matches_oracle():
    rng = np.random.default_rng(21)
    specs = [W.chain_instance(rng, 60 + 50 * i, 300) for i in range(3)]
    models = [qed.Model(s, precision="split_fp16x2", scheme="strang") for s in specs]
    rhos, refs = [], []
    for s, gm in zip(specs, models):
        b = oracle.enumerate_basis(s)
        rho0 = oracle.initial_density(s, b)
        rhos.append(_cuda(rho0))
        refs.append(oracle.evolve(s, rho0=rho0, n_steps=150, basis=b, return_records=False, scheme="strang"))
    qed.evolve_batched(models, rhos, 150)
    torch.cuda.synchronize()
    for r, ref in zip(rhos, refs):
        assert np.abs(r.cpu().numpy() - ref).max() <= RHO_TOL


def test_scheme_errors():
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    a = qed.Model(m, precision="split_fp16x2")
    c = qed.Model(m, precision="split_fp16x2", scheme="strang")
    rhos = [_cuda(oracle.initial_density(m, b)) for _ in range(2)]
    with pytest.raises(qed.QedError):  # one scheme per batch
        qed.evolve_batched([a, c], rhos, 5)


def _close(a, b, rtol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() <= rtol * max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("k", [7, 100])
def test_fp64_strang_adjoint_matches_oracle(k):
    """The adjoint of the Strang step (FP64 path) against the oracle's, on a 3 x 3 lattice
    (leaks) with ragged checkpoint segments and with every state kept, and on a two-cavity
    model with photon loss, atom decay and dephasing from a random mixed state."""
    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=60, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    ref = oracle.adjoint_gradients(m, w, basis=b, scheme="strang")
    gm = qed.Model(m, precision="fp64", scheme="strang")
    loss, gg, gz, gj = gm.adjoint(_cuda(oracle.initial_density(m, b)), 60, _cuda(w), checkpoint_every=k)
    assert abs(float(loss) - ref[0]) <= 1e-12
    for x, y in zip((gg, gz, gj), ref[1:]):
        assert _close(x.cpu().numpy(), y, 1e-9)

    m2 = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m2.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
              zeta=[0.006], dt=0.1)
    m2["jumps"] = list(m2["jumps"]) + [(1, 0, 0.01)]
    b2 = oracle.enumerate_basis(m2)
    rho0 = W.random_density(b2.dim, seed=5)
    w2 = np.random.default_rng(3).uniform(-1, 1, b2.dim)
    ref2 = oracle.adjoint_gradients(m2, w2, n_steps=30, rho0=rho0, basis=b2, scheme="strang")
    g2 = qed.Model(m2, precision="fp64", scheme="strang")
    loss2, gg2, gz2, gj2 = g2.adjoint(_cuda(rho0), 30, _cuda(w2), checkpoint_every=k)
    assert abs(float(loss2) - ref2[0]) <= 1e-12
    for x, y in zip((gg2, gz2, gj2), ref2[1:]):
        assert _close(x.cpu().numpy(), y, 1e-9)


# split precision: the bar of the split Lie adjoint tests (N x 2^-22 relative for N <= 100)
SPLIT_GRAD_RTOL = 2.4e-5
SPLIT_LOSS_ATOL = 1e-7


@pytest.mark.parametrize("k", [7, 100])
def test_split_strang_adjoint_matches_oracle(k):
    """The adjoint of the Strang step in split precision (the twin model's stages, X_n mu_n
    on the tensor cores) against the oracle's Strang adjoint: a 3 x 3 lattice with leaks
    (ragged checkpoint segments, and every state kept), an 8 x 8 lattice (dim 129, two
    128-row tiles), and two cavities with photon loss, atom decay and dephasing from a random
    mixed state with observable weights up to 5."""
    cases = []
    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=60, start=(0, 0))
    b = oracle.enumerate_basis(m)
    cases.append((m, b, oracle.initial_density(m, b), oracle.loss_diag(m, b, photons=[0], atoms=[0]), 60))
    m = W.lattice(8, 8, seed=4, gamma=0.02, dt=0.1, n_steps=50, start=(0, 0))
    b = oracle.enumerate_basis(m)
    cases.append((m, b, oracle.initial_density(m, b), oracle.loss_diag(m, b, photons=[0], atoms=[0]), 50))
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    m["jumps"] = list(m["jumps"]) + [(1, 0, 0.01)]
    b = oracle.enumerate_basis(m)
    cases.append((m, b, W.random_density(b.dim, seed=5), np.random.default_rng(3).uniform(-5, 5, b.dim), 30))
    for m, b, rho0, w, n in cases:
        ref = oracle.adjoint_gradients(m, w, n_steps=n, rho0=rho0, basis=b, scheme="strang")
        gm = qed.Model(m, precision="split_fp16x2", scheme="strang")
        loss, gg, gz, gj = gm.adjoint(_cuda(rho0), n, _cuda(w), checkpoint_every=k)
        got = [x.cpu().numpy() for x in (gg, gz, gj)]
        errs = [np.abs(x - y).max() / max(np.abs(y).max(), 1e-30) for x, y in zip(got, ref[1:]) if len(y)]
        print(f"split strang adjoint D={b.dim}: |dloss|={abs(float(loss) - ref[0]):.2e} rel errs={errs}")
        assert abs(float(loss) - ref[0]) <= 5 * SPLIT_LOSS_ATOL
        for x, y in zip(got, ref[1:]):
            assert _close(x, y, SPLIT_GRAD_RTOL)


def test_split_strang_adjoint_agrees_with_fp64_strang_adjoint():
    """Both paths' Strang adjoints of one model (the FP64 one matches the oracle to 1e-9)."""
    m = W.lattice(4, 4, seed=2, gamma=0.01, dt=0.1, n_steps=80, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = _cuda(oracle.loss_diag(m, b, photons=[0], atoms=[0]))
    rho0 = _cuda(oracle.initial_density(m, b))
    r64 = qed.Model(m, precision="fp64", scheme="strang").adjoint(rho0, 80, w, checkpoint_every=20)
    rs = qed.Model(m, precision="split_fp16x2", scheme="strang").adjoint(rho0, 80, w, checkpoint_every=20)
    assert abs(float(r64[0]) - float(rs[0])) <= SPLIT_LOSS_ATOL
    for x, y in zip(rs[1:], r64[1:]):
        assert _close(x.cpu().numpy(), y.cpu().numpy(), SPLIT_GRAD_RTOL)
