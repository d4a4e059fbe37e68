"""GPU state space selection (qed_select_states, Sec. 3.2) against the oracle's
select_states: the same kept states (the thresholds sit orders of magnitude away from
every probability and growth speed of these seeded runs), the same reduced density
matrix, and a reduced model that keeps evolving like the oracle's projected problem."""
import numpy as np
import pytest
import scipy.sparse as sp

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


def _select(m, precision, eps, steps, rounds, rho0=None, scheme="lie"):
    b = oracle.enumerate_basis(m)
    rho0 = oracle.initial_density(m, b) if rho0 is None else rho0
    ref_keep, ref_rho, ref_sizes = oracle.select_states(m, eps, steps, rounds, rho0=rho0, basis=b, scheme=scheme)
    gm = qed.Model(m, precision=precision, scheme=scheme)
    red, rho, keep, sizes = qed.select_states(gm, _cuda(rho0), steps, rounds, eps)
    return b, (ref_keep, ref_rho, ref_sizes), (red, rho.cpu().numpy(), keep, list(sizes))


def test_fp64_selection_dim512_matches_oracle_and_keeps_evolving():
    """The dim-512 workload, eps 1e-20 (the nearest value is 9 orders away), 3 rounds of 100
    steps: 512 -> 8 states.  The GPU's Pade U and the oracle's eigh U differ by ~1e-15, so
    rho agrees to 2 n ||dU|| ~ 1e-12; then 200 more steps of the reduced model."""
    m = W.hb_shaped()
    b, (rk, rr, rs), (red, rho, keep, sizes) = _select(m, "fp64", 1e-20, 100, 3)
    print(f"fp64 selection sizes {sizes} (oracle {rs})")
    assert np.array_equal(keep, rk) and sizes == rs and red.dim == len(rk)
    assert np.abs(rho - rr).max() <= 1e-11
    # the reduced model is the projected problem: continue both
    H = oracle.hamiltonian(m, b)[np.ix_(rk, rk)]
    U = oracle.propagator(H, m["dt"])
    js = [(g, sp.csr_matrix(A[rk][:, rk])) for g, A in oracle.jump_operators(m, b)]
    ref = rr
    for _ in range(200):
        ref = oracle.step(ref, U, js, m["dt"])
    cur = _cuda(rho)
    red.evolve(cur, 200)
    red.sync()
    assert np.abs(cur.cpu().numpy() - ref).max() <= 1e-11
    labels = red.labels()
    assert np.array_equal(labels, b.digits[rk])


def test_split_selection_dim512_matches_oracle():
    """Split precision carries ~1e-7 absolute error in the populations, so its threshold
    must sit above that floor: eps 1e-4 keeps 3 of 512 states (nearest values 8.9e-6 and
    6.2e-4)."""
    m = W.hb_shaped()
    b, (rk, rr, rs), (red, rho, keep, sizes) = _select(m, "split_fp16x2", 1e-4, 100, 2)
    print(f"split selection sizes {sizes} (oracle {rs})")
    assert np.array_equal(keep, rk) and sizes == rs
    assert np.abs(rho - rr).max() <= 1e-5


def test_fp64_selection_eps_zero_keeps_everything_strang():
    """eps = 0 deletes nothing; with the Strang scheme the rounds reproduce the oracle's
    Strang trajectory from a random mixed state (dim 72)."""
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    rho0 = W.random_density(72, seed=3)
    b, (rk, rr, rs), (red, rho, keep, sizes) = _select(m, "fp64", 0.0, 40, 3, rho0=rho0, scheme="strang")
    assert sizes == [72, 72, 72] and np.array_equal(keep, np.arange(72)) and red.scheme == "strang"
    assert np.abs(rho - rr).max() <= 1e-12


def test_selection_argument_errors():
    m = W.jch_two_cavities()
    gm = qed.Model(m, precision="fp64")
    rho = _cuda(oracle.initial_density(m, oracle.enumerate_basis(m)))
    with pytest.raises(qed.QedError):
        qed.select_states(gm, rho, 0, 1, 1e-10)      # no steps
    with pytest.raises(qed.QedError):
        qed.select_states(gm, rho, 10, 1, 2.0)       # every state below eps
