"""Fitting couplings to final populations with the adjoint gradients
(fit_final_populations; point 4 of Sec. 2): recovery of a Rabi coupling, and the fit of
two couplings of the dim-36 model to populations the oracle computes."""
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


def test_fit_recovers_rabi_coupling():
    """Single JC cavity from |e, 1>: the target is the oracle's populations at g* = 0.05
    after 300 steps; from g = 0.046 the fit returns g* to 1e-7."""
    g_true, steps = 0.05, 300
    m_true = W.jc_single(n_max=3, g=g_true, dt=0.1, n_steps=steps, init_photons=1)
    b = oracle.enumerate_basis(m_true)
    target = np.real(np.diag(oracle.evolve(m_true, n_steps=steps, basis=b, return_records=False)))
    start = dict(m_true, g=[0.046])
    fitted, hist = qed.fit_final_populations(start, target, steps, names=("g",))
    print(f"rabi fit: F {hist[0]:.2e} -> {hist[-1]:.2e} in {len(hist) - 1} iterations, g = {fitted['g'][0]:.10f}")
    assert all(b2 <= a2 for a2, b2 in zip(hist, hist[1:]))
    assert abs(fitted["g"][0] - g_true) <= 1e-7


def test_fit_two_couplings_to_oracle_populations():
    """Two JC cavities (dim 36) with photon loss: the target is the oracle's populations
    after 200 steps; from couplings off by +8 % and -7 % the fitted model reproduces them to
    1e-6 (F falls by more than 1e6).  At this time the populations hardly depend on the
    second cavity's coupling, so only the first is required to come back."""
    steps = 200
    m_true = W.jch_two_cavities()
    b = oracle.enumerate_basis(m_true)
    target = np.real(np.diag(oracle.evolve(m_true, n_steps=steps, basis=b, return_records=False)))
    g0 = m_true["g"]
    start = dict(m_true, g=[g0[0] * 1.08, g0[1] * 0.93])
    fitted, hist = qed.fit_final_populations(start, target, steps, names=("g",))
    print(f"two-coupling fit: F {hist[0]:.2e} -> {hist[-1]:.2e}, g = {fitted['g']}")
    assert hist[-1] <= 1e-6 * hist[0]
    p = np.real(np.diag(oracle.evolve(fitted, n_steps=steps, basis=b, return_records=False)))
    assert np.abs(p - target).max() <= 1e-6
    assert abs(fitted["g"][0] / g0[0] - 1.0) <= 1e-4
