"""The 32 x 32 photon-motion lattice (ground + one excitation, dim 2049), Sec. 4.2:
split precision against a closed form over all 2000 steps (closed system), against the
stored oracle trajectory with photon leaks, and the mirror symmetry of Sec. 4.2."""
import os

import numpy as np
import pytest

import oracle  # noqa: E402
import qed_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")

from closed_forms import lattice_single_excitation_state as closed_form_state  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    build.build()


def test_lattice_32x32_closed_full_length_split():
    m = W.lattice(gamma=0.0)
    gm = qed.Model(m, precision="split_fp16x2")
    D = gm.dim
    assert D == 2049
    i0 = gm.initial_index()
    rho = torch.zeros((D, D), dtype=torch.complex128, device="cuda")
    rho[i0, i0] = 1.0
    rec = gm.evolve(rho, m["n_steps"], record_every=m["record_every"], obs_ids=list(range(D)))
    gm.sync()
    psi = closed_form_state(32, 32, 1.0, 0.01, 0.01, m["dt"] * m["n_steps"], (16, 16))
    want = np.outer(psi, psi.conj())
    got = rho.cpu().numpy()
    err = np.abs(got - want).max()
    perr = np.abs(np.real(np.diag(got)) - np.abs(psi) ** 2).max()
    print(f"lattice 32x32 closed, 2000 split steps: max|drho|={err:.2e} max|dpop|={perr:.2e}")
    assert err <= 1e-5 and perr <= 1e-6
    assert np.abs(rec[-1].cpu().numpy() - np.real(np.diag(got))).max() <= 1e-12


def test_lattice_mirror_symmetry_odd_grid_split():
    """Odd grid, photon started on the mirror axis: P(i, j) = P(L-1-i, j) (Sec. 4.2)."""
    m = W.lattice(33, 9, gamma=1e-3, start=(16, 0), n_steps=500)
    gm = qed.Model(m, precision="split_fp16x2")
    D = gm.dim
    i0 = gm.initial_index()
    rho = torch.zeros((D, D), dtype=torch.complex128, device="cuda")
    rho[i0, i0] = 1.0
    gm.evolve(rho, m["n_steps"])
    gm.sync()
    p = np.real(np.diag(rho.cpu().numpy()))[1::2].reshape(33, 9)
    assert np.abs(p - p[::-1, :]).max() <= 1e-7


def test_lattice_32x32_against_stored_oracle():
    path = os.path.join(GOLDEN, "lattice_32x32_d2049_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("stored oracle trajectory not generated")
    g = np.load(path)
    m = W.lattice()
    gm = qed.Model(m, precision="split_fp16x2")
    D = gm.dim
    i0 = gm.initial_index()
    rho = torch.zeros((D, D), dtype=torch.complex128, device="cuda")
    rho[i0, i0] = 1.0
    rec = gm.evolve(rho, m["n_steps"], record_every=m["record_every"], obs_ids=list(range(D)))
    gm.sync()
    got = rho.cpu().numpy()
    err = np.abs(got[g["rho_rows"]] - g["rho_sample"]).max()
    perr = np.abs(rec.cpu().numpy() - g["records"]).max()
    print(f"lattice 32x32 leaky, 2000 split steps: max|drho| (rows)={err:.2e} max|dpop|={perr:.2e}")
    assert err <= 1e-5 and perr <= 1e-6


def test_lattice_fp64_and_split_short_vs_oracle():
    m = W.lattice(n_steps=20)
    b = oracle.enumerate_basis(m)
    rho_ref = oracle.evolve(m, basis=b, return_records=False)
    for prec, tol in (("fp64", 1e-12), ("split_fp16x2", 1e-7)):
        gm = qed.Model(m, precision=prec)
        if prec == "fp64":
            gm.set_U(torch.from_numpy(oracle.propagator(oracle.hamiltonian(m, b), m["dt"])).cuda())
        rho = torch.from_numpy(oracle.initial_density(m, b)).cuda()
        gm.evolve(rho, 20)
        gm.sync()
        assert np.abs(rho.cpu().numpy() - rho_ref).max() <= tol, prec


@pytest.mark.parametrize("start,steps", [((40, 0), 1000), ((20, 0), 500)])
def test_photon_plane_81x51_paper_size_split(start, steps):
    """The paper's plane (Sec. 4.2: length 81, height 51, area 4131, one photon, symmetric
    start (40, 0) and asymmetric start (20, 0)) on the split-precision path against the
    separable closed form; the symmetric start keeps P(i, j) = P(80 - i, j)."""
    from closed_forms import plane_photon_state
    m = W.photon_plane(start=start)
    gm = qed.Model(m, precision="split_fp16x2")
    D = gm.dim
    assert D == 4131
    cav = np.array([int(np.flatnonzero(d)[0]) for d in gm.labels()])  # cavity of each basis state
    i0 = gm.initial_index()
    rho = torch.zeros((D, D), dtype=torch.complex128, device="cuda")
    rho[i0, i0] = 1.0
    gm.evolve(rho, steps)
    gm.sync()
    r = rho.cpu().numpy()
    amp = plane_photon_state(81, 51, 1.0, m["zeta"][0], m["dt"] * steps, start).reshape(-1)[cav]
    pop_err = np.abs(np.real(np.diag(r)) - np.abs(amp) ** 2).max()
    rows = [0, i0, D // 2, D - 1]
    rho_err = np.abs(r[rows] - np.outer(amp[rows], amp.conj())).max()
    print(f"plane 81x51 from {start}, {steps} steps: max|dpop|={pop_err:.2e} max|drho| (rows)={rho_err:.2e}")
    assert pop_err <= 1e-6 and rho_err <= 1e-5
    assert abs(np.trace(r).real - 1.0) <= 1e-7
    if start == (40, 0):
        P = np.zeros(D)
        P[cav] = np.real(np.diag(r))
        P = P.reshape(81, 51)
        assert np.abs(P - P[::-1, :]).max() <= 1e-6
