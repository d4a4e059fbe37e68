"""GPU adjoint gradients (qed_adjoint) against the oracle's discrete adjoint, central
finite differences of the GPU forward, and the closed-form Rabi gradient."""
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


def _gpu_adjoint(m, steps, w, k, rho0=None, b=None):
    b = b or oracle.enumerate_basis(m)
    gm = qed.Model(m)
    rho0 = oracle.initial_density(m, b) if rho0 is None else rho0
    loss, gg, gz, gj = gm.adjoint(_cuda(rho0), steps, _cuda(w), checkpoint_every=k)
    return float(loss), gg.cpu().numpy(), gz.cpu().numpy(), gj.cpu().numpy()


def _close(a, b, rtol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    scale = max(np.abs(b).max(), 1e-30)
    return np.abs(a - b).max() <= rtol * scale


@pytest.mark.parametrize("k", [7, 60, 1])
def test_adjoint_matches_oracle_lattice(k):
    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=60, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    ref = oracle.adjoint_gradients(m, w, basis=b)
    got = _gpu_adjoint(m, 60, w, k, b=b)
    assert abs(got[0] - ref[0]) <= 1e-12
    for x, y in zip(got[1:], ref[1:]):
        assert _close(x, y, 1e-9)


def test_adjoint_matches_oracle_cavities_and_dephasing():
    """Photon-loss jumps on a full product basis plus extra-digit dephasing, random mixed
    initial state, ragged checkpoint segments."""
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=11)
    w = np.random.default_rng(2).uniform(0, 1, b.dim)
    ref = oracle.adjoint_gradients(m, w, n_steps=45, rho0=rho0, basis=b)
    got = _gpu_adjoint(m, 45, w, 10, rho0=rho0, b=b)
    assert abs(got[0] - ref[0]) <= 1e-12
    for x, y in zip(got[1:], ref[1:]):
        assert _close(x, y, 1e-9)


def test_rabi_gradient_closed_form():
    g, dt, steps, n = 0.05, 0.1, 300, 1
    m = W.jc_single(n_max=3, g=g, dt=dt, n_steps=steps, init_photons=n)
    b = oracle.enumerate_basis(m)
    w = (b.digits[:, b.atom_digit(0)] == 1).astype(float)
    loss, gg, _, _ = _gpu_adjoint(m, steps, w, 64, b=b)
    t, s = dt * steps, np.sqrt(n + 1)
    assert abs(loss - np.cos(g * s * t) ** 2) <= 1e-12
    assert abs(gg[0] - (-s * t * np.sin(2 * g * s * t))) <= 1e-9


def test_adjoint_against_gpu_finite_differences():
    """Fourth-order central differences (h = 1e-3) of the GPU FP64 forward."""
    m = W.lattice(4, 4, seed=9, gamma=0.01, dt=0.1, n_steps=80, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    loss, gg, gz, gj = _gpu_adjoint(m, 80, w, 16, b=b)
    rho0 = oracle.initial_density(m, b)

    def forward(mm):
        gm = qed.Model(mm)
        rho = _cuda(rho0)
        gm.evolve(rho, 80)
        gm.sync()
        return float(np.sum(w * np.real(np.diag(rho.cpu().numpy()))))

    h = 1e-3
    for name, i, grad in (("g", 0, gg[0]), ("g", 5, gg[5]), ("zeta", 1, gz[1]), ("zeta", 3, gz[3])):
        def f(d):
            mm = dict(m)
            arr = list(mm[name])
            arr[i] += d
            mm[name] = arr
            return forward(mm)
        fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
        assert abs(grad - fd) <= 1e-6 * abs(fd) + 1e-10, (name, i, grad, fd)
    j = 0

    def fj(d):
        jumps = [(kk, s, gmm + (d if q == j else 0.0)) for q, (kk, s, gmm) in enumerate(m["jumps"])]
        return forward(dict(m, jumps=jumps))
    fd = (-fj(2 * h) + 8 * fj(h) - 8 * fj(-h) + fj(-2 * h)) / (12 * h)
    assert abs(gj[j] - fd) <= 1e-6 * abs(fd) + 1e-10


def test_autograd_function():
    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=30, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    ref = oracle.adjoint_gradients(m, w, n_steps=30, basis=b)
    g = torch.tensor(m["g"], dtype=torch.float64, requires_grad=True)
    z = torch.tensor(m["zeta"], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor([x[2] for x in m["jumps"]], dtype=torch.float64, requires_grad=True)
    loss = qed.qme_loss(g, z, gam, m, _cuda(oracle.initial_density(m, b)), 30, _cuda(w), 8)
    (2.0 * loss).backward()
    assert abs(float(loss.detach()) - ref[0]) <= 1e-12
    assert _close(g.grad.numpy(), 2 * ref[1], 1e-9)
    assert _close(z.grad.numpy(), 2 * ref[2], 1e-9)
    assert _close(gam.grad.numpy(), 2 * ref[3], 1e-9)


def test_adjoint_argument_errors():
    m = W.jch_two_cavities()
    gm = qed.Model(m)
    rho = torch.zeros((36, 36), dtype=torch.complex128, device="cuda")
    with pytest.raises(qed.QedError):
        gm.adjoint(rho, 10, torch.zeros(36, dtype=torch.float64, device="cuda"), checkpoint_every=0)


def _gpu_adjoint_prec(m, steps, w, k, precision, rho0=None, b=None):
    b = b or oracle.enumerate_basis(m)
    gm = qed.Model(m, precision=precision)
    rho0 = oracle.initial_density(m, b) if rho0 is None else rho0
    loss, gg, gz, gj = gm.adjoint(_cuda(rho0), steps, _cuda(w), checkpoint_every=k)
    return float(loss), gg.cpu().numpy(), gz.cpu().numpy(), gj.cpu().numpy()


# The split-precision adjoint carries each step's products to about 2^-22 = 2.4e-7 relative
# (FP16 hi/lo pieces, FP32 accumulation) and the state as double-floats; over N <= 100 steps
# the rounding errors add up to at most N * 2.4e-7 = 2.4e-5 of the largest gradient component
# (measured: <= 3.1e-6), and to far less on the loss (measured: <= 2e-9).
SPLIT_GRAD_RTOL = 2.4e-5
SPLIT_LOSS_ATOL = 1e-7


@pytest.mark.parametrize("nx,ny,steps,k", [(4, 4, 80, 16), (8, 8, 100, 30), (3, 3, 25, 100)])
def test_split_adjoint_matches_oracle_lattice(nx, ny, steps, k):
    """Several 128-row tiles at 8x8 (D = 129), ragged checkpoint segments, k > n_steps."""
    m = W.lattice(nx, ny, seed=4, gamma=0.02, dt=0.1, n_steps=steps, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    ref = oracle.adjoint_gradients(m, w, n_steps=steps, basis=b)
    got = _gpu_adjoint_prec(m, steps, w, k, "split_fp16x2", b=b)
    errs = [np.abs(np.asarray(x) - y).max() / max(np.abs(y).max(), 1e-30) for x, y in zip(got[1:], ref[1:])]
    print(f"split adjoint {nx}x{ny}: |dloss|={abs(got[0] - ref[0]):.2e} rel grad errs={errs}")
    assert abs(got[0] - ref[0]) <= SPLIT_LOSS_ATOL
    for x, y in zip(got[1:], ref[1:]):
        assert _close(x, y, SPLIT_GRAD_RTOL)


def test_split_adjoint_cavities_dephasing_large_observable():
    """Observable weights up to 5 (the co-state is run at o / 8 and scaled back), random mixed
    initial state, photon loss and extra-digit dephasing."""
    m = W.hb_shaped(gamma=0.02, gamma_pos=0.03)
    m.update(n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2], g=[0.013, 0.017], bonds=[(0, 1)],
             zeta=[0.006], dt=0.1)
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=11)
    w = np.random.default_rng(2).uniform(-5, 5, b.dim)
    ref = oracle.adjoint_gradients(m, w, n_steps=45, rho0=rho0, basis=b)
    got = _gpu_adjoint_prec(m, 45, w, 10, "split_fp16x2", rho0=rho0, b=b)
    assert abs(got[0] - ref[0]) <= 5 * SPLIT_LOSS_ATOL
    for x, y in zip(got[1:], ref[1:]):
        assert _close(x, y, SPLIT_GRAD_RTOL)


def test_split_adjoint_autograd():
    m = W.lattice(3, 3, seed=4, gamma=0.02, dt=0.1, n_steps=30, start=(0, 0))
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, photons=[0], atoms=[0])
    ref = oracle.adjoint_gradients(m, w, n_steps=30, basis=b)
    g = torch.tensor(m["g"], dtype=torch.float64, requires_grad=True)
    z = torch.tensor(m["zeta"], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor([x[2] for x in m["jumps"]], dtype=torch.float64, requires_grad=True)
    loss = qed.qme_loss(g, z, gam, m, _cuda(oracle.initial_density(m, b)), 30, _cuda(w), 8,
                        precision="split_fp16x2")
    loss.backward()
    assert abs(float(loss.detach()) - ref[0]) <= SPLIT_LOSS_ATOL
    assert _close(g.grad.numpy(), ref[1], SPLIT_GRAD_RTOL)
    assert _close(z.grad.numpy(), ref[2], SPLIT_GRAD_RTOL)
    assert _close(gam.grad.numpy(), ref[3], SPLIT_GRAD_RTOL)


def _full_size_adjoint(precision):
    import os
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             "adjoint_lattice_24x24_d1153_oracle.npz"))
    m = W.adjoint_lattice()
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, **m["loss_states"])
    got = _gpu_adjoint_prec(m, m["n_steps"], w, m["checkpoint_every"], precision, b=b)
    ref = (float(g["loss"]), g["grad_g"], g["grad_zeta"], g["grad_gamma"])
    errs = [np.abs(np.asarray(x) - y).max() / np.abs(y).max() for x, y in zip(got[1:], ref[1:])]
    print(f"adjoint 24x24 {precision}: loss {got[0]:.6e} (oracle {ref[0]:.6e}), "
          f"max err / max |grad| (g, zeta, gamma) = {errs}")
    return got, ref


def test_split_adjoint_24x24_full_size_against_stored_oracle():
    """The 24 x 24 adjoint workload at full size (dim 1153, 1000 steps, every state kept) on
    the split-precision path, as the bench runs it: all 576 g, 1104 zeta and 576 rate
    gradients against the oracle's discrete adjoint (tests/golden/make_golden.py)."""
    got, ref = _full_size_adjoint("split_fp16x2")
    assert abs(got[0] - ref[0]) <= 1e-6
    for x, y in zip(got[1:], ref[1:]):
        assert _close(x, y, 1e-4)


def test_fp64_adjoint_24x24_full_size_against_stored_oracle():
    """The same on the FP64 path.  The GPU's Pade U and the oracle's eigh U differ by ~1e-15
    per element, so after n = 1000 steps rho_N (and the loss) may differ by up to
    2 n ||dU||_2 ~ 1e-11 (measured 1.2e-12); the gradients agree to 2e-12 relative."""
    got, ref = _full_size_adjoint("fp64")
    assert abs(got[0] - ref[0]) <= 1e-11
    for x, y in zip(got[1:], ref[1:]):
        assert _close(x, y, 1e-9)


def test_split_adjoint_24x24_full_size_against_finite_differences():
    """Sixteen seeded couplings within three hops of the corner (qed_workloads.fd_parameters)
    of the full-size 24 x 24 workload: the split-precision adjoint against fourth-order
    central differences (h = 1e-3) of the split-precision forward.  Bound: 1e-4 relative
    plus the stencil's noise floor.  The split forward's loss carries ~1e-9 of rounding
    noise that does not vary smoothly with the parameters; the stencil's weights
    (1 + 8 + 8 + 1) / (12 h) turn that into a few 1e-6 on a derivative (measured up to
    4.2e-6 on these sixteen), so |adjoint - fd| <= 1e-4 |fd| + 1e-5.  The gradients span
    1e-6 to 30; the adjoint itself agrees with the oracle's to 1.5e-7 (printed), which the
    full-size comparison with the stored oracle gradients checks on all 2256."""
    import os
    m = W.adjoint_lattice()
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, **m["loss_states"])
    N = m["n_steps"]
    loss, gg, gz, _ = _gpu_adjoint_prec(m, N, w, m["checkpoint_every"], "split_fp16x2", b=b)
    rho0 = _cuda(oracle.initial_density(m, b))
    wd = _cuda(w)

    def forward(mm):
        gm = qed.Model(mm, precision="split_fp16x2")
        rho = rho0.clone()
        gm.evolve(rho, N)
        gm.sync()
        out = float(torch.sum(wd * torch.real(torch.diagonal(rho))))
        gm.close()
        return out

    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             "adjoint_lattice_24x24_d1153_oracle.npz"))
    h = 1e-3
    for name, i in W.fd_parameters(m):
        def f(d):
            mm = dict(m)
            arr = list(mm[name])
            arr[i] += d
            mm[name] = arr
            return forward(mm)
        fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
        ad = (gg if name == "g" else gz)[i]
        ref = (g["grad_g"] if name == "g" else g["grad_zeta"])[i]
        print(f"{name}[{i}]: adjoint {ad:.8e} fd {fd:.8e} oracle {ref:.8e}")
        assert abs(ad - fd) <= 1e-4 * abs(fd) + 1e-5, (name, i, ad, fd)
