"""Batched evolution of uneven instances (qed_evolve_batched): every instance against the
FP64 oracle (at small sizes run here, at the workload's own scale from stored oracle
trajectories), and against the same model evolved on its own."""
import os

import numpy as np
import pytest

import oracle
import qed_workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    build.build()


def _setup(specs, precision):
    models, rhos = [], []
    for m in specs:
        gm = qed.Model(m, precision=precision)
        i0 = gm.initial_index()
        r = torch.zeros((gm.dim, gm.dim), dtype=torch.complex128, device="cuda")
        r[i0, i0] = 1.0
        models.append(gm)
        rhos.append(r)
    return models, rhos


def _oracle_U(m, b):
    return oracle.propagator(oracle.hamiltonian(m, b), m["dt"])


@pytest.mark.parametrize("precision,tol_rho,tol_pop", [("split_fp16x2", 1e-5, 1e-6), ("fp64", 1e-12, 1e-12)])
def test_batched_instances_match_oracle(precision, tol_rho, tol_pop):
    """16 seeded chains (dims 32..256, several tiles, ragged), 300 steps, records every 50.
    The oracle steps with its own eigendecomposition U; the FP64 instances are given that U
    (qed_set_U), so the comparison isolates the step, and the GPU's own Pade U is checked
    against it separately."""
    specs = W.batched_chains(16, seed=3, dim_lo=32, dim_hi=256, n_steps=300, record_every=50)
    models, rhos = _setup(specs, precision)
    bases = [oracle.enumerate_basis(m) for m in specs]
    Us = [_oracle_U(m, b) for m, b in zip(specs, bases)]
    if precision == "fp64":
        for gm, U in zip(models, Us):
            assert np.abs(gm.get_U().cpu().numpy() - U).max() <= 1e-14
            gm.set_U(torch.from_numpy(U).cuda())
    recs = qed.evolve_batched(models, rhos, 300, record_every=50)
    torch.cuda.synchronize()
    worst = 0.0
    for m, b, U, r, rec in zip(specs, bases, Us, rhos, recs):
        rho_ref, rec_ref = oracle.evolve(m, n_steps=300, record_every=50, basis=b, U=U,
                                         obs_ids=list(range(b.dim)))
        err = np.abs(r.cpu().numpy() - rho_ref).max()
        perr = np.abs(rec.cpu().numpy() - rec_ref).max()
        worst = max(worst, err)
        assert err <= tol_rho and perr <= tol_pop, (m["name"], err, perr)
    print(f"batched {precision}: worst max|drho| over 16 instances = {worst:.2e}")


U_ROUND = 2.0 ** -53


@pytest.mark.parametrize("precision,tol_rho,tol_pop", [("split_fp16x2", 1e-5, 1e-6), ("fp64", None, None)])
def test_batched_chains_full_size_against_stored_oracle(precision, tol_rho, tol_pop):
    """The batched-chains workload at its own scale: the first 16 of its 512 seeded instances
    (dims 53..1008, the instances the bench's run starts with), 1000 steps of dt 0.1,
    populations every 100 steps, against the oracle trajectories stored by
    tests/golden/make_golden.py (every population record and eight rows of each final rho).
    Split precision runs exactly as benchmarked (the GPU's own U); the FP64 instances are
    given the oracle's eigendecomposition U (qed_set_U) so the 1e-12 bar applies to the step,
    and each GPU Pade U is checked against that U to 1e-14.

    FP64 bound: both sides compute V = U rho U^+ as two products of length D in a different
    summation order.  Each product's entries are sums of D terms whose magnitudes add up to at
    most 1 (unit-norm rows of U, columns of a density matrix of norm <= 1), so each product
    errs by at most D u per entry (u = 2^-53) and a step by 2 D u; over n steps that adds up
    to at most 2 n D u (about 1.8e-10 at D = 793, n = 1000; the dim-36 workload keeps the
    1e-12 bar in test_gpu_fp64.py)."""
    g = np.load(os.path.join(GOLDEN, "batched_chains_d53_1008_oracle.npz"))
    specs = W.batched_chains(int(g["n"]), seed=0)
    assert specs[0]["n_steps"] == 1000 and specs[0]["record_every"] == 100
    models, rhos = _setup(specs, precision)
    dims = [gm.dim for gm in models]
    assert min(dims) == 53 and max(dims) == 1008
    if precision == "fp64":
        for m, gm in zip(specs, models):
            U = _oracle_U(m, oracle.enumerate_basis(m))
            assert np.abs(gm.get_U().cpu().numpy() - U).max() <= 1e-14
            gm.set_U(torch.from_numpy(U).cuda())
    recs = qed.evolve_batched(models, rhos, 1000, record_every=100)
    torch.cuda.synchronize()
    worst, worst_p = 0.0, 0.0
    for i, (r, rec) in enumerate(zip(rhos, recs)):
        rows = g[f"rows_{i}"]
        err = np.abs(r.cpu().numpy()[rows] - g[f"rho_rows_{i}"]).max()
        perr = np.abs(rec.cpu().numpy() - g[f"records_{i}"]).max()
        worst, worst_p = max(worst, err), max(worst_p, perr)
        tr = tol_rho if tol_rho is not None else 2 * 1000 * dims[i] * U_ROUND
        tp = tol_pop if tol_pop is not None else 2 * 1000 * dims[i] * U_ROUND
        assert err <= tr and perr <= tp, (i, dims[i], err, perr, tr)
    print(f"batched chains d53..1008 {precision}, 1000 steps: max|drho| (sampled rows) = {worst:.2e}, "
          f"max|dpop| = {worst_p:.2e}")


def test_batched_chains_full_size_fp64_own_U():
    """The first six instances of the same workload in FP64 with the GPU's own Pade U (no
    qed_set_U), against the same stored oracle trajectories (the oracle's eigendecomposition
    U).  The step maps differ by dU = U_gpu - U_oracle; each step moves the state by at most
    2 ||dU||_2 (unit-trace rho) and the Lindblad part and later steps do not enlarge that, so
    after n steps the gap is at most 2 n ||dU||_2 plus the rounding bound 2 n D u above."""
    g = np.load(os.path.join(GOLDEN, "batched_chains_d53_1008_oracle.npz"))
    specs = W.batched_chains(int(g["n"]), seed=0)[:6]
    models, rhos = _setup(specs, "fp64")
    dUs = []
    for m, gm in zip(specs, models):
        U = _oracle_U(m, oracle.enumerate_basis(m))
        dUs.append(np.linalg.norm(gm.get_U().cpu().numpy() - U, 2))
        assert dUs[-1] <= 1e-14
    recs = qed.evolve_batched(models, rhos, 1000, record_every=100)
    torch.cuda.synchronize()
    for i, (gm, r, rec) in enumerate(zip(models, rhos, recs)):
        rows = g[f"rows_{i}"]
        err = np.abs(r.cpu().numpy()[rows] - g[f"rho_rows_{i}"]).max()
        perr = np.abs(rec.cpu().numpy() - g[f"records_{i}"]).max()
        bound = 2 * 1000 * dUs[i] + 2 * 1000 * gm.dim * U_ROUND
        assert err <= bound and perr <= bound, (i, gm.dim, err, perr, bound)


def test_batched_equals_single_model_runs():
    specs = W.batched_chains(24, seed=5, dim_lo=32, dim_hi=640, n_steps=200)
    models, rhos = _setup(specs, "split_fp16x2")
    singles = [r.clone() for r in rhos]
    qed.evolve_batched(models, rhos, 200)
    for gm, r in zip(models, singles):
        gm.evolve(r, 200)
    torch.cuda.synchronize()
    for r, s_ in zip(rhos, singles):
        # same kernels; only the split-K slicing of the products differs
        assert (r - s_).abs().max().item() <= 1e-7


def test_batched_autotune_keeps_parity():
    """qed_autotune_batched times the GEMM1 tile widths on whole batched steps and stores the
    fastest in the models; the next batched run (whatever width it uses) still matches the
    oracle on instances with 128-column remainders."""
    specs = W.batched_chains(8, seed=11, dim_lo=100, dim_hi=700, n_steps=150, record_every=50)
    bases = [oracle.enumerate_basis(m) for m in specs]
    refs = [oracle.evolve(m, n_steps=150, record_every=50, basis=b, obs_ids=list(range(b.dim)))
            for m, b in zip(specs, bases)]
    models, _ = _setup(specs, "split_fp16x2")
    choice = qed.autotune_batched(models, steps=3)
    print(choice)
    assert choice.startswith("gemm1 ") and "256-wide" in choice and "128-wide" in choice
    _, rhos = _setup(specs, "split_fp16x2")
    recs = qed.evolve_batched(models, rhos, 150, record_every=50)
    torch.cuda.synchronize()
    for (rho_ref, rec_ref), r, rec in zip(refs, rhos, recs):
        assert np.abs(r.cpu().numpy() - rho_ref).max() <= 1e-5
        assert np.abs(rec.cpu().numpy() - rec_ref).max() <= 1e-6
    with pytest.raises(qed.QedError):
        qed.autotune_batched([models[0], models[0]])
    m64, _ = _setup(specs[:1], "fp64")
    with pytest.raises(qed.QedError):
        qed.autotune_batched(m64)


_WIDTH_REFS = {}


@pytest.mark.parametrize("widths", [(256, 256), (128, 256), (128, 128)])
def test_batched_tile_widths_keep_parity(widths):
    """The grouped launches with each pair of tile widths (set on every model with
    qed_set_plan): uneven chains with 128-column remainders and up to six jumps."""
    specs = W.batched_chains(6, seed=13, dim_lo=60, dim_hi=660, n_steps=120, record_every=60)
    if "refs" not in _WIDTH_REFS:
        _WIDTH_REFS["refs"] = []
        for m in specs:
            b = oracle.enumerate_basis(m)
            _WIDTH_REFS["refs"].append(oracle.evolve(m, n_steps=120, record_every=60, basis=b,
                                                     obs_ids=list(range(b.dim))))
    models, rhos = _setup(specs, "split_fp16x2")
    for gm in models:
        gm.set_plan(widths[0], 1, widths[1], 1)
    recs = qed.evolve_batched(models, rhos, 120, record_every=60)
    torch.cuda.synchronize()
    for (rho_ref, rec_ref), gm, r, rec in zip(_WIDTH_REFS["refs"], models, rhos, recs):
        assert np.abs(r.cpu().numpy() - rho_ref).max() <= 1e-5, (widths, gm.dim)
        assert np.abs(rec.cpu().numpy() - rec_ref).max() <= 1e-6, (widths, gm.dim)


def test_batched_argument_errors():
    specs = W.batched_chains(2, seed=1, dim_lo=32, dim_hi=64)
    models, rhos = _setup(specs, "split_fp16x2")
    with pytest.raises(qed.QedError):
        qed.evolve_batched([models[0], models[0]], [rhos[0], rhos[0].clone()], 5)
    m64, r64 = _setup(specs[:1], "fp64")
    with pytest.raises(qed.QedError):
        qed.evolve_batched([models[0], m64[0]], [rhos[0], r64[0]], 5)
    # split precision: a rho that is not a density matrix is reported by the call itself
    bad = rhos[1].clone()
    bad[0, 1] += 1e-3
    with pytest.raises(qed.QedError) as ei:
        qed.evolve_batched(models, [rhos[0], bad], 5)
    assert ei.value.status == qed.QED_EINVAL
