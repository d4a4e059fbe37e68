"""Batched evolution of uneven instances (qed_evolve_batched): every instance against the
FP64 oracle, and against the same model evolved on its own."""
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


@pytest.mark.parametrize("precision,tol_rho,tol_pop", [("split_fp16x2", 1e-5, 1e-6), ("fp64", 1e-12, 1e-12)])
def test_batched_instances_match_oracle(precision, tol_rho, tol_pop):
    """16 seeded chains (dims 32..256, several tiles, ragged), 300 steps, records every 50."""
    specs = W.batched_chains(16, seed=3, dim_lo=32, dim_hi=256, n_steps=300, record_every=50)
    models, rhos = _setup(specs, precision)
    recs = qed.evolve_batched(models, rhos, 300, record_every=50)
    torch.cuda.synchronize()
    worst = 0.0
    for m, gm, r, rec in zip(specs, models, rhos, recs):
        b = oracle.enumerate_basis(m)
        U = None
        if precision == "fp64":
            U = gm.get_U().cpu().numpy()
        rho_ref, rec_ref = oracle.evolve(m, n_steps=300, record_every=50, basis=b, U=U,
                                         obs_ids=list(range(b.dim)))
        err = np.abs(r.cpu().numpy() - rho_ref).max()
        perr = np.abs(rec.cpu().numpy() - rec_ref).max()
        worst = max(worst, err)
        assert err <= tol_rho and perr <= tol_pop, (m["name"], err, perr)
    print(f"batched {precision}: worst max|drho| over 16 instances = {worst:.2e}")


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


def test_batched_argument_errors():
    specs = W.batched_chains(2, seed=1, dim_lo=32, dim_hi=64)
    models, rhos = _setup(specs, "split_fp16x2")
    with pytest.raises(qed.QedError):
        qed.evolve_batched([models[0], models[0]], [rhos[0], rhos[0].clone()], 5)
    m64, r64 = _setup(specs[:1], "fp64")
    with pytest.raises(qed.QedError):
        qed.evolve_batched([models[0], m64[0]], [rhos[0], r64[0]], 5)
