"""Error paths that are tested without faulting the GPU: a bounded device wait that runs out
(the wait-gate hook: a flag that nothing clears) and device allocations that fail (the
allocation-budget hook).  Each returns its status code and leaves the library usable."""
import gc

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
    yield
    qed.set_alloc_budget(-1)


def _rho0(m, b):
    return torch.from_numpy(oracle.initial_density(m, b)).cuda()


@pytest.mark.parametrize("make", [lambda: W.jch_two_cavities(), lambda: W.hb_shaped()])
def test_wait_gate_times_out_then_model_recovers(make):
    m = make()
    b = oracle.enumerate_basis(m)
    gm = qed.Model(m, precision="split_fp16x2")
    gm.set_wait_gate(True, budget_cycles=20000)
    rho = _rho0(m, b)
    gm.evolve(rho, 6)
    with pytest.raises(qed.QedError) as ei:
        gm.sync()
    assert ei.value.status == qed.QED_ETIMEOUT
    # the flag stays reported once: the next check is clean
    gm.sync()
    gm.set_wait_gate(False)
    rho = _rho0(m, b)
    rec = gm.evolve(rho, 200, record_every=50, obs_ids=list(range(b.dim)))
    gm.sync()
    rho_ref, rec_ref = oracle.evolve(m, n_steps=200, record_every=50, basis=b, obs_ids=list(range(b.dim)))
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= 1e-5
    assert np.abs(rec.cpu().numpy() - rec_ref).max() <= 1e-6


def test_wait_gate_rejected_on_fp64():
    gm = qed.Model(W.jch_two_cavities(), precision="fp64")
    with pytest.raises(qed.QedError) as ei:
        gm.set_wait_gate(True)
    assert ei.value.status == qed.QED_EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "split_fp16x2"])
def test_alloc_budget_gives_enomem_and_frees(precision):
    m = W.hb_shaped()
    qed.Model(m, precision=precision).close()  # warm-up: modules loaded, pools settled
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for budget in (0, 1 << 20, 8 << 20):
        qed.set_alloc_budget(budget)
        with pytest.raises(qed.QedError) as ei:
            qed.Model(m, precision=precision)
        assert ei.value.status == qed.QED_ENOMEM
    qed.set_alloc_budget(-1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # the failed builds freed what they had
    gm = qed.Model(m, precision=precision)
    b = oracle.enumerate_basis(m)
    rho = _rho0(m, b)
    gm.evolve(rho, 20)
    gm.sync()
    rho_ref = oracle.evolve(m, n_steps=20, basis=b, return_records=False)
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= (1e-12 if precision == "fp64" else 1e-5)


def test_alloc_budget_in_the_adjoint():
    m = W.jc_single(n_max=3, g=0.02, dt=0.1, n_steps=40)
    gm = qed.Model(m, precision="split_fp16x2")
    b = oracle.enumerate_basis(m)
    w = torch.ones(b.dim, dtype=torch.float64, device="cuda")
    qed.set_alloc_budget(0)
    with pytest.raises(qed.QedError) as ei:
        gm.adjoint(_rho0(m, b), 40, w, checkpoint_every=10)
    assert ei.value.status == qed.QED_ENOMEM
    qed.set_alloc_budget(-1)
    loss, *_ = gm.adjoint(_rho0(m, b), 40, w, checkpoint_every=10)
    assert abs(float(loss) - 1.0) <= 1e-6  # the trace of a closed unit-trace evolution


def test_alloc_budget_in_tc_gemm():
    A = torch.zeros((2, 128, 64), dtype=torch.float16, device="cuda")
    qed.set_alloc_budget(0)
    with pytest.raises(qed.QedError) as ei:
        qed.tc_gemm(A, A)
    assert ei.value.status == qed.QED_ENOMEM
    qed.set_alloc_budget(-1)
    assert float(qed.tc_gemm(A, A).abs().max()) == 0.0
