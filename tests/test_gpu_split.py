"""GPU checks of the split-precision path: the tcgen05 product against an FP64 reference
of the same three-term FP16 product, and the increment-form evolution against the FP64
oracle (max|drho| <= 1e-5 and populations <= 1e-6, the bars of the method's accuracy
contract)."""
import os

import numpy as np
import pytest

import oracle
import qed_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
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


def _planes(rng, rows, K, scale):
    x = rng.standard_normal((rows, K)) * scale
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float64)).astype(np.float16)
    return np.stack([hi, lo])


def _planes3(rng, rows, K, scale):
    x = rng.standard_normal((rows, K)) * scale
    hi = x.astype(np.float16)
    r = x - hi.astype(np.float64)
    mid = r.astype(np.float16)
    lo = (r - mid.astype(np.float64)).astype(np.float16)
    return np.stack([hi, mid, lo])


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (256, 384, 512, 1), (256, 128, 1024, 3),
                                          (384, 256, 256, 4)])
def test_tc_gemm_three_term_product(M, N, K, splits):
    """out = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T, checked elementwise against FP64
    within the FP32 accumulation bound 3K * 2^-23 * (|A_hi| + |A_lo|)(|B_hi| + |B_lo|)^T."""
    rng = np.random.default_rng(M + N + K + splits)
    A = _planes(rng, M, K, 1.0)
    B = _planes(rng, N, K, 1.0)
    out = qed.tc_gemm(_cuda(A), _cuda(B), splits=splits).cpu().numpy().astype(np.float64)
    Ah, Al = A[0].astype(np.float64), A[1].astype(np.float64)
    Bh, Bl = B[0].astype(np.float64), B[1].astype(np.float64)
    want = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    bound = 3 * K * 2.0 ** -23 * ((np.abs(Ah) + np.abs(Al)) @ (np.abs(Bh) + np.abs(Bl)).T)
    got = out.sum(axis=0)
    assert out.shape == (splits, M, N)
    assert np.all(np.abs(got - want) <= bound)
    print(f"tc_gemm {M}x{N}x{K}/{splits}: max err / (sum|ab| 2^-24) = "
          f"{(np.abs(got - want) / (bound / (6 * K))).max():.1f}")
    # the lo terms are really there: the result is far closer to the three-term product
    # than to hi*hi alone
    assert np.abs(got - want).max() < 0.1 * np.abs(want - Ah @ Bh.T).max()


def test_tc_gemm_four_segments_three_planes():
    """The step's GEMM1 form: A in three pieces, B in two, four plane pairs."""
    rng = np.random.default_rng(7)
    M, N, K = 256, 128, 256
    A = _planes3(rng, M, K, 1.0)
    B = _planes(rng, N, K, 1.0)
    seg = ((0, 0), (0, 1), (1, 0), (2, 0))
    out = qed.tc_gemm(_cuda(A), _cuda(B), segments=seg, splits=2).cpu().numpy().astype(np.float64).sum(0)
    Af = A.astype(np.float64)
    Bf = B.astype(np.float64)
    want = sum(Af[p] @ Bf[q].T for p, q in seg)
    bound = 4 * K * 2.0 ** -23 * (np.abs(Af).sum(0) @ np.abs(Bf).sum(0).T)
    assert np.all(np.abs(out - want) <= bound)


def test_tc_gemm_rejects_bad_shapes():
    a = torch.zeros((2, 100, 64), dtype=torch.float16, device="cuda")
    b = torch.zeros((2, 128, 64), dtype=torch.float16, device="cuda")
    with pytest.raises(qed.QedError):
        qed.tc_gemm(a, b)
    b2 = torch.zeros((2, 128, 64), dtype=torch.float16, device="cuda")
    with pytest.raises(qed.QedError):
        qed.tc_gemm(b2, b2, segments=((0, 2),))


def _evolve(model, n_steps, precision, rho0=None, U=None, record_every=0, obs=None):
    b = oracle.enumerate_basis(model)
    gm = qed.Model(model, precision=precision)
    if U is not None:
        gm.set_U(_cuda(U))
    rho = _cuda(oracle.initial_density(model, b) if rho0 is None else rho0)
    rec = gm.evolve(rho, n_steps, record_every=record_every, obs_ids=obs)
    gm.sync()
    return rho.cpu().numpy(), (None if rec is None else rec.cpu().numpy())


@pytest.mark.parametrize("make,steps", [
    (lambda: W.jch_two_cavities(), 2000),
    (lambda: W.hb_shaped(), 500),
    (lambda: W.lattice(6, 5, seed=7, gamma=5e-3), 300),
    (lambda: W.chain_instance(np.random.default_rng(4), 100, 257), 300),
])
def test_split_parity_reduced_steps(make, steps):
    """Split precision vs the oracle on several tiles and ragged dimensions."""
    m = make()
    b = oracle.enumerate_basis(m)
    obs = list(range(b.dim))
    rho_ref, rec_ref = oracle.evolve(m, n_steps=steps, record_every=50, basis=b, obs_ids=obs)
    rho, rec = _evolve(m, steps, "split_fp16x2", record_every=50, obs=obs)
    err, perr = np.abs(rho - rho_ref).max(), np.abs(rec - rec_ref).max()
    print(f"{m['name']} D={b.dim} steps={steps}: max|drho|={err:.2e} max|dpop|={perr:.2e}")
    assert err <= RHO_TOL and perr <= POP_TOL


def test_split_random_mixed_state():
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=9)
    rho_ref = oracle.evolve(m, rho0=rho0, n_steps=200, basis=b, return_records=False)
    rho, _ = _evolve(m, 200, "split_fp16x2", rho0=rho0)
    assert np.abs(rho - rho_ref).max() <= RHO_TOL


def test_split_jch2_full_length():
    """Two JC cavities (dim 36, padded to one 128 tile), all 20000 steps."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    obs = list(range(b.dim))
    rho_ref, rec_ref = oracle.evolve(m, basis=b, obs_ids=obs)
    rho, rec = _evolve(m, m["n_steps"], "split_fp16x2", record_every=m["record_every"], obs=obs)
    err, perr = np.abs(rho - rho_ref).max(), np.abs(rec - rec_ref).max()
    print(f"jch2 split 20000 steps: max|drho|={err:.2e} max|dpop|={perr:.2e}")
    assert err <= RHO_TOL and perr <= POP_TOL


def test_split_hb_shaped_full_length_against_stored_oracle():
    """The dim-512 workload at full length (10000 steps), in the configuration the bench
    times, against the stored oracle trajectory (populations every 100 steps and every
    element of the final 512 x 512 rho), written by tests/golden/make_golden.py."""
    g = np.load(os.path.join(GOLDEN, "hb_shaped_d512_oracle.npz"))
    m = W.hb_shaped()
    rho, rec = _evolve(m, m["n_steps"], "split_fp16x2", record_every=m["record_every"],
                       obs=list(range(512)))
    assert g["rho"].shape == rho.shape == (512, 512)
    err = np.abs(rho - g["rho"]).max()
    perr = np.abs(rec - g["records"]).max()
    print(f"hb_shaped split 10000 steps: max|drho| (all 262144 elements)={err:.2e} max|dpop|={perr:.2e}")
    assert perr <= POP_TOL and err <= RHO_TOL
    assert abs(np.trace(rho).real - 1.0) <= 1e-7
    assert np.abs(rho - rho.conj().T).max() <= 1e-12


def test_split_invariants_and_renormalisation():
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    gm = qed.Model(m, precision="split_fp16x2")
    gm.set_renorm_every(50)
    rho = _cuda(W.random_density(b.dim, seed=3, rank=4))
    gm.evolve(rho, 400)
    gm.sync()
    r = rho.cpu().numpy()
    assert abs(np.trace(r).real - 1.0) <= 1e-12
    assert np.abs(r - r.conj().T).max() <= 1e-15
    assert np.linalg.eigvalsh(r).min() >= -1e-6


@pytest.mark.parametrize("defect", ["not_hermitian", "trace_half", "trace_two"])
def test_split_rejects_non_density_input(defect):
    """The split path needs a Hermitian, unit-trace rho (its first product reads rho^T as
    conj(rho), the second forms a Hermitian X, the renormalisation divides by the trace):
    other inputs are reported as EINVAL by qed_sync_status.  The FP64 path takes them and
    matches the oracle's step of the same matrix."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    rho0 = W.random_density(b.dim, seed=11)
    if defect == "not_hermitian":
        rho0 = rho0.copy()
        rho0[3, 7] += 1e-3j
    else:
        rho0 = rho0 * (0.5 if defect == "trace_half" else 2.0)
    gs = qed.Model(m, precision="split_fp16x2")
    rho = _cuda(rho0)
    gs.evolve(rho, 10)
    with pytest.raises(qed.QedError) as ei:
        gs.sync()
    assert ei.value.status == qed.QED_EINVAL
    # the model stays usable: a proper density matrix afterwards passes
    ok = _cuda(W.random_density(b.dim, seed=12))
    gs.evolve(ok, 10)
    gs.sync()
    # the FP64 path accepts any matrix and follows the oracle's map of it
    U = oracle.propagator(oracle.hamiltonian(m, b), m["dt"])
    rho_ref = oracle.evolve(m, rho0=rho0, n_steps=10, U=U, basis=b, return_records=False)
    r64, _ = _evolve(m, 10, "fp64", rho0=rho0, U=U)
    assert np.abs(r64 - rho_ref).max() <= 1e-12


def test_split_accepts_its_own_output():
    """A state the split path returned mid-way between renormalisations (here 150 steps
    with the default interval of 100) passes the density check of the next call."""
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    gs = qed.Model(m, precision="split_fp16x2")
    rho = _cuda(W.random_density(b.dim, seed=4, rank=3))
    gs.evolve(rho, 150)
    gs.sync()
    gs.evolve(rho, 20)
    gs.sync()


def test_split_nonfinite_is_reported():
    m = W.jch_two_cavities()
    gm = qed.Model(m, precision="split_fp16x2")
    gm.set_renorm_every(1)
    rho = torch.zeros((36, 36), dtype=torch.complex128, device="cuda")
    rho[0, 0] = float("nan")
    gm.evolve(rho, 2)
    with pytest.raises(qed.QedError) as ei:
        gm.sync()
    assert ei.value.status == qed.QED_ENUMERIC


def test_split_two_bond_size_d4096_against_fp64_gpu():
    """The size of the paper's two-hydrogen-bond run (Sec. 3.1, dim 2^12 = 4096, seven jump
    operators): 20 split steps against 20 FP64 GPU steps (the FP64 path matches the oracle
    to 1e-12 at smaller sizes; an oracle step at this size takes seconds of CPU), then the
    invariants after the paper's 3000 iterations."""
    m = W.hb_two_bonds()
    g64 = qed.Model(m, precision="fp64")
    gs = qed.Model(m, precision="split_fp16x2")
    assert g64.dim == gs.dim == 4096
    i0 = gs.initial_index()
    rho0 = torch.zeros((4096, 4096), dtype=torch.complex128, device="cuda")
    rho0[i0, i0] = 1.0
    r64, rs = rho0.clone(), rho0.clone()
    g64.evolve(r64, 20)
    gs.evolve(rs, 20)
    gs.sync()
    assert float((r64 - rs).abs().max()) <= RHO_TOL
    gs.evolve(rs, 2980)
    gs.sync()
    r = rs.cpu().numpy()
    assert abs(np.trace(r).real - 1.0) <= 1e-7
    # the step keeps rho Hermitian to the double-float rounding of its element kernels
    # (~1e-13 per step); the last symmetrisation was 80 steps before the end
    assert np.abs(r - r.conj().T).max() <= 1e-10
    assert np.real(np.diag(r)).min() >= -1e-6


@pytest.mark.parametrize("make,steps", [(lambda: W.jch_two_cavities(), 400), (lambda: W.hb_shaped(), 200)])
def test_autotuned_plan_keeps_parity(make, steps):
    """qed_autotune times the tile widths and split-K factors of both products and keeps the
    fastest; whatever it picks, the step still matches the oracle."""
    m = make()
    b = oracle.enumerate_basis(m)
    gm = qed.Model(m, precision="split_fp16x2")
    choice = gm.autotune(10)
    print(f"{m['name']}: {choice}")
    assert choice.startswith("gemm1 ")
    obs = list(range(b.dim))
    rho_ref, rec_ref = oracle.evolve(m, n_steps=steps, record_every=50, basis=b, obs_ids=obs)
    rho = _cuda(oracle.initial_density(m, b))
    rec = gm.evolve(rho, steps, record_every=50, obs_ids=obs)
    gm.sync()
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= RHO_TOL
    assert np.abs(rec.cpu().numpy() - rec_ref).max() <= POP_TOL


def test_split_runs_are_bitwise_repeatable():
    """Every reduction of the split path has a fixed order (split-K slices summed in cluster
    rank order, block reductions in shared memory, no atomics), so two runs from the same
    state give the same bits: single models (the headline workload and a ragged dim-129
    lattice), a batch of uneven chains, and the adjoint's loss and gradients."""
    for m in (W.hb_shaped(), W.lattice(8, 8, seed=2)):
        gm = qed.Model(m, precision="split_fp16x2")
        rho0 = _cuda(W.random_density(gm.dim, seed=8, rank=4))
        r1, r2 = rho0.clone(), rho0.clone()
        gm.evolve(r1, 300)
        gm.evolve(r2, 300)
        gm.sync()
        assert torch.equal(r1, r2), m["name"]
    specs = W.batched_chains(6, seed=9, dim_lo=40, dim_hi=400, n_steps=100)
    models = [qed.Model(s, precision="split_fp16x2") for s in specs]
    runs = []
    for _ in range(2):
        rhos = [_cuda(W.random_density(gm.dim, seed=3, rank=2)) for gm in models]
        qed.evolve_batched(models, rhos, 100)
        runs.append(rhos)
    torch.cuda.synchronize()
    for a, b in zip(*runs):
        assert torch.equal(a, b)
    m = W.adjoint_lattice(6, 6, seed=1)
    gm = qed.Model(m, precision="split_fp16x2")
    rho0 = _cuda(oracle.initial_density(m, oracle.enumerate_basis(m)))
    w = torch.zeros(gm.dim, dtype=torch.float64, device="cuda")
    w[1] = 1.0
    g1 = [x.clone() for x in gm.adjoint(rho0, 50, w, checkpoint_every=20)]
    g2 = [x.clone() for x in gm.adjoint(rho0, 50, w, checkpoint_every=20)]
    for a, b in zip(g1, g2):
        assert torch.equal(a, b)


_PLAN_REF = {}


def _plan_ref(key, make, steps):
    if key not in _PLAN_REF:
        m = make()
        b = oracle.enumerate_basis(m)
        rho0 = W.random_density(b.dim, seed=12, rank=3)
        rho_ref, rec_ref = oracle.evolve(m, rho0=rho0, n_steps=steps, record_every=steps // 2, basis=b,
                                         obs_ids=list(range(b.dim)))
        _PLAN_REF[key] = (m, rho0, rho_ref, rec_ref)
    return _PLAN_REF[key]


@pytest.mark.parametrize("plan", [(256, 1, 256, 1), (256, 2, 256, 2), (128, 4, 256, 4), (256, 1, 128, 1),
                                  (128, 8, 128, 2), (256, 4, 256, 1)])
@pytest.mark.parametrize("key,make,steps", [
    ("lattice_d129", lambda: W.lattice(8, 8, seed=2), 150),
    ("hb_d512", lambda: W.hb_shaped(), 100),
    ("chain_d600", lambda: W.chain_instance(np.random.default_rng(4), 600, 600), 60),
])
def test_tile_plans_keep_parity(key, make, steps, plan):
    """Every tile plan qed_set_plan accepts gives the oracle's step: 128- and 256-wide tiles
    for both products (a 256-wide GEMM2 tile covers two 64-column groups, the second past D
    at dim 129; the last 256-wide GEMM1 column tile at dims 129 and 600 has 128 columns),
    1 to 8 K slices summed in the cluster, from a random mixed state (every element
    nonzero)."""
    m, rho0, rho_ref, rec_ref = _plan_ref(key, make, steps)
    gm = qed.Model(m, precision="split_fp16x2")
    kb = 2 * (-(-gm.dim // 128) * 128) // 64  # 64-wide K blocks of both products (K = 2 Dp)

    def splits_fit(sp):
        return -(-kb // -(-kb // sp)) == sp
    if not (splits_fit(plan[1]) and splits_fit(plan[3])):
        # e.g. 8 slices of 20 K blocks: the slices would not be equal powers of two
        with pytest.raises(qed.QedError) as ei:
            gm.set_plan(*plan)
        assert ei.value.status == qed.QED_EINVAL
        return
    gm.set_plan(*plan)
    rho = _cuda(rho0)
    rec = gm.evolve(rho, steps, record_every=steps // 2, obs_ids=list(range(gm.dim)))
    gm.sync()
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= RHO_TOL, plan
    assert np.abs(rec.cpu().numpy() - rec_ref).max() <= POP_TOL, plan


def test_set_plan_rejects_bad_plans():
    gm = qed.Model(W.jch_two_cavities(), precision="split_fp16x2")
    for bad in [(64, 1, 128, 1), (128, 3, 128, 1), (128, 1, 128, 8), (128, 16, 128, 1), (256, 1, 512, 1)]:
        with pytest.raises(qed.QedError) as ei:
            gm.set_plan(*bad)
        assert ei.value.status == qed.QED_EINVAL
    g64 = qed.Model(W.jch_two_cavities(), precision="fp64")
    with pytest.raises(qed.QedError) as ei:
        g64.set_plan(128, 1, 128, 1)
    assert ei.value.status == qed.QED_EUNSUPPORTED


def test_profile_replay():
    """qed_profile_replay times each kernel of the Lie step replayed back to back; it leaves
    the caller's rho untouched and the model's next evolution matches the oracle."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    gm = qed.Model(m, precision="split_fp16x2")
    rho = _cuda(oracle.initial_density(m, b))
    before = rho.clone()
    kern = gm.profile_replay(rho, 20)
    assert list(kern) == ["gemm1_tc", "gemm2_tc_v", "dissipate"] and all(v > 0 for v in kern.values())
    assert torch.equal(rho, before)
    rho_ref = oracle.evolve(m, n_steps=100, basis=b, return_records=False)
    gm.evolve(rho, 100)
    gm.sync()
    assert np.abs(rho.cpu().numpy() - rho_ref).max() <= RHO_TOL
    g64 = qed.Model(m, precision="fp64")
    with pytest.raises(qed.QedError) as ei:
        g64.profile_replay(before, 5)
    assert ei.value.status == qed.QED_EUNSUPPORTED
