"""Host-side checks of libqed (no GPU): the library loads and exports every declared
symbol, and its C++ model builder reproduces the oracle's basis (bit-exact), Hamiltonian
and jump operators, and rejects malformed specifications."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import qed_workloads as W

qed = pytest.importorskip("paper_2403_07042_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_07042_gb300 import build
    build.build()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:qed_status|const char\s*\*)\s*(qed_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert {"qed_build", "qed_evolve", "qed_observables", "qed_last_error"} <= names
    L = qed.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


MODELS = {
    "jch2_d36": lambda: W.jch_two_cavities(),
    "hb_shaped_d512": lambda: W.hb_shaped(),
    "lattice_6x5": lambda: W.lattice(6, 5, seed=3),
    "lattice_sector": lambda: W.lattice(7, 3, atoms=False, basis_kind=4, gamma=0.0),
    "cap": lambda: W._model(n_cavities=3, atoms_per_cavity=[2, 1, 2], n_max=[2, 1, 3], basis_kind=1,
                            excitation_cap=3, g=[0.01, 0.02, 0.03, 0.04, 0.05], bonds=[(0, 1), (1, 2)],
                            zeta=[0.004, 0.006], jumps=[(0, 0, 1e-3), (1, 2, 2e-3), (0, 2, 5e-3)]),
    "first_d": lambda: W.chain_instance(np.random.default_rng(11), 32, 300),
}


@pytest.mark.parametrize("name", sorted(MODELS))
def test_basis_matches_oracle(name):
    m = MODELS[name]()
    b = oracle.enumerate_basis(m)
    digits = qed.spec_basis(m)
    assert digits.shape == b.digits.shape
    assert np.array_equal(digits, b.digits)


def test_workload_bases_match_oracle():
    for m in (W.lattice(), W.adjoint_lattice()):
        b = oracle.enumerate_basis(m)
        assert np.array_equal(qed.spec_basis(m), b.digits)
    for m in W.batched_chains(16, seed=0):
        b = oracle.enumerate_basis(m)
        assert np.array_equal(qed.spec_basis(m), b.digits)


@pytest.mark.parametrize("name", sorted(MODELS))
def test_hamiltonian_and_jumps_match_oracle(name):
    m = MODELS[name]()
    b = oracle.enumerate_basis(m)
    H = qed.spec_hamiltonian(m)
    assert np.abs(H - oracle.hamiltonian(m, b)).max() <= 1e-15
    for j, (gamma, A) in enumerate(oracle.jump_operators(m, b)):
        assert np.abs(qed.spec_jump(m, j) - A.toarray()).max() == 0.0


def test_paper_dimensions_from_builder():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "paper_dimensions.json")) as f:
        entries = json.load(f)["entries"]
    from test_oracle_pins import _golden_model
    for e in entries:
        assert qed.spec_dim(_golden_model(e["model"]))[0] == e["dim"], e["what"]


@pytest.mark.parametrize("patch,msg", [
    ({"jumps": [(0, 0, -1e-3)]}, "rate"),
    ({"jumps": [(0, 5, 1e-3)]}, "site"),
    ({"jumps": [(9, 0, 1e-3)]}, "kind"),
    ({"bonds": [(0, 7)], "zeta": [0.1]}, "bond"),
    ({"basis_kind": 7}, "basis"),
    ({"basis_kind": 3, "dim_cap": 10 ** 9}, "dim_cap"),
    ({"n_max": [-1, 2]}, "n_max"),
])
def test_malformed_specs_are_rejected(patch, msg):
    m = W.jch_two_cavities()
    m.update(patch)
    with pytest.raises(qed.QedError) as ei:
        qed.spec_dim(m) if "jumps" not in patch and "bonds" not in patch else qed.spec_hamiltonian(m)
    assert ei.value.status == qed.QED_EINVAL
    assert msg in str(ei.value)


def test_empty_sector_is_rejected():
    m = W.lattice(2, 2, atoms=False, basis_kind=4, gamma=0.0)
    m["excitation_cap"] = 9
    with pytest.raises(qed.QedError):
        qed.spec_dim(m)


@pytest.mark.parametrize("name", ["hb_shaped_d512", "lattice_6x5"])
def test_restricted_operators_match_oracle_projection(name):
    """The model on a subset of the basis (what qed_select_states builds after deleting
    states): P H P and P A_j P equal the oracle's operators restricted to the kept rows and
    columns, and d_k = sum_j gamma_j (A_j^+ A_j)_kk of the projected jumps."""
    m = W.hb_shaped() if name == "hb_shaped_d512" else W.lattice(6, 5, seed=7, gamma=5e-3)
    b = oracle.enumerate_basis(m)
    keep = np.sort(np.random.default_rng(1).choice(b.dim, size=b.dim // 3, replace=False))
    H, d = qed.spec_restricted(m, keep, -1)
    assert np.abs(H - oracle.hamiltonian(m, b)[np.ix_(keep, keep)]).max() <= 1e-15
    d_ref = np.zeros(len(keep))
    for j, (gamma, A) in enumerate(oracle.jump_operators(m, b)):
        Ak = A.toarray()[np.ix_(keep, keep)]
        Aj, _ = qed.spec_restricted(m, keep, j)
        assert np.abs(Aj - Ak).max() == 0.0
        d_ref += gamma * np.real(np.diag(Ak.conj().T @ Ak))
    assert np.abs(d - d_ref).max() <= 1e-15


def test_restricted_operators_reject_bad_lists():
    m = W.jch_two_cavities()
    with pytest.raises(qed.QedError):
        qed.spec_restricted(m, [3, 1], -1)      # not increasing
    with pytest.raises(qed.QedError):
        qed.spec_restricted(m, [0, 99], -1)     # outside the basis


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libqed.so every call raises instead of computing elsewhere."""
    import paper_2403_07042_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "libqed.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pkg.spec_dim(W.jch_two_cavities())
