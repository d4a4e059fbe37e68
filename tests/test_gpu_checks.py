"""The debug build with device bounds checks (QED_CHECKS=1, libqed_checks.so): every index the
split step's kernels read from a table (jump sources of the per-jump, padded and list
tables, the warp-shared long merges, GEMM1's output rows) is checked before it is used, a
failed check is reported by qed_sync_status and the access skipped.  Run on the workloads'
table kinds, the checked build must report nothing and give the regular build's results."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")

# one run per table kind: per-jump table (dim 512, three jumps), lists with long merges
# (lattice, 64 leaks into the vacuum), padded table and per-jump table in a batch
_SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    import paper_2403_07042_gb300 as qed
    import qed_workloads as W
    if {lib!r}:
        qed.LIB_PATH = {lib!r}
    out = {{}}
    for name, m, steps in [("hb", W.hb_shaped(), 60), ("lattice", W.lattice(8, 8, seed=2), 80)]:
        gm = qed.Model(m, precision="split_fp16x2")
        rho = torch.tensor(W.random_density(gm.dim, seed=6, rank=3), dtype=torch.complex128, device="cuda")
        gm.evolve(rho, steps)
        gm.sync()
        out[name] = rho.cpu().numpy()
    specs = W.batched_chains(5, seed=21, dim_lo=40, dim_hi=300, n_steps=50)
    models = [qed.Model(s, precision="split_fp16x2") for s in specs]
    rhos = [torch.tensor(W.random_density(gm.dim, seed=2, rank=2), dtype=torch.complex128, device="cuda")
            for gm in models]
    qed.evolve_batched(models, rhos, 50)
    for i, (gm, r) in enumerate(zip(models, rhos)):
        gm.sync()
        out[f"batch{{i}}"] = r.cpu().numpy()
    np.savez({path!r}, **out)
""")


def _run(lib, path):
    script = _SCRIPT.format(root=ROOT, lib=lib, path=path)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


def test_checked_build_reports_nothing_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    plain_lib = build.build()
    checked_lib = build.build(checks=True)
    assert checked_lib != plain_lib and os.path.exists(checked_lib)
    got = _run(checked_lib, str(tmp_path / "checked.npz"))
    ref = _run(plain_lib, str(tmp_path / "plain.npz"))
    assert set(got.files) == set(ref.files)
    for k in ref.files:
        # the checks only guard loads and stores; the arithmetic is the same code
        assert np.abs(got[k] - ref[k]).max() <= 1e-12, k
