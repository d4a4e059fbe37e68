"""Writes the stored oracle trajectories used by the full-length GPU parity tests.

Calls only the FP64 oracle (and the seeded workload module).  Usage:
    python tests/golden/make_golden.py hb_shaped_d512
    python tests/golden/make_golden.py jch2_d36
    python tests/golden/make_golden.py batched_chains_d53_1008
    python tests/golden/make_golden.py adjoint_lattice_24x24_d1153
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import qed_workloads as W  # noqa: E402

def hb_shaped_d512():
    """The hydrogen-bond-shaped workload (dim 512), 10000 steps of dt 0.05: populations
    every 100 steps and the whole final density matrix (512 x 512 complex128)."""
    m = W.hb_shaped()
    b = oracle.enumerate_basis(m)
    t0 = time.time()
    rho, rec = oracle.evolve(m, basis=b, obs_ids=list(range(b.dim)))
    np.savez_compressed(os.path.join(HERE, "hb_shaped_d512_oracle.npz"), records=rec, rho=rho,
                        trace=np.trace(rho).real, seconds=time.time() - t0)


def batched_chains_d53_1008():
    """The first 16 instances of the batched-chains workload (seed 0: the same instances the
    512-instance bench run starts with; dims 53..1008), 1000 steps of dt 0.1 each:
    populations every 100 steps and eight rows of each final density matrix (evenly spaced,
    first and last included).  Instance i's arrays are stored under the suffix _i."""
    specs = W.batched_chains(16, seed=0)
    out = {}
    t0 = time.time()
    for i, m in enumerate(specs):
        b = oracle.enumerate_basis(m)
        rho, rec = oracle.evolve(m, basis=b, obs_ids=list(range(b.dim)))
        rows = np.unique(np.linspace(0, b.dim - 1, 8).round().astype(np.int64))
        out[f"records_{i}"] = rec
        out[f"rows_{i}"] = rows
        out[f"rho_rows_{i}"] = rho[rows]
        out[f"trace_{i}"] = np.trace(rho).real
        print(f"instance {i}: dim {b.dim}, {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(os.path.join(HERE, "batched_chains_d53_1008_oracle.npz"), n=len(specs),
                        seconds=time.time() - t0, **out)


def jch2_d36():
    """Two coupled JC cavities (dim 36), 20000 steps of dt 0.1: populations every 100 steps
    and the whole final density matrix."""
    m = W.jch_two_cavities()
    b = oracle.enumerate_basis(m)
    t0 = time.time()
    rho, rec = oracle.evolve(m, basis=b, obs_ids=list(range(b.dim)))
    np.savez_compressed(os.path.join(HERE, "jch2_d36_oracle.npz"), records=rec, rho=rho,
                        trace=np.trace(rho).real, seconds=time.time() - t0)


def lattice_32x32_d2049():
    """The 32 x 32 lattice (dim 2049), 2000 steps of dt 0.1: the vacuum, photon and atom
    populations every 100 steps (all 2049 diagonal entries) and rows of the final rho."""
    m = W.lattice()
    b = oracle.enumerate_basis(m)
    t0 = time.time()
    rho, rec = oracle.evolve(m, basis=b, obs_ids=list(range(b.dim)))
    rows = [0, 1, 2, 1 + 2 * (16 * 32 + 16), 2 + 2 * (16 * 32 + 16), 2047, 2048]
    np.savez_compressed(os.path.join(HERE, "lattice_32x32_d2049_oracle.npz"), records=rec,
                        rho_rows=np.array(rows), rho_sample=rho[rows], trace=np.trace(rho).real,
                        seconds=time.time() - t0)


def adjoint_lattice_24x24_d1153():
    """The 24 x 24 adjoint workload (dim 1153, 1000 steps of dt 0.1): the loss (photon +
    atom population of the corner cavity) and its gradients with respect to all 576 g,
    1104 zeta and 576 leak rates, from the oracle's discrete adjoint."""
    m = W.adjoint_lattice()
    b = oracle.enumerate_basis(m)
    w = oracle.loss_diag(m, b, **m["loss_states"])
    t0 = time.time()
    loss, gg, gz, gj = oracle.adjoint_gradients(m, w, basis=b)
    np.savez_compressed(os.path.join(HERE, "adjoint_lattice_24x24_d1153_oracle.npz"), loss=loss, grad_g=gg,
                        grad_zeta=gz, grad_gamma=gj, seconds=time.time() - t0)


if __name__ == "__main__":
    for name in sys.argv[1:]:
        globals()[name]()
