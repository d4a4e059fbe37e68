"""Seeded synthetic model specifications for the cavity-QED master-equation workloads.

This module is the one piece shared by the CUDA path's Python binding, the tests, the
bench and the CPU oracle.  It only draws parameters and describes models as plain
dictionaries; it contains none of the method's arithmetic (no basis enumeration, no
Hamiltonian, no time stepping).

A model dictionary has the keys

    n_cavities        C, number of optical cavities (photon modes)
    atoms_per_cavity  list[C] of two-level atoms in each cavity
    n_max             list[C] photon-number truncation per cavity
    n_extra           number of extra two-level degrees of freedom (e.g. a particle
                      position that tunnels between two sites)
    basis_kind        0 full product, 1 excitations <= cap, 2 ground + single excitation,
                      3 first dim_cap states in (excitation, mixed-radix) order,
                      4 exactly `excitation_cap` excitations
    excitation_cap, dim_cap
    omega_c, omega_a  cavity and atom frequencies (hbar = 1)
    g                 list[A] atom-field coupling per atom (atoms numbered cavity by cavity)
    bonds, zeta       photon-hopping edges (i, j) between cavities and their amplitudes
    extra_tunnel      list[n_extra] sigma_x amplitude on each extra two-level DOF
    jumps             list of (kind, site, gamma): kind 0 = a_c, 1 = sigma_a (atom lowering),
                      2 = sigma_z on an extra DOF (dephasing), 3 = leak |G><photon_c|
    dt, n_steps, record_every
    init              pure initial basis state given by its excitations:
                      {"photons": {c: n}, "atoms": {a: 1}, "extra": {x: 1}}

The five workloads follow the model families of the paper: Jaynes-Cummings-Hubbard
cavities (Sec. 4.2, Eq. 12 for hopping), Tavis-Cummings terms shaped like the
hydrogen-bond model (Sec. 4.1, Eqs. 6-9) and the photon-motion lattice in the
single-excitation subspace (Sec. 4.2, Eqs. 10-11).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "jch_two_cavities",
    "hb_shaped",
    "lattice",
    "chain_instance",
    "batched_chains",
    "adjoint_lattice",
    "jc_single",
    "WORKLOADS",
]


def _model(**kw):
    base = dict(
        n_cavities=1, atoms_per_cavity=[0], n_max=[1], n_extra=0,
        basis_kind=0, excitation_cap=0, dim_cap=0,
        omega_c=1.0, omega_a=1.0, g=[], bonds=[], zeta=[], extra_tunnel=[],
        jumps=[], dt=0.1, n_steps=1, record_every=1,
        init={"photons": {}, "atoms": {}, "extra": {}},
    )
    base.update(kw)
    for key in ("photons", "atoms", "extra"):
        base["init"].setdefault(key, {})
    return base


def jc_single(n_max=3, g=0.01, omega=1.0, gamma=0.0, dt=0.1, n_steps=100, init_photons=0,
              init_atom=1, atom_gamma=0.0):
    """One cavity with one two-level atom (the Jaynes-Cummings model)."""
    jumps = []
    if gamma:
        jumps.append((0, 0, gamma))
    if atom_gamma:
        jumps.append((1, 0, atom_gamma))
    return _model(name="jc_single", n_cavities=1, atoms_per_cavity=[1], n_max=[n_max],
                  omega_c=omega, omega_a=omega, g=[g], jumps=jumps, dt=dt, n_steps=n_steps,
                  record_every=1,
                  init={"photons": {0: init_photons} if init_photons else {},
                        "atoms": {0: 1} if init_atom else {}})


def jch_two_cavities(n_steps=20000, record_every=100, gamma=1e-3, g=0.01, zeta=0.005):
    """Two coupled cavities, one atom each, photons truncated at n <= 2 (dim 36)."""
    jumps = [(0, 0, gamma), (0, 1, gamma)] if gamma else []
    return _model(name="jch2_d36", n_cavities=2, atoms_per_cavity=[1, 1], n_max=[2, 2],
                  omega_c=1.0, omega_a=1.0, g=[g, g], bonds=[(0, 1)], zeta=[zeta],
                  jumps=jumps, dt=0.1, n_steps=n_steps, record_every=record_every,
                  init={"atoms": {0: 1}})


def hb_shaped(seed=0, n_steps=10000, record_every=100, gamma=1e-3, gamma_pos=1e-4, tunnel=0.005):
    """Two cavities with two atoms each (n <= 3) plus a tunnelling position bit (dim 512)."""
    rng = np.random.default_rng(seed)
    g = [float(x) for x in rng.uniform(0.005, 0.02, size=4)]
    jumps = []
    if gamma:
        jumps += [(0, 0, gamma), (0, 1, gamma)]
    if gamma_pos:
        jumps += [(2, 0, gamma_pos)]
    return _model(name="hb_shaped_d512", n_cavities=2, atoms_per_cavity=[2, 2], n_max=[3, 3],
                  n_extra=1, omega_c=1.0, omega_a=1.0, g=g, extra_tunnel=[tunnel],
                  jumps=jumps, dt=0.05, n_steps=n_steps, record_every=record_every,
                  init={"atoms": {0: 1}})


def hb_two_bonds(seed=0, n_steps=3000, record_every=100, gamma=1e-3, gamma_pos=1e-4, tunnel=0.005):
    """The size of the paper's two-hydrogen-bond model (Sec. 3.1: 12 binary digits, 2^12 =
    4096 states, 3000 iterations): six two-level modes in two chains of three, an atom on
    the outer modes of each chain, two tunnelling digits; seven jump operators (loss from
    each mode, dephasing of the first tunnelling digit).  The paper prints neither its
    parameters nor its operators; this model matches its dimension, digit count and number
    of iterations."""
    rng = np.random.default_rng(seed)
    g = [float(x) for x in rng.uniform(0.005, 0.02, size=4)]
    zeta = [float(x) for x in rng.uniform(0.002, 0.01, size=4)]
    jumps = [(0, c, gamma) for c in range(6)] + [(2, 0, gamma_pos)]
    return _model(name="hb_two_bonds_d4096", n_cavities=6, atoms_per_cavity=[1, 0, 1, 1, 0, 1], n_max=[1] * 6,
                  n_extra=2, omega_c=1.0, omega_a=1.0, g=g, bonds=[(0, 1), (1, 2), (3, 4), (4, 5)], zeta=zeta,
                  extra_tunnel=[tunnel, tunnel], jumps=jumps, dt=0.05, n_steps=n_steps,
                  record_every=record_every, init={"atoms": {0: 1}})


def _grid_bonds(length, width):
    """Nearest-neighbour edges of a length x width grid, cavity c = i * width + j."""
    bonds = []
    for i in range(length):
        for j in range(width):
            c = i * width + j
            if i + 1 < length:
                bonds.append((c, (i + 1) * width + j))
            if j + 1 < width:
                bonds.append((c, c + 1))
    return bonds


def lattice(length=32, width=32, g=0.01, zeta=0.01, gamma=1e-3, dt=0.1, n_steps=2000,
            record_every=100, start=None, atoms=True, seed=None, g_range=None, zeta_range=None,
            basis_kind=2):
    """A 2-D grid of cavities with one atom each, restricted to ground + one excitation.

    Cavity (i, j) has index c = i * width + j (row-major).  With `seed` and ranges the
    couplings are drawn per cavity and per bond instead of being uniform.
    """
    n = length * width
    bonds = _grid_bonds(length, width)
    if seed is not None:
        rng = np.random.default_rng(seed)
        gs = [float(x) for x in rng.uniform(*(g_range or (0.005, 0.02)), size=n)]
        zs = [float(x) for x in rng.uniform(*(zeta_range or (0.002, 0.01)), size=len(bonds))]
    else:
        gs = [g] * n
        zs = [zeta] * len(bonds)
    if not atoms:
        gs = []
    if start is None:
        start = (length // 2, width // 2)
    c0 = start[0] * width + start[1]
    jumps = [(3, c, gamma) for c in range(n)] if gamma else []
    return _model(name=f"lattice_{length}x{width}", n_cavities=n,
                  atoms_per_cavity=[1 if atoms else 0] * n, n_max=[1] * n,
                  basis_kind=basis_kind, excitation_cap=1, omega_c=1.0, omega_a=1.0,
                  g=gs, bonds=bonds, zeta=zs, jumps=jumps, dt=dt, n_steps=n_steps,
                  record_every=record_every, init={"photons": {c0: 1}},
                  lattice=(length, width))


def photon_plane(length=81, width=51, zeta=0.1, dt=0.1, n_steps=2000, record_every=100, start=(40, 0)):
    """The photon-motion plane of Sec. 4.2 at the paper's size: one photon on a length x
    width grid of cavities without atoms (basis |i>|j>, dim = area = 4131), closed (no
    jumps), nearest-neighbour hopping zeta; start (40, 0) is the paper's symmetric initial
    state, (20, 0) its asymmetric one."""
    m = lattice(length, width, zeta=zeta, gamma=0.0, dt=dt, n_steps=n_steps, record_every=record_every,
                start=start, atoms=False, basis_kind=4)
    m["name"] = f"photon_plane_{length}x{width}"
    return m


def _product_dim(L, k, n):
    return ((n + 1) * 2 ** k) ** L


def chain_instance(rng, dim_lo=32, dim_hi=1024, n_steps=1000, record_every=100):
    """One JCH/TCH chain: D ~ U{dim_lo..dim_hi}; (L, k, n_max) redrawn until the product
    space holds at least D states; the basis keeps the first D states ordered by
    excitation number, then mixed-radix index."""
    D = int(rng.integers(dim_lo, dim_hi + 1))
    while True:
        L = int(rng.integers(2, 7))
        k = int(rng.integers(1, 4))
        n = int(rng.integers(1, 4))
        if _product_dim(L, k, n) >= D:
            break
    n_atoms = L * k
    g = [float(x) for x in rng.uniform(0.005, 0.02, size=n_atoms)]
    bonds = [(c, c + 1) for c in range(L - 1)]
    zeta = [float(x) for x in rng.uniform(0.002, 0.01, size=len(bonds))]
    gamma = float(10.0 ** rng.uniform(-4.0, -2.0))
    return _model(name=f"chain_L{L}_k{k}_n{n}_D{D}", n_cavities=L, atoms_per_cavity=[k] * L,
                  n_max=[n] * L, basis_kind=3, dim_cap=D, omega_c=1.0, omega_a=1.0, g=g,
                  bonds=bonds, zeta=zeta, jumps=[(0, c, gamma) for c in range(L)], dt=0.1,
                  n_steps=n_steps, record_every=record_every, init={"atoms": {0: 1}})


def batched_chains(n_instances=512, seed=0, dim_lo=32, dim_hi=1024, n_steps=1000,
                   record_every=100):
    """Independent chains of uneven dimension, drawn in order from one seeded stream."""
    rng = np.random.default_rng(seed)
    return [chain_instance(rng, dim_lo, dim_hi, n_steps, record_every)
            for _ in range(n_instances)]


def adjoint_lattice(length=24, width=24, seed=0, gamma=1e-3, dt=0.1, n_steps=1000,
                    checkpoint_every=None):
    """24 x 24 lattice with per-cavity g and per-bond zeta; the photon starts in the
    corner cavity (0, 0), and the loss is the photon + atom population there.  By default
    every state of the trajectory is kept for the backward pass (checkpoint_every =
    n_steps: 2 x 1000 x 21 MB = 42 GB of device memory) and nothing is recomputed."""
    m = lattice(length, width, gamma=gamma, dt=dt, n_steps=n_steps, record_every=n_steps,
                start=(0, 0), seed=seed)
    m["name"] = f"adjoint_lattice_{length}x{width}"
    m["checkpoint_every"] = n_steps if checkpoint_every is None else checkpoint_every
    m["loss_states"] = {"photons": [0], "atoms": [0]}
    return m


def fd_parameters(model, n_params=16, seed=0, radius=3):
    """Parameters for a finite-difference check: indices of g (per atom) and zeta (per
    bond) whose cavities lie within Manhattan distance `radius` of the corner (0, 0)."""
    length, width = model["lattice"]
    near = lambda c: (c // width) + (c % width) <= radius
    cand = [("g", a) for a in range(len(model["g"])) if near(a)]
    cand += [("zeta", b) for b, (i, j) in enumerate(model["bonds"]) if near(i) and near(j)]
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(cand), size=min(n_params, len(cand)), replace=False)
    return [cand[i] for i in sorted(pick)]


WORKLOADS = {
    "jch2_d36": jch_two_cavities,
    "hb_shaped_d512": hb_shaped,
    "lattice_32x32_d2049": lattice,
    "batched_chains": batched_chains,
    "adjoint_lattice_24x24_d1153": adjoint_lattice,
}


def full_product_dim(model):
    """Size of the unrestricted product space (used to size tests, not by the method)."""
    d = 2 ** model["n_extra"]
    for c in range(model["n_cavities"]):
        d *= (model["n_max"][c] + 1) * 2 ** model["atoms_per_cavity"][c]
    return d


def density_from_state(dim, index):
    """|index><index| as a complex128 numpy array (seeded inputs are pure basis states)."""
    rho = np.zeros((dim, dim), dtype=np.complex128)
    rho[index, index] = 1.0
    return rho


def random_density(dim, seed=0, rank=None):
    """A random full-rank (or rank-r) density matrix: W W^dagger / tr, W Gaussian."""
    rng = np.random.default_rng(seed)
    r = rank or dim
    w = rng.standard_normal((dim, r)) + 1j * rng.standard_normal((dim, r))
    rho = w @ w.conj().T
    return rho / np.trace(rho).real

