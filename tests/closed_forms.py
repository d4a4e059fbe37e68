"""Closed-form solutions used as pins (independent of the oracle and of the library)."""
import numpy as np


def lattice_single_excitation_state(L, Wd, omega, g, zeta, t, start):
    """One excitation on an L x Wd grid, atoms resonant with the cavities: the hopping
    matrix has the separable open-boundary modes phi_p(i) phi_q(j), energies
    2 zeta (cos k_p + cos k_q); each mode is a 2 x 2 JC block [[omega + eps, g], [g, omega]]
    whose exponential is written out.  Returns amplitudes in the ground + single basis."""
    def modes(n):
        k = np.pi * np.arange(1, n + 1) / (n + 1)
        return np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(np.arange(1, n + 1), k)), k
    phi_i, ki = modes(L)
    phi_j, kj = modes(Wd)
    i0, j0 = start
    eps = 2 * zeta * (np.cos(ki)[:, None] + np.cos(kj)[None, :])
    # exp(-i t [[w+e, g], [g, w]]) applied to (1, 0): centre c = w + e/2, half-splitting r
    c = omega + eps / 2
    r = np.sqrt((eps / 2) ** 2 + g * g)
    ph = np.exp(-1j * c * t)
    a_ph = ph * (np.cos(r * t) - 1j * (eps / 2) / r * np.sin(r * t))
    a_at = ph * (-1j * g / r * np.sin(r * t))
    w0 = phi_i[i0][:, None] * phi_j[j0][None, :]
    photon = phi_i @ (w0 * a_ph) @ phi_j.T
    atom = phi_i @ (w0 * a_at) @ phi_j.T
    psi = np.zeros(1 + 2 * L * Wd, dtype=complex)
    psi[1::2] = photon.reshape(-1)
    psi[2::2] = atom.reshape(-1)
    return psi


def plane_photon_state(L, Wd, omega, zeta, t, start):
    """One photon on an L x Wd grid of cavities without atoms (open boundaries): the hopping
    matrix has the separable modes phi_p(i) phi_q(j), phi_p(i) = sqrt(2/(n+1)) sin(k_p (i+1)),
    k_p = pi p/(n+1), energies omega + 2 zeta (cos k_p + cos k_q).  Returns the amplitude
    grid psi[i, j] at time t from the photon in cavity `start`."""
    def modes(n):
        k = np.pi * np.arange(1, n + 1) / (n + 1)
        return np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(np.arange(1, n + 1), k)), k
    phi_i, ki = modes(L)
    phi_j, kj = modes(Wd)
    i0, j0 = start
    e = omega + 2 * zeta * (np.cos(ki)[:, None] + np.cos(kj)[None, :])
    w = phi_i[i0][:, None] * phi_j[j0][None, :] * np.exp(-1j * e * t)
    return phi_i @ w @ phi_j.T
