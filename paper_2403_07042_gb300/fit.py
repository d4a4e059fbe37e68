"""Parameter fitting on top of the binding (point 4 of Sec. 2: choosing a model's
parameters so that its dynamics match data), driven by qed_adjoint's gradients.

This is the one module of the package that does arithmetic of its own on the host and in
eager torch: the least-squares loss of the final populations, their residual as the
adjoint's observable, and a steepest-descent line search over the couplings.  The master
equation itself (forward steps and the adjoint) runs in libqed's kernels.
"""
from __future__ import annotations

import numpy as np

from . import Model


def fit_final_populations(model, target, n_steps, names=("g",), precision="fp64", rho0=None, iters=60,
                          step=1e-3, tol=1e-24, checkpoint_every=None):
    """Fits couplings to measured final populations (point 4 of Sec. 2: choosing the model's
    parameters to match data): least squares F(theta) = sum_k (p_k(theta) - target_k)^2 with
    p = diag rho after n_steps, theta the couplings listed in `names` ("g", "zeta").  The
    gradient comes from one qed_adjoint call with obs_diag = 2 (p - target), since
    dF/dtheta = sum_k 2 (p_k - target_k) dp_k/dtheta; steepest descent with a step that
    doubles after a success and halves after a failure.  `model` is a model dictionary;
    target a length-D array.  Returns (fitted model dictionary, list of F per iteration)."""
    import torch
    m = dict(model)
    tgt = torch.tensor(np.asarray(target, dtype=np.float64), device="cuda")  # a copy: target may be read-only
    k = checkpoint_every or n_steps

    def run(mm):
        gm = Model(mm, precision=precision)
        r0 = rho0
        if r0 is None:
            r0 = torch.zeros((gm.dim, gm.dim), dtype=torch.complex128, device="cuda")
            i0 = gm.initial_index()
            r0[i0, i0] = 1.0
        rho = r0.clone()
        gm.evolve(rho, n_steps)
        gm.sync()
        p = torch.real(torch.diagonal(rho)).contiguous()
        return gm, r0, p, float(torch.sum((p - tgt) ** 2))

    def theta(mm):
        return np.concatenate([np.asarray(mm[n], dtype=np.float64) for n in names])

    def with_theta(mm, th):
        out, i = dict(mm), 0
        for n in names:
            c = len(mm[n])
            out[n] = [float(x) for x in th[i:i + c]]
            i += c
        return out

    gm, r0, p, F = run(m)
    hist = [F]
    for _ in range(iters):
        if F <= tol:
            break
        _, gg, gz, _ = gm.adjoint(r0, n_steps, 2.0 * (p - tgt), checkpoint_every=k)
        grads = {"g": gg.cpu().numpy(), "zeta": gz.cpu().numpy()}
        gvec = np.concatenate([grads[n] for n in names])
        gnorm = np.linalg.norm(gvec)
        if not gnorm > 0:
            break
        th = theta(m)
        while True:
            trial = with_theta(m, th - step * gvec / gnorm)
            gm2, r2, p2, F2 = run(trial)
            if F2 < F:
                m, gm, r0, p, F = trial, gm2, r2, p2, F2
                step *= 2.0
                break
            gm2.close()
            step *= 0.5
            if step < 1e-15:
                break
        hist.append(F)
        if step < 1e-15:
            break
    return m, hist
