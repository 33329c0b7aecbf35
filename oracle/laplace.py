"""Laplace approximation of log Z for the MLP (emulator-style) likelihood.

Test infrastructure, like the rest of oracle/: a second, approximate route to
the evidence of the MLP likelihood, whose whole nested-sampling run is too
long for the FP64 oracle.  Plain PyTorch CPU operations in FP64.

With log L(theta) = -1/2 sum_k ((MLP(theta)_k - data_k) / sigma_k)^2 on the
unit box (prior density 1):

  theta_hat  mode, by Gauss-Newton steps from theta* (the data's generator)
  F          Fisher matrix J^T J of the whitened residuals at theta_hat (or
             the negative Hessian of log L)
  log Z ~ log L(theta_hat) + (d/2) log 2 pi - 1/2 log det F + log P_box,

P_box being the mass of N(theta_hat, F^-1) inside the box (Monte Carlo).  The
Gaussian form is exact for a linear network; for the emulator it is an
approximation whose error is the posterior's departure from a Gaussian.
"""
import math

import numpy as np


def _torch():
    import torch
    return torch


def laplace_logz(problem, n_mc=400000, seed=0, hessian=False, max_steps=50):
    """Returns dict(log_z, log_z_untruncated, box_mass, theta_hat, logl_hat,
    cov): cov = F^-1, the covariance of the Gaussian approximation."""
    torch = _torch()
    spec = problem.mlp
    dt = torch.float64
    Ws = [torch.tensor(np.asarray(w, dtype=np.float64), dtype=dt) for w in spec.weights]
    Bs = [torch.tensor(np.asarray(b, dtype=np.float64), dtype=dt) for b in spec.biases]
    data = torch.tensor(np.asarray(spec.data, dtype=np.float64), dtype=dt)
    sig = torch.tensor(np.asarray(spec.sigma_out, dtype=np.float64), dtype=dt)

    def residual(th):  # whitened residuals (MLP(theta) - data) / sigma; SiLU between layers
        h = th
        for i, (w, b) in enumerate(zip(Ws, Bs)):
            h = w @ h + b
            if i + 1 < len(Ws):
                h = h * torch.sigmoid(h)
        return (h - data) / sig

    def loglike(th):
        r = residual(th)
        return -0.5 * torch.dot(r, r)

    th = torch.tensor(np.asarray(spec.theta_star, dtype=np.float64), dtype=dt)
    for _ in range(max_steps):
        J = torch.autograd.functional.jacobian(residual, th)
        step = torch.linalg.solve(J.T @ J, -(J.T @ residual(th)))
        th = th + step
        if float(step.norm()) < 1e-12:
            break
    if hessian:
        F = -torch.autograd.functional.hessian(loglike, th)
    else:
        J = torch.autograd.functional.jacobian(residual, th)
        F = J.T @ J
    d = th.numel()
    l_hat = float(loglike(th))
    logdet = float(torch.linalg.slogdet(F)[1])
    lz = l_hat + 0.5 * d * math.log(2.0 * math.pi) - 0.5 * logdet
    C = torch.linalg.inv(F)
    L = torch.linalg.cholesky(0.5 * (C + C.T))
    g = torch.Generator().manual_seed(int(seed))
    z = torch.randn(int(n_mc), d, generator=g, dtype=dt)
    s = th + z @ L.T
    mass = float(((s >= 0) & (s <= 1)).all(1).to(dt).mean())
    return {"log_z": lz + math.log(max(mass, 1e-300)), "log_z_untruncated": lz, "box_mass": mass,
            "theta_hat": th.numpy(), "logl_hat": l_hat, "cov": (0.5 * (C + C.T)).numpy()}
