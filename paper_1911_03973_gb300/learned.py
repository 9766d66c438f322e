"""Training workflow of the learned preconditioner (host orchestration only).

Every numerical step runs in libebe.so: the samples come from the library's
own Jacobi-PCG (ebe_solve), the training steps are ebe_mpnn_train_step
(forward and backward kernels, Adam), and the trained network is used by
ebe_solve_learned.  Inputs are seeded and synthetic: jittered squares with
random Fourier loads and nu ~ U[0, 10] (meshgen).
"""
from __future__ import annotations

import math

import numpy as np

from . import meshgen


def training_problem(n: int, seed: int):
    """Jittered n x n square, f = 8 random Fourier modes, nu ~ U[0, 10], Dirichlet 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    prob = meshgen.fourier_square(n, float(rng.uniform(0.0, 10.0)), seed)
    prob["coords"] = meshgen.jitter_interior(prob["coords"], 1.0 / (n - 1), 0.2, seed)
    return prob


def harvest(ebe, torch, h, n_n: int, n_samples: int, device, rtol_exact: float = 1e-12):
    """(r, e) pairs along a Jacobi-PCG solve: x* to rtol_exact, then the
    iterates x_k after k = n_samples evenly spread iteration counts from x0 = 0;
    r_k = mask(b - A x_k), e_k = x* - x_k (device float64 tensors)."""
    xs = torch.zeros(n_n, dtype=torch.float64, device=device)
    info = ebe.ebe_solve(h, xs, rtol=rtol_exact, precision=ebe.EBE_PREC_FP64)
    total = max(int(info["iterations"]), n_samples)
    ks = np.unique(np.linspace(1, max(1, int(0.95 * total)), n_samples).astype(int))
    out = []
    for k in ks:
        xk = torch.zeros(n_n, dtype=torch.float64, device=device)
        ebe.ebe_solve(h, xk, rtol=1e-300, maxit=int(k), precision=ebe.EBE_PREC_FP64)
        rk = torch.empty_like(xk)
        ebe.ebe_residual(h, xk, rk)
        out.append((rk, xs - xk))
    return out


def train(ebe, net, samples, steps: int, lr: float = 3e-3, seed: int = 0, lr_final: float = 3e-4):
    """Adam steps over shuffled samples [(handle, r, e)]; cosine step-size decay.
    Returns the list of losses (each before its step)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    losses = []
    order = []
    for t in range(steps):
        if not order:
            order = list(rng.permutation(len(samples)))
        h, r, e = samples[order.pop()]
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * t / max(steps - 1, 1)))
        losses.append(ebe.ebe_mpnn_train_step(net, h, r, e, a))
    return losses
