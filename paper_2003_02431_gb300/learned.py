"""Training driver of the learned cut-cell correction (see the learned-correction section of
include/xdg.h). Orchestration only: samples, losses, gradients and Adam steps run in libxdg's
kernels; this module strings the calls together and concatenates device tensors.

Samples come from the plain solver: the residuals r_k = b - M x_k of its iterates x_k (one
preconditioned CG step per call, from the previous iterate); for every r_k the library runs
the plain cycle z = B r_k and records, per unit, the network input for the residual r_k - M z,
the normalised residual and the optimal local energy decrease (the exact local solve).
"""
from __future__ import annotations

from . import xdg


def attach_units(H, prob):
    """Units (cut-cell block pairs) and their geometry features of a generated problem."""
    pairs, geom, _ = prob.learned_units()
    H.units_setup(pairs, geom)
    return pairs, geom


def solver_residuals(H, b, iters, precision=xdg.XDG_PREC_F64):
    """r_0 = b and the residuals of `iters - 1` successive one-step solves from x = 0."""
    import torch
    x = torch.zeros_like(b)
    out = [b.clone()]
    for _ in range(iters - 1):
        H.solve(b, x, tol=0.0, maxit=1, precision=precision, raise_on_error=False)
        r = torch.empty_like(b)
        H.residual(1, b, x, r)
        out.append(r)
    return out


def samples(H, residuals, precision=xdg.XDG_PREC_F64):
    """(X, R, C) of all units for every residual, stacked (CUDA tensors)."""
    import torch
    Xs, Rs, Cs = [], [], []
    for r in residuals:
        X, R, C = H.units_samples(r, precision)
        Xs.append(X)
        Rs.append(R)
        Cs.append(C)
    return torch.cat(Xs), torch.cat(Rs), torch.cat(Cs)


class SampleSet:
    """Samples of several problems with their unit matrices: uid indexes the stacked Mloc."""

    def __init__(self):
        self.parts = []

    def add(self, H, residuals, precision=xdg.XDG_PREC_F64):
        import torch
        X, R, C = samples(H, residuals, precision)
        Mloc = H.units_local()
        U = Mloc.shape[0]
        uid = torch.arange(U, dtype=torch.int32, device=X.device).repeat(len(residuals))
        keep = C > 0  # a unit without residual carries no information
        self.parts.append((X[keep], uid[keep], Mloc, R[keep], C[keep]))

    def tensors(self):
        import torch
        X, uid, M, R, C, off = [], [], [], [], [], 0
        for x, u, m, r, c in self.parts:
            X.append(x)
            uid.append(u + off)
            M.append(m)
            R.append(r)
            C.append(c)
            off += m.shape[0]
        return (torch.cat(X).contiguous(), torch.cat(uid).contiguous(), torch.cat(M).contiguous(),
                torch.cat(R).contiguous(), torch.cat(C).contiguous())


def train(mlp, sample_set, epochs=30, batch=256, lr=2e-3, seed=1):
    X, uid, M, R, C = sample_set.tensors()
    return mlp.train(X, uid, M, R, C, epochs=epochs, batch=batch, lr=lr, seed=seed)


def evaluate(mlp, sample_set):
    """Mean loss of the network on the samples (-1: the exact local solve, 0: no gain)."""
    X, uid, M, R, C = sample_set.tensors()
    loss, _ = mlp.loss_grad(X, uid, M, R, C)
    return loss


def n_inputs(prob):
    return (1 << prob.D) + 3 + 2 * prob.Np


def network_for(prob, seed=0, stream=None):
    return xdg.Mlp(n_inputs(prob), 2 * prob.Np, seed=seed, stream=stream)


__all__ = ["attach_units", "solver_residuals", "samples", "SampleSet", "train", "evaluate", "network_for",
           "n_inputs"]
