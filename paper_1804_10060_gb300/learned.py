"""Training and use of the learned CG initial guess (driver around the CUDA kernels).

Every numerical step runs in libthermoamg: the training targets are
displacements the AMG-PCG solver itself computes (to rtol 1e-8), the features
come from tam_node_features, the network is trained by tam_mlp_train_step
(hand-written forward/backward/Adam kernels) and evaluated by
tam_learned_guess, which smooths the network's output and discards it unless
its preconditioned residual energy is below the zero guess's.
This module only chooses data, batches and the learning-rate schedule.
"""
from __future__ import annotations

import numpy as np
import torch

from . import meshgen
from . import thermoamg as tam


def solve(pb, params=None, x0=None, rtol=1e-8):
    """(features, displacement, iterations, K, rhs, device dict) of one problem."""
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], params)
    x = torch.zeros_like(rhs) if x0 is None else x0.clone()
    it, rel, _ = tam.amg_pcg_solve(H, rhs, x, rtol=rtol, max_iter=1000)
    dist = torch.from_numpy(meshgen.clamp_distance(pb)).cuda()
    F = tam.tam_node_features(d["coords"], d["cells"], d["T"], dist)
    H.destroy()
    return F, x, it, K, rhs, d


def training_set(problems, params=None):
    """Stack the node features and solved displacements of several problems."""
    Xs, Ys = [], []
    for pb in problems:
        F, x, _, K, _, _ = solve(pb, params)
        Xs.append(F)
        Ys.append(x.float())
        K.destroy()
    return torch.cat(Xs), torch.cat(Ys)


def normalization(X, Y):
    """Per-feature mean/std of the inputs and per-component std of the outputs."""
    Xd = X.double()
    shift = Xd.mean(0).cpu().numpy()
    std = Xd.std(0).cpu().numpy()
    scale = np.where(std > 0, 1.0 / np.where(std > 0, std, 1.0), 1.0)
    ostd = Y.double().std(0).cpu().numpy()
    out_scale = np.where(ostd > 0, ostd, 1.0)
    return shift, scale, out_scale


def train(net: tam.Mlp, X, Y, steps=1500, batch=32768, lr=3e-3, seed=0, log_every=0):
    """Adam on random mini-batches with a cosine-decayed learning rate; returns the loss history."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    n = X.shape[0]
    hist = []
    for k in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device="cuda", generator=g)
        lr_k = lr * 0.5 * (1 + np.cos(np.pi * k / steps)) + 1e-5
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr_k)
        hist.append(loss)
        if log_every and k % log_every == 0:
            print(f"step {k} loss {loss:.3e}", flush=True)
    return hist


def evaluate(net: tam.Mlp, pb, params=None, rtol=1e-8, bf16=True, smooth_degree=8):
    """Iterations from zero vs from the learned guess on one problem (same tolerance)."""
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], params)
    dist = torch.from_numpy(meshgen.clamp_distance(pb)).cuda()
    F = tam.tam_node_features(d["coords"], d["cells"], d["T"], dist)
    x0 = torch.zeros_like(rhs)
    it0, rel0, _ = tam.amg_pcg_solve(H, rhs, x0, rtol=rtol, max_iter=1000)
    # the raw network output's error, before the guard
    raw = net.forward(F, bf16=bf16).double()
    raw_err = float(torch.linalg.norm(raw - x0) / torch.linalg.norm(x0))
    xg, used, energy = tam.tam_learned_guess(net, H, F, rhs, bf16=bf16, smooth_degree=smooth_degree)
    x1 = xg.clone()
    it1, rel1, _ = tam.amg_pcg_solve(H, rhs, x1, rtol=rtol, max_iter=1000)
    err = float(torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0))
    H.destroy()
    K.destroy()
    return {"iters_zero": it0, "iters_guess": it1, "guess_used": used, "guess_energy_ratio": energy,
            "guess_rel_error": raw_err, "solution_diff": err, "rel_resid_zero": rel0, "rel_resid_guess": rel1,
            "n_dof": pb.n_dof}
