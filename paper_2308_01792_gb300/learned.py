"""Training pairs and training of the learned local smoother.

Pairs of two kinds:
* ``make_noise_pairs`` (default): error fields e drawn as seeded white noise
  on the non-Dirichlet DoFs (the rough error a smoother exists to remove)
  with their residuals r = A e computed by the GPU operator of a field seed;
* ``make_pairs``: states of plain FP32 multigrid (see below).

Orchestration only: every arithmetic step runs in the library's kernels
(V-cycles, residuals, the pair sampling kernel, the tensor-core forward /
backward and Adam kernels).  A training pair is the state of plain FP32
multigrid on the finest level before the pre-smoother of a cycle: the
residual r = b - A x and the error e = x* - x against a converged FP64
solution x*, taken right after the coarse-grid correction of a V-cycle
(the input of the post-smoother): there the error is mostly the
high-frequency part that a local smoother can see in a residual
neighbourhood, whereas before the pre-smoother it is dominated by smooth
components that no 15-point neighbourhood determines.  Each pair contributes every `stride`-th macro-cell-interior
DoF as a sample (features: D^-1 r on the 15-point neighbourhood; target
e - omega D^-1 r; both divided by the neighbourhood's norm, which the
network's positive homogeneity makes harmless).
"""
from __future__ import annotations

import numpy as np

from . import (GMG, HG_OP_P1_DIVKGRAD, HG_PREC_F64, MLP, Hierarchy, Mesh, Operator,
               learn_samples)


def lognormal_coefficient(xyz, seed):
    import synthgen as sg
    try:
        return sg.rff_eval_torch(sg.rff_params(seed), xyz)
    except Exception:
        return sg.rff_eval(sg.rff_params(seed), xyz)


def make_pairs(macro, lmin, level, field_seeds, cycles, stride, omega=2.0 / 3.0, rhs_seed=7,
               hier=None):
    """Samples (X bf16 [N,16], t float32 [N]) from `cycles` pairs per field seed."""
    import torch
    import synthgen as sg
    H = hier or Hierarchy(Mesh(macro.xyz, macro.cells), lmin, level)
    _, xyz, dirich = H.canonical_info(level)
    Xs, ts = [], []
    npairs = 0
    for s in field_seeds:
        op = Operator(H, HG_OP_P1_DIVKGRAD, coeff=lognormal_coefficient(xyz, s))
        G = GMG(op, lmin=lmin, omega=omega)
        bc = sg.uniform_vector(rhs_seed + s, len(xyz))
        bc[dirich] = 0.0
        b64 = H.from_canonical(level, torch.tensor(bc, device="cuda"))
        xs64 = H.zeros(level, torch.float64)
        G.solve(xs64, b64, tol=1e-11, max_iter=200, precision=HG_PREC_F64)
        b32, xs32 = b64.float(), xs64.float()
        x32 = H.zeros(level, torch.float32)
        t32 = H.zeros(level, torch.float32)
        r32 = H.zeros(level, torch.float32)
        bc32 = H.zeros(level - 1, torch.float32)
        xc32 = H.zeros(level - 1, torch.float32)

        def smooth(nu):
            for _ in range(nu):
                op.jacobi(level, x32, b32, t32, omega=omega)
                x32.copy_(t32)

        for c in range(cycles):
            # one V(3,3) cycle spelled out, sampling after the coarse correction
            smooth(3)
            op.residual(level, x32, b32, r32)
            H.restrict(level, r32, bc32)
            xc32.zero_()
            G.vcycle(level - 1, xc32, bc32)
            H.prolong_add(level, xc32, x32)
            op.residual(level, x32, b32, r32)
            X, t = learn_samples(op, level, r32, xs32, x32, omega, stride, (s + c) % stride)
            Xs.append(X)
            ts.append(t)
            npairs += 1
            smooth(3)
        del op, G
    return torch.cat(Xs), torch.cat(ts), npairs


def make_noise_pairs(macro, lmin, level, field_seeds, draws, stride, omega=2.0 / 3.0,
                     noise_seed=100, hier=None):
    """Samples from `draws` white-noise errors per field seed: r = A e, x* = 0."""
    import torch
    import synthgen as sg
    H = hier or Hierarchy(Mesh(macro.xyz, macro.cells), lmin, level)
    _, xyz, dirich = H.canonical_info(level)
    Xs, ts = [], []
    npairs = 0
    z = H.zeros(level, torch.float32)
    r = H.zeros(level, torch.float32)
    for s in field_seeds:
        op = Operator(H, HG_OP_P1_DIVKGRAD, coeff=lognormal_coefficient(xyz, s))
        for c in range(draws):
            e = sg.uniform_vector(noise_seed * s + c, len(xyz))
            e[dirich] = 0.0
            x = H.from_canonical(level, torch.tensor(-e, dtype=torch.float32, device="cuda"))
            op.residual(level, x, z, r)          # r = 0 - A x = A e
            X, t = learn_samples(op, level, r, z, x, omega, stride, (s + c) % stride)
            Xs.append(X)
            ts.append(t)
            npairs += 1
        del op
    return torch.cat(Xs), torch.cat(ts), npairs


def train(X, t, steps=2000, batch=65536, lr=2e-3, seed=11, mlp=None):
    """Train a network (He-initialised from `seed`) with Adam; returns (mlp, loss)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0, np.sqrt(2.0 / 16), size=(32, 16))
    W1[:, 15] = 0.0
    W2 = rng.normal(0, np.sqrt(2.0 / 32), size=(32, 32))
    w3 = rng.normal(0, 0.1 * np.sqrt(1.0 / 32), size=32)
    if mlp is None:
        mlp = MLP(np.concatenate([W1.ravel(), W2.ravel(), w3]))
    loss = mlp.train(X, t, steps=steps, batch=batch, lr=lr)
    return mlp, loss


def main(argv=None):
    """Generate 2000 pairs on the 4x4x4 Kuhn cube at level 4 (fields of seeds
    1..250, 8 per field): white-noise errors (default), states of the GPU
    multigrid after the coarse correction (--pairs gmg), or half of each
    (--pairs mixed); train, and save the parameters (.npy)."""
    import argparse
    import torch
    import synthgen as sg
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", type=int, default=250)
    ap.add_argument("--draws", type=int, default=8)
    ap.add_argument("--stride", type=int, default=16)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--pairs", choices=["noise", "gmg", "mixed"], default="noise")
    a = ap.parse_args(argv)
    macro = sg.kuhn_cube(4)
    if a.pairs == "mixed":
        H = Hierarchy(Mesh(macro.xyz, macro.cells), 0, 4)
        half = range(1, a.seeds // 2 + 1)
        Xn, tn, nn = make_noise_pairs(macro, 0, 4, half, a.draws, a.stride, hier=H)
        Xg, tg, ng = make_pairs(macro, 0, 4, half, a.draws, a.stride, hier=H)
        X, t, npairs = torch.cat([Xn, Xg]), torch.cat([tn, tg]), nn + ng
    elif a.pairs == "gmg":
        X, t, npairs = make_pairs(macro, 0, 4, range(1, a.seeds + 1), a.draws, a.stride)
    else:
        X, t, npairs = make_noise_pairs(macro, 0, 4, range(1, a.seeds + 1), a.draws, a.stride)
    net, loss = train(X, t, steps=a.steps, batch=65536, lr=1e-3)
    np.save(a.out, net.params())
    print(f"{npairs} pairs, {len(t)} samples, final loss {loss:.6g}, zero-net loss "
          f"{MLP().grad(X, t)[0]:.6g} -> {a.out}")


if __name__ == "__main__":
    main()
