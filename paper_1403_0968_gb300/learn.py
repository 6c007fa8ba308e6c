"""Training of the learned element-local preconditioner from Jacobi-PCG residuals.

Orchestration only: every arithmetic step runs in the library's kernels (Jacobi-PCG and the
FP64-accurate residual for the iterates, sem_mlp_samples for the element-local solves, features and
targets, sem_mlp_train_step for forward, backward and Adam).  The random draws (initial weights,
sampled elements, minibatch order, kappa fields) come from numpy generators with explicit seeds and
are passed in as data.

A pair: for a seeded kappa field and a seeded random right-hand side, take the residual r_k of
Jacobi-PCG after k steps (by default k = 0, the initial residual: rough, like the residuals the
flexible CG hands to the preconditioner later on), and for a random subset of elements the
residual-to-error pair of the element's own shifted Neumann problem (A_e + sigma_e M_e) x_e =
W_e r_e, solved by Jacobi-PCG on the element: input r_e (normalised, with the geometric features),
target x_e (minus the Jacobi step (D^-1 r)_e on the Jacobi base), scaled by dbar_e / |r_e|.
"""
from __future__ import annotations

import math

import numpy as np

from . import MLP_EPS, MLP_H1, MLP_H2, SEM_FEAT_EMU, SEM_FEAT_FP32, SEM_FEAT_MLP, SEM_FEAT_PCG, MlpTrainer, \
    Problem, mlp_param_count


def he_init(N: int, seed: int, h1: int = MLP_H1, h2: int = MLP_H2) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)) and zero biases, FP32, in the library's layout."""
    n3 = (N + 1) ** 3
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_in, fan_out in ((n3 + 6, h1), (h1, h2), (h2, n3)):
        parts.append(g.normal(0.0, math.sqrt(2.0 / fan_in), size=fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == mlp_param_count(N, h1, h2)
    return p


def generate_pairs(problems, per_field: int, iterates=(0,), rhs_per_field: int = 8, seed: int = 0,
                   eps: float = MLP_EPS, jacobi_base: bool = True):
    """problems: iterable of dicts (N, box, vertices, kappa_modes) -> X, T on the device.

    For each problem, rhs_per_field seeded random right-hand sides (U(-1, 1), zero on Dirichlet
    nodes); for each, the residual of Jacobi-PCG after k steps for every k in ``iterates`` (k = 0:
    the initial residual, the right-hand side itself); for each residual, per_field /
    (rhs_per_field * len(iterates)) random elements give one pair each (sem_mlp_samples)."""
    import torch

    g = np.random.Generator(np.random.PCG64(seed))
    Xs, Ts = [], []
    for pr in problems:
        P = Problem(pr["N"], pr["vertices"], box=pr["box"], kappa_modes=pr.get("kappa_modes"), bc="box",
                    features=SEM_FEAT_EMU | SEM_FEAT_FP32 | SEM_FEAT_PCG | SEM_FEAT_MLP)
        per = max(1, per_field // (rhs_per_field * len(iterates)))
        for _ in range(rhs_per_field):
            raw = torch.from_numpy(g.uniform(-1.0, 1.0, P.nglobal)).cuda()
            zero = torch.zeros_like(raw)
            b = P.residual(raw, zero)  # M (raw - A 0): the right-hand side without its Dirichlet entries
            for k in iterates:
                if k == 0:
                    r = b
                else:
                    xk, _ = P.pcg(b, rtol=1e-14, max_it=k, mode="fp64", apply_prec="fp64_emu", use_graph=False,
                                  raise_on_error=False)
                    r = P.residual(b, xk)
                elems = torch.from_numpy(g.choice(P.nelem, size=min(per, P.nelem), replace=False).astype(np.int32))
                X, T, _ = P.mlp_samples(r, elems.cuda(), eps=eps, jacobi_base=jacobi_base)
                Xs.append(X)
                Ts.append(T)
        del P
    return torch.cat(Xs), torch.cat(Ts)


def train(N: int, X, T, epochs: int = 20, batch: int = 256, lr: float = 1e-3, seed: int = 0, params=None):
    """Adam on minibatches (seeded shuffles); returns (params on the device, per-epoch mean loss)."""
    import torch

    g = np.random.Generator(np.random.PCG64(seed + 1))
    p = torch.from_numpy(he_init(N, seed) if params is None else params).cuda()
    tr = MlpTrainer(N, p, batch, lr=lr)
    n = X.shape[0]
    history = []
    for _ in range(epochs):
        perm = torch.from_numpy(g.permutation(n)).cuda()
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        steps = 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            tot += tr.step(X[idx], T[idx])
            steps += 1
        history.append(float(tot.item()) / max(1, steps))
    return tr.params, history


# ---- checkpoints: the weights, and for resuming training the Adam state ----
CHECKPOINT_VERSION = 1


def _host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def save_checkpoint(path, N: int, params, trainer=None, jacobi_base: bool = True, h1: int = MLP_H1,
                    h2: int = MLP_H2) -> None:
    """Writes the network (order N, hidden widths h1, h2, the library's parameter layout) to an
    .npz file; with a trainer, also its Adam moments, step count and learning rate, so that
    training resumes where it stopped (resume_trainer).  jacobi_base records how the weights were
    trained (sem_mlp_load takes the same flag)."""
    n = mlp_param_count(N, h1, h2)
    p = _host(params).astype(np.float32, copy=False).reshape(-1)
    if p.shape != (n,):
        raise ValueError(f"params has {p.size} values, the network (N={N}, {h1}, {h2}) has {n}")
    arrays = {"version": np.int64(CHECKPOINT_VERSION), "shape": np.array([N, h1, h2], dtype=np.int64),
              "jacobi_base": np.int64(1 if jacobi_base else 0), "params": p}
    if trainer is not None:
        if (trainer.N, trainer.h1, trainer.h2) != (N, h1, h2):
            raise ValueError("the trainer belongs to another network shape")
        m = _host(trainer.m).astype(np.float32, copy=False).reshape(-1)
        v = _host(trainer.v).astype(np.float32, copy=False).reshape(-1)
        if m.shape != (n,) or v.shape != (n,):
            raise ValueError("the trainer's Adam moments do not match the parameter count")
        arrays.update(m=m, v=v, step=np.int64(trainer.step_count), lr=np.float64(trainer.lr))
    with open(path, "wb") as f:
        np.savez(f, **arrays)


def load_checkpoint(path) -> dict:
    """Reads a checkpoint written by save_checkpoint -> {"N", "h1", "h2", "jacobi_base", "params"
    (float32 numpy)} and, when it holds a trainer's state, "m", "v", "step", "lr".  Refuses (ValueError)
    another format version, a parameter count that does not match the shape, and non-finite
    weights or moments: a corrupted file must not reach the preconditioner."""
    with np.load(path) as f:
        version = int(f["version"]) if "version" in f.files else -1
        if version != CHECKPOINT_VERSION:
            raise ValueError(f"checkpoint format {version}, expected {CHECKPOINT_VERSION}")
        N, h1, h2 = (int(x) for x in f["shape"])
        n = mlp_param_count(N, h1, h2)
        out = {"N": N, "h1": h1, "h2": h2, "jacobi_base": bool(int(f["jacobi_base"])),
               "params": f["params"].astype(np.float32)}
        names = ["params"]
        if "m" in f.files:
            out.update(m=f["m"].astype(np.float32), v=f["v"].astype(np.float32), step=int(f["step"]),
                       lr=float(f["lr"]))
            names += ["m", "v"]
            if out["step"] < 0:
                raise ValueError("negative Adam step count")
    for k in names:
        if out[k].shape != (n,):
            raise ValueError(f"{k} has {out[k].size} values, the network (N={N}, {h1}, {h2}) has {n}")
        if not np.all(np.isfinite(out[k])):
            raise ValueError(f"{k} holds non-finite values")
    return out


def resume_trainer(ck: dict, batch: int) -> MlpTrainer:
    """An MlpTrainer on the device that continues from a checkpoint: its weights, and its Adam
    moments and step count when the checkpoint holds them (otherwise a fresh Adam state)."""
    import torch

    tr = MlpTrainer(ck["N"], torch.from_numpy(ck["params"]).cuda(), batch, h1=ck["h1"], h2=ck["h2"],
                    lr=ck.get("lr", 1e-3))
    if "m" in ck:
        tr.m.copy_(torch.from_numpy(ck["m"]))
        tr.v.copy_(torch.from_numpy(ck["v"]))
        tr.step_count = ck["step"]
    return tr
