"""Training data and training loop of the learned spectral interval, through
the C-ABI: the state features, the power iteration (Sec. 2.2) that labels a
state, the label targets (phix_learned_targets: the interval and substep rule
of the Leja path itself) and the training all run in libphix; this module
only orders the calls and keeps the label set.

Labelling is checkpointed in shards: a run that stops (or is stopped) keeps
every finished shard, and a later run with the same problems resumes after
the last one and ends with the same arrays, bit for bit, as an uninterrupted
run (each label depends only on its own problem).
"""
import math
import os

import numpy as np

from . import phix

NPARAM = phix.PHIX_MLP_NPARAM
NFEAT = phix.PHIX_MLP_NFEAT


def initial_params(seed=0):
    """Weights ~ N(0, 1/fan_in) from numpy's seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM, dtype=np.float32)
    o = 0
    for r, c in [(64, 16), (64, 64), (3, 64)]:
        p[o:o + r * c] = rng.standard_normal(r * c) / math.sqrt(c)
        o += r * c + r
    return p


def label(ctx, op, h, feats):
    """(features float32[16], targets float32[3], power-iteration matvecs) of
    one state: op.state on the device, feats a float32[16] device buffer."""
    phix.phix_features(ctx, op, h, feats)
    rho, s = phix.phix_spectrum(ctx, op, phix.phix_opts_default())
    t = phix.phix_learned_targets(ctx, op, h, rho)
    return feats.cpu().numpy(), np.asarray(t, dtype=np.float32), int(s.power_mv)


def _shard_name(start, end):
    return "labels_%09d_%09d.npz" % (start, end)


def label_loop(n, label_fn, ckpt_dir=None, shard=8192, tag=""):
    """Labels 0..n-1 by label_fn(i) -> (x[16], t[3], matvecs), in shards of
    `shard`; with ckpt_dir each finished shard is saved there (written to a
    temporary name, then renamed) and a later call resumes after the shards it
    finds.  `tag` names the problem set: a shard saved under another tag is an
    error, not a silent mix.  Returns (X float32[n,16], T float32[n,3], total
    matvecs, labels computed by this call)."""
    X = np.empty((n, NFEAT), dtype=np.float32)
    T = np.empty((n, 3), dtype=np.float32)
    mv = np.zeros(n, dtype=np.int64)
    done = 0
    if ckpt_dir:
        os.makedirs(ckpt_dir, exist_ok=True)
        while done < n:
            end = min(n, done + shard)
            path = os.path.join(ckpt_dir, _shard_name(done, end))
            if not os.path.exists(path):
                break
            with np.load(path) as z:
                if str(z["tag"]) != tag:
                    raise ValueError("checkpoint %s belongs to problem set %r, not %r" % (path, str(z["tag"]), tag))
                X[done:end], T[done:end], mv[done:end] = z["X"], z["T"], z["mv"]
            done = end
    computed = 0
    for start in range(done, n, shard):
        end = min(n, start + shard)
        for i in range(start, end):
            x, t, m = label_fn(i)
            X[i], T[i], mv[i] = x, t, m
            computed += 1
        if ckpt_dir:
            path = os.path.join(ckpt_dir, _shard_name(start, end))
            tmp = path + ".tmp.npz"
            np.savez(tmp, X=X[start:end], T=T[start:end], mv=mv[start:end], tag=np.array(tag))
            os.replace(tmp, path)
    return X, T, int(mv.sum()), computed


def make_dataset(ctx, problem, torch, n=None, ckpt_dir=None, shard=8192, tag=""):
    """Labels of problem(i) = (op, h, state tensor), i < n (or of a list of
    such triples).  Returns (X float32[n,16], T float32[n,3], matvecs)."""
    if isinstance(problem, (list, tuple)):
        lst = problem
        problem = lst.__getitem__
        n = len(lst)
    feats = torch.empty(NFEAT, dtype=torch.float32, device="cuda")

    def fn(i):
        op, h, _ = problem(i)
        return label(ctx, op, h, feats)

    X, T, mv, _ = label_loop(n, fn, ckpt_dir, shard, tag)
    return X, T, mv


def train(ctx, X, T, torch, seed=0, batch=256, schedule=((3e-3, 2000), (1e-3, 2000), (3e-4, 1000))):
    """Adam on the GPU over contiguous batches; returns (params tensor, last loss)."""
    n = (len(X) // batch) * batch
    params = torch.tensor(initial_params(seed), device="cuda")
    m = torch.zeros(NPARAM, device="cuda")
    v = torch.zeros(NPARAM, device="cuda")
    Xd = torch.tensor(X[:n], device="cuda")
    Td = torch.tensor(T[:n], device="cuda")
    step, loss = 0, float("nan")
    for lr, nsteps in schedule:
        step, loss = phix.phix_mlp_train(ctx, params, m, v, step, Xd, Td, batch, nsteps, lr)
    return params, loss
