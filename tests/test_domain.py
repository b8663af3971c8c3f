"""The domain-decomposed Newton-Leja driver (paper_2211_08948_gb300.domain)
on CPU: decomposition geometry, the halo exchange, the allreduce schedule
(blocking and lagged by one iteration) and the stop logic, with the per-block
kernels replaced by NumPy (tests/domain_util.py), against the unsplit
oracle: in one process (LocalComm) and over gloo ranks (TorchComm, world
size 2 and 4)."""
import os
import socket

import numpy as np
import pytest
import torch

import synth
from domain_util import CpuBackend, oracle_pass
from oracle import leja
from oracle.operators import AdvDiff, GrayScott, Burgers
from paper_2211_08948_gb300 import domain


def test_decomposition_geometry():
    dec = domain.Decomposition(10, 7, 3, 2, 2)
    assert [b["bx"] for b in dec.blocks[:3]] == [4, 3, 3]
    assert [b["by"] for b in dec.blocks[::3]] == [4, 3]
    # periodic neighbours
    assert dec.neighbour(0, "W") == 2 and dec.neighbour(2, "E") == 0
    assert dec.neighbour(0, "S") == 3 and dec.neighbour(3, "N") == 0
    for r in range(dec.count):
        for f in domain.FACES:
            assert dec.neighbour(dec.neighbour(r, f), domain.OPPOSITE[f]) == r
    v = np.arange(2 * 10 * 7, dtype=np.float64)
    parts = {r: dec.interior(r, v) for r in range(dec.count)}
    assert sum(p.size for p in parts.values()) == v.size
    assert np.array_equal(dec.assemble(parts), v)


def test_halo_exchange_fills_every_ring_from_its_neighbours():
    nx, ny = 9, 6
    dec = domain.Decomposition(nx, ny, 3, 2, 1)
    be = CpuBackend()
    comm = domain.LocalComm()
    op = domain.BlockedOperator(be, comm, dec, 0, [1.0, 0.0, 0.0])
    g = np.arange(nx * ny, dtype=np.float64).reshape(ny, nx)
    pads = {}
    for r in range(dec.count):
        pads[r] = op.padded(r)
        be.set_interior(op.blk[r], pads[r], dec.interior(r, g.reshape(-1)))
    op.halo(pads)
    for r in range(dec.count):
        b = dec.blocks[r]
        yp = pads[r].numpy().reshape(b["by"] + 2, b["bx"] + 2)
        rows = [(b["y0"] + j - 1) % ny for j in range(b["by"] + 2)]
        cols = [(b["x0"] + i - 1) % nx for i in range(b["bx"] + 2)]
        want = g[np.ix_(rows, cols)]
        # the ring without its corners (a 5-point stencil reads no corner)
        assert np.array_equal(yp[1:-1, :], want[1:-1, :])
        assert np.array_equal(yp[:, 1:-1], want[:, 1:-1])


def _advdiff_case(n=24):
    p = synth.advdiff_params(n, mult=20.0)
    v = synth.advdiff_gaussian(n)
    return p, v, AdvDiff(n, p["D"], p["ax"], p["ay"])


@pytest.mark.parametrize("px,py", [(2, 2), (3, 2), (1, 3)])
@pytest.mark.parametrize("lag", [0, 1])
def test_local_blocks_advdiff_vs_unsplit_oracle(px, py, lag):
    n = 24
    p, v, aop = _advdiff_case(n)
    dec = domain.Decomposition(n, n, px, py, 1)
    be = CpuBackend()
    op = domain.BlockedOperator(be, domain.LocalComm(), dec, 0, [p["D"], p["ax"], p["ay"]])
    outs = [(0, 1.0), (1, 1.0), (2, 0.5)]
    rho = 8.0 * p["D"] * n * n
    res, info = domain.leja_phi(op, {r: dec.interior(r, v) for r in range(dec.count)}, p["h"], outs, 1e-10,
                                interval=(-rho, 0.0), lag=lag)
    ref, m = oracle_pass(aop.jv, v, p["h"], -rho, 0.0, outs, 1e-10, iters_extra=lag)
    assert info["status"] == 0 and info["iters"] == m
    for k in range(len(outs)):
        got = dec.assemble({r: res[r][k] for r in res})
        assert np.linalg.norm(got - ref[k]) <= 1e-12 * np.linalg.norm(ref[k])


@pytest.mark.parametrize("kind", ["grayscott", "burgers"])
def test_local_blocks_nonlinear_with_power_iteration(kind):
    """Interval by the blocked power iteration (same SplitMix64 start by
    global index), state halos exchanged once, vertical outputs."""
    n = 20
    if kind == "grayscott":
        prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=20.0)
        state = synth.grayscott_state(n, seed=3, patch=8)
        params, kd = [prm["Du"], prm["Dv"], prm["F"], prm["k"]], 1
        oop = GrayScott(n, *params, state=state)
        h = prm["h"]
    else:
        prm = synth.burgers_params(n, nu=2e-2, mult=5.0)
        state = synth.burgers_state(n, seed=3)
        params, kd = [prm["nu"]], 2
        oop = Burgers(n, prm["nu"], state=state)
        h = prm["h"]
    nc = 2 if kd == 1 else 1
    dec = domain.Decomposition(n, n, 2, 3, nc)
    be = CpuBackend()
    op = domain.BlockedOperator(be, domain.LocalComm(), dec, kd, params,
                                {r: dec.interior(r, state) for r in range(dec.count)})
    v = np.random.default_rng(8).standard_normal(nc * n * n)
    outs = [(1, 0.5), (1, 1.0)]
    res, info = domain.leja_phi(op, {r: dec.interior(r, v) for r in range(dec.count)}, h, outs, 1e-10, lag=1)
    rho, mv = leja.power_iteration(oop.jv, v.size)
    assert info["power_mv"] == mv
    ref, m = oracle_pass(oop.jv, v, h, -1.2 * rho, 0.0, outs, 1e-10, iters_extra=1)
    assert info["iters"] == m
    for k in range(len(outs)):
        got = dec.assemble({r: res[r][k] for r in res})
        assert np.linalg.norm(got - ref[k]) <= 1e-11 * np.linalg.norm(ref[k])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, px, py, bpr, lag, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 18
        prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=20.0)
        state = synth.grayscott_state(n, seed=5, patch=6)
        params = [prm["Du"], prm["Dv"], prm["F"], prm["k"]]
        dec = domain.Decomposition(n, n, px, py, 2)
        comm = domain.TorchComm(dist, blocks_per_rank=bpr)
        owned = comm.owned(dec)
        be = CpuBackend()
        op = domain.BlockedOperator(be, comm, dec, 1, params, {r: dec.interior(r, state) for r in owned})
        v = np.random.default_rng(9).standard_normal(2 * n * n)
        res, info = domain.leja_phi(op, {r: dec.interior(r, v) for r in owned}, prm["h"], [(0, 1.0), (1, 1.0)],
                                    1e-10, lag=lag)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), iters=info["iters"], mv=info["power_mv"],
                 **{"b%d_%d" % (r, k): res[r][k] for r in owned for k in range(2)})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,px,py,bpr,lag", [(2, 2, 1, 1, 1), (2, 2, 2, 2, 0), (4, 2, 2, 1, 1)])
def test_gloo_ranks_vs_unsplit_oracle(tmp_path, world, px, py, bpr, lag):
    """world_size 2 and 4 gloo ranks, one or two blocks each, Gray-Scott with
    the blocked power iteration: every rank's blocks, assembled, equal the
    unsplit oracle's pass element by element."""
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), px, py, bpr, lag, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    n = 18
    prm = synth.grayscott_params(n, Du=2e-3, Dv=1e-3, mult=20.0)
    state = synth.grayscott_state(n, seed=5, patch=6)
    oop = GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"], state=state)
    v = np.random.default_rng(9).standard_normal(2 * n * n)
    rho, mv = leja.power_iteration(oop.jv, v.size)
    ref, m = oracle_pass(oop.jv, v, prm["h"], -1.2 * rho, 0.0, [(0, 1.0), (1, 1.0)], 1e-10, iters_extra=lag)
    dec = domain.Decomposition(n, n, px, py, 2)
    parts = {0: {}, 1: {}}
    for q in range(world):
        z = np.load(os.path.join(str(tmp_path), "rank%d.npz" % q))
        assert int(z["iters"]) == m and int(z["mv"]) == mv
        for key in z.files:
            if key.startswith("b"):
                r, k = (int(x) for x in key[1:].split("_"))
                parts[k][r] = z[key]
    for k in range(2):
        got = dec.assemble(parts[k])
        assert np.linalg.norm(got - ref[k]) <= 1e-11 * np.linalg.norm(ref[k])
