"""Domain-decomposed Newton-Leja phi-actions: the multi-GPU form of the Leja
path.

The paper's argument for Leja interpolation at scale is communication: a
Newton-Leja iteration (Sec. 2.2) needs one stencil product and the norms of
the stop test, where Arnoldi needs several inner products per step (Sec. 1,
Sec. 2.1).  So the global periodic grid is split into px x py rectangular
blocks; each iteration

  1. exchanges a one-cell halo of y_m across the four faces of every block,
  2. runs the block kernel  y_{m+1} = (1/gamma) J y_m - (c/gamma + xi_m) y_m,
     p_k += d_k[m+1] y_{m+1}  and its block sums ||y||^2, ||p_k||^2,
  3. sums those K + 1 numbers over all blocks (one small allreduce),
  4. applies the stop test |d_k[m]| ||y_m|| <= tol ||p_m^(k)||.

With lag = 1 the allreduce of iteration m is waited for only after
iteration m + 1 has been queued, so its latency hides behind the next
stencil product; the pass then ends one iteration later and its result
carries that one extra Newton term (smaller than tol ||p||).  With lag = 0
the pass is the single-domain method, iteration for iteration.

The spectral interval comes from the caller or from a power iteration run
the same way (one exchange and one allreduce per matvec, start vector the
SplitMix64 stream by global index, as on a single device).

This module is orchestration only.  The arithmetic runs in the backend's
kernels: GpuBackend calls libphix (phix_block_newton, phix_block_faces,
phix_block_start, phix_leja_stop, phix_leja_points,
phix_divided_differences); the exchange and the allreduce go through a Comm:
LocalComm for every block in this process, TorchComm for one or more blocks
per rank of a torch.distributed group (NCCL on GPUs, gloo on CPUs).
"""
import math

import numpy as np

FACES = ("S", "N", "W", "E")
OPPOSITE = {"S": "N", "N": "S", "W": "E", "E": "W"}
TRAVEL = ("N", "S", "E", "W")  # the order every rank issues the exchange in


def _split(n, parts):
    """Sizes of `parts` near-equal contiguous pieces of n (the first n % parts one larger)."""
    q, r = divmod(n, parts)
    return [q + (1 if i < r else 0) for i in range(parts)]


class Decomposition:
    """px x py blocks of an nx x ny periodic grid with ncomp species; block
    r = iy * px + ix covers columns x0..x0+bx-1 and rows y0..y0+by-1."""

    def __init__(self, nx, ny, px, py, ncomp):
        if px < 1 or py < 1 or px > nx or py > ny:
            raise ValueError("px, py must be in 1..nx, 1..ny")
        self.nx, self.ny, self.px, self.py, self.ncomp = nx, ny, px, py, ncomp
        sx, sy = _split(nx, px), _split(ny, py)
        ox = np.concatenate([[0], np.cumsum(sx)[:-1]]).astype(int)
        oy = np.concatenate([[0], np.cumsum(sy)[:-1]]).astype(int)
        self.blocks = []
        for iy in range(py):
            for ix in range(px):
                self.blocks.append(dict(ix=ix, iy=iy, x0=int(ox[ix]), y0=int(oy[iy]), bx=sx[ix], by=sy[iy]))

    @property
    def count(self):
        return len(self.blocks)

    def neighbour(self, r, face):
        """Block across `face` of block r (periodic)."""
        b = self.blocks[r]
        ix, iy = b["ix"], b["iy"]
        if face == "N":
            iy = (iy + 1) % self.py
        elif face == "S":
            iy = (iy - 1) % self.py
        elif face == "E":
            ix = (ix + 1) % self.px
        else:
            ix = (ix - 1) % self.px
        return iy * self.px + ix

    def face_slices(self, r):
        """Slices of the packed face buffer [S | N | W | E] of block r."""
        b = self.blocks[r]
        ns, nw = self.ncomp * b["bx"], self.ncomp * b["by"]
        return {"S": slice(0, ns), "N": slice(ns, 2 * ns), "W": slice(2 * ns, 2 * ns + nw),
                "E": slice(2 * ns + nw, 2 * ns + 2 * nw)}

    def face_len(self, r):
        b = self.blocks[r]
        return self.ncomp * (2 * b["bx"] + 2 * b["by"])

    def interior(self, r, v_global):
        """Block r's part of a global planar vector (species, row, column) as
        its planar bx x by vector (for setting up inputs and checking)."""
        b = self.blocks[r]
        g = np.asarray(v_global).reshape(self.ncomp, self.ny, self.nx)
        return np.ascontiguousarray(g[:, b["y0"]:b["y0"] + b["by"], b["x0"]:b["x0"] + b["bx"]]).reshape(-1)

    def assemble(self, parts):
        """Global planar vector from every block's planar part (inverse of interior)."""
        g = np.zeros((self.ncomp, self.ny, self.nx))
        for r, v in parts.items():
            b = self.blocks[r]
            g[:, b["y0"]:b["y0"] + b["by"], b["x0"]:b["x0"] + b["bx"]] = np.asarray(v).reshape(self.ncomp, b["by"],
                                                                                               b["bx"])
        return g.reshape(-1)


class _Done:
    def wait(self):
        return None


class LocalComm:
    """Every block of the decomposition lives in this process."""

    def owned(self, dec):
        return list(range(dec.count))

    def exchange(self, dec, send, recv, backend):
        """recv[r][halo face] <- send[nbr][interior face] for every owned block."""
        for t in TRAVEL:
            for r in self.owned(dec):
                dst = dec.neighbour(r, t)
                backend.copy(recv[dst], dec.face_slices(dst)[OPPOSITE[t]], send[r], dec.face_slices(r)[t])

    def allreduce(self, t):
        return _Done()


class TorchComm:
    """Blocks spread over the ranks of a torch.distributed group: rank q owns
    blocks q*bpr .. q*bpr + bpr - 1 (bpr = blocks per rank).  Faces between
    ranks travel as point-to-point messages, faces within a rank are copied;
    every rank issues its messages in one global order (travel direction,
    then block index), so the pairs match on NCCL as on gloo."""

    def __init__(self, dist, blocks_per_rank=1):
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.bpr = blocks_per_rank

    def owner(self, r):
        return r // self.bpr

    def owned(self, dec):
        if dec.count != self.world * self.bpr:
            raise ValueError("decomposition has %d blocks; the group holds %d x %d" % (dec.count, self.world, self.bpr))
        return list(range(self.rank * self.bpr, (self.rank + 1) * self.bpr))

    def exchange(self, dec, send, recv, backend):
        dist = self.dist
        ops = []
        for ti, t in enumerate(TRAVEL):
            for r in range(dec.count):
                dst = dec.neighbour(r, t)
                mine_src, mine_dst = self.owner(r) == self.rank, self.owner(dst) == self.rank
                tag = ti * dec.count + dst
                if mine_src and mine_dst:
                    backend.copy(recv[dst], dec.face_slices(dst)[OPPOSITE[t]], send[r], dec.face_slices(r)[t])
                elif mine_src:
                    ops.append(dist.P2POp(dist.isend, backend.view(send[r], dec.face_slices(r)[t]), self.owner(dst),
                                          tag=tag))
                elif mine_dst:
                    ops.append(dist.P2POp(dist.irecv, backend.view(recv[dst], dec.face_slices(dst)[OPPOSITE[t]]),
                                          self.owner(r), tag=tag))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()

    def allreduce(self, t):
        return self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, async_op=True)


class GpuBackend:
    """libphix kernels on torch CUDA tensors (float64)."""

    def __init__(self, phix, ctx, torch):
        self.phix, self.ctx, self.torch = phix, ctx, torch

    def zeros(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64, device="cuda")

    def view(self, buf, sl):
        return buf[sl]

    def copy(self, dst, dsl, src, ssl):
        dst[dsl].copy_(src[ssl])

    def to_host(self, t):
        return t.cpu().numpy()

    def accumulate(self, dst, srcs):
        """dst <- sum of the block sums (in block order)."""
        dst.copy_(srcs[0])
        for t in srcs[1:]:
            dst.add_(t)

    def set_interior(self, blk, y_pad, v):
        """Interior of a padded block <- v (planar bx x by per species): a strided copy."""
        nc = y_pad.numel() // ((blk.bx + 2) * (blk.by + 2))
        yp = y_pad.view(nc, blk.by + 2, blk.bx + 2)
        yp[:, 1:blk.by + 1, 1:blk.bx + 1].copy_(self.torch.as_tensor(v, dtype=self.torch.float64,
                                                                        device="cuda").view(nc, blk.by, blk.bx))

    def block(self, kind, dec, r, params, state_pad):
        b = dec.blocks[r]
        return self.phix.make_block(kind, dec.nx, dec.ny, b["x0"], b["y0"], b["bx"], b["by"], params, state_pad)

    def newton(self, blk, y_in, y_out, p, dk, a, b, norms):
        self.phix.phix_block_newton(self.ctx, blk, y_in, y_out, p, dk, a, b, norms)

    def faces(self, blk, direction, y_pad, buf):
        self.phix.phix_block_faces(self.ctx, blk, direction, y_pad, buf)

    def start(self, blk, seed, y_pad):
        self.phix.phix_block_start(self.ctx, blk, seed, y_pad)

    def stop(self, K, m, m_min, dkm, tol, ysq, psq):
        return self.phix.phix_leja_stop(K, m, m_min, dkm, tol, ysq, psq)

    def leja_points(self, m):
        return self.phix.phix_leja_points(m)

    def divided_differences(self, l, a, b, m):
        return self.phix.phix_divided_differences(l, a, b, m)


class BlockedOperator:
    """The Jacobian operator of one problem over a decomposition: per owned
    block its phix_block description and its padded state (halo filled), and
    the face buffers of the halo exchange."""

    def __init__(self, backend, comm, dec, kind, params, state_parts=None):
        self.backend, self.comm, self.dec, self.kind = backend, comm, dec, kind
        self.params = list(params)
        self.owned = comm.owned(dec)
        self.send = {r: backend.zeros(dec.face_len(r)) for r in self.owned}
        self.recv = {r: backend.zeros(dec.face_len(r)) for r in self.owned}
        self.blk = {r: backend.block(kind, dec, r, self.params, None) for r in self.owned}
        if state_parts is not None:
            st = {r: self.padded(r) for r in self.owned}
            for r in self.owned:
                backend.set_interior(self.blk[r], st[r], state_parts[r])
            self.halo(st)
            self.blk = {r: backend.block(kind, dec, r, self.params, st[r]) for r in self.owned}

    def padded(self, r):
        b = self.dec.blocks[r]
        return self.backend.zeros(self.dec.ncomp * (b["bx"] + 2) * (b["by"] + 2))

    def halo(self, pads):
        """Fill the halo ring of every owned padded block from its neighbours."""
        be = self.backend
        for r in self.owned:
            be.faces(self.blk[r], 0, pads[r], self.send[r])
        self.comm.exchange(self.dec, self.send, self.recv, be)
        for r in self.owned:
            be.faces(self.blk[r], 1, pads[r], self.recv[r])


class _Norms:
    """Per-iteration block sums, their allreduce and the host copy."""

    def __init__(self, op, K):
        self.op, self.K = op, K
        self.buf = [op.backend.zeros(K + 1) for _ in op.owned]
        self.total = op.backend.zeros(K + 1)
        self.handle = None

    def start(self):
        self.op.backend.accumulate(self.total, self.buf)
        self.handle = self.op.comm.allreduce(self.total)

    def result(self):
        self.handle.wait()
        v = self.op.backend.to_host(self.total)
        return float(v[0]), [float(x) for x in v[1:]]


def power_iteration(op, seed=0x5EED, max_it=50, rel=1e-2):
    """rho = ||J v_k|| by power iteration over the decomposition (the
    single-domain rule: stop at relative change <= rel from k >= 2, or after
    max_it matvecs).  Returns (rho, matvecs)."""
    be, dec = op.backend, op.dec
    y = {r: op.padded(r) for r in op.owned}
    y2 = {r: op.padded(r) for r in op.owned}
    for r in op.owned:
        be.start(op.blk[r], seed, y[r])
    nm = _Norms(op, 0)
    for i, r in enumerate(op.owned):
        be.newton(op.blk[r], y[r], None, [], [], 1.0, 0.0, nm.buf[i])
    nm.start()
    nrm = math.sqrt(nm.result()[0])
    rho_prev, rho = 0.0, 0.0
    for k in range(1, max_it + 1):
        op.halo(y)
        for i, r in enumerate(op.owned):
            be.newton(op.blk[r], y[r], y2[r], [], [], 1.0 / nrm, 0.0, nm.buf[i])
        nm.start()
        rho = math.sqrt(nm.result()[0])
        if rho == 0.0 or not math.isfinite(rho):
            return rho, k
        if k >= 2 and abs(rho - rho_prev) <= rel * rho:
            return rho, k
        rho_prev = rho
        nrm = rho
        y, y2 = y2, y
    return rho, max_it


def leja_phi(op, v_parts, h, outputs, tol, interval=None, safety=1.2, lag=1, m_max=500, m_min=3,
             gamma_cap=200.0, power_kw=None):
    """phi_{l_k}(s_k h J) v for outputs [(l_k, s_k)] (at most 4) in one
    vertical Newton-Leja pass over the decomposition.

    v_parts: {block: planar bx x by (x ncomp) part of v} for the owned blocks.
    interval: (alpha, beta) of J's real spectrum, or None for power iteration
    (alpha = -safety * rho, beta = 0).  Returns ({block: [p_k parts]}, info)
    with info iters, matvecs (power iteration), status (0 ok, 2 not converged,
    3 non-finite).  The pass must not need substeps (s h gamma <= gamma_cap)."""
    be, dec = op.backend, op.dec
    K = len(outputs)
    if not 1 <= K <= 4:
        raise ValueError("1..4 outputs")
    info = dict(iters=0, power_mv=0, status=0, lag=lag)
    if interval is None:
        rho, mv = power_iteration(op, **(power_kw or {}))
        info["power_mv"] = mv
        interval = (-safety * rho, 0.0)
    alpha, beta = interval
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    if gamma == 0.0:  # a zero spectrum: phi_l(0) v = v / l!
        return {r: [np.asarray(v_parts[r]) / math.factorial(l) for (l, _) in outputs] for r in op.owned}, info
    for (_, s) in outputs:
        if s * h * gamma > gamma_cap * (1 + 1e-12):
            raise ValueError("the action needs substeps (s h gamma > gamma_cap); not supported by the blocked pass")
    xi = be.leja_points(m_max + 1)
    d = [be.divided_differences(l, s * h * c, s * h * gamma, m_max + 1) for (l, s) in outputs]
    y = {r: op.padded(r) for r in op.owned}
    y2 = {r: op.padded(r) for r in op.owned}
    p = {}
    for r in op.owned:
        b = dec.blocks[r]
        p[r] = [be.zeros(dec.ncomp * b["bx"] * b["by"]) for _ in range(K)]
        be.set_interior(op.blk[r], y[r], v_parts[r])
    norms = [_Norms(op, K), _Norms(op, K)]  # ping-pong: one may be in flight

    def step(m, src, dst, nb):
        """y_{m+1} from y_m (halo exchange + block kernels) and its norms' allreduce."""
        op.halo(src)
        for i, r in enumerate(op.owned):
            be.newton(op.blk[r], src[r], dst[r], p[r], [d[k][m + 1] for k in range(K)], 1.0 / gamma,
                      -(c / gamma + xi[m]), nb.buf[i])
        nb.start()

    for i, r in enumerate(op.owned):
        be.newton(op.blk[r], y[r], None, p[r], [d[k][0] for k in range(K)], 1.0, 0.0, norms[0].buf[i])
    norms[0].start()
    status, m = 2, m_max
    for m in range(0, m_max + 1):
        cur, nxt = norms[m % 2], norms[(m + 1) % 2]
        if lag and m < m_max:
            step(m, y, y2, nxt)           # queue iteration m + 1 before waiting for m's sums
        ysq, psq = cur.result()
        st = be.stop(K, m, m_min, [d[k][m] for k in range(K)], tol, ysq, psq)
        if st != 0:
            status = 0 if st == 1 else 3
            if lag and m < m_max:
                m += 1                    # the queued iteration's term is in p
            break
        if m == m_max:
            break
        if not lag:
            step(m, y, y2, nxt)
        y, y2 = y2, y
    info["iters"] = m
    info["status"] = status
    return {r: [be.to_host(t) for t in p[r]] for r in op.owned}, info
