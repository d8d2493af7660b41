"""One event split into z slabs, one rank per GPU (the C ABI's
glasma_slab_* calls; include/glasma.h states the halo protocol).

The beam axis is the lattice's long axis (Sec. 4), so a run on several GPUs
gives each rank a slab of consecutive z slices.  Every step, each rank packs
two messages on the device (its top slice for the rank above, its bottom
slice for the rank below), the ranks exchange them, and each unpacks what it
received into its halo slices before glasma_step.  Observables are gathered
in rank order: the T^{mu nu}(z) rows of the owned slices, summed in z order
for the total energy exactly as a single context sums them, and the Gauss
residual maxima.

Under the improved scheme (Sec. 3, Fig. wilson (b)) a step is the same
exchange, then glasma_implicit_begin, sweeps whose maxima (the largest
change of E and the largest E over the owned slices) are folded with max
across the ranks before the stopping rule (glasma_implicit_converged), and
glasma_implicit_end: every rank takes the sweeps the whole lattice would.
The sweeps exchange nothing else.

Transports: `DistTransport` sends the messages with torch.distributed
point-to-point calls (NCCL between GPUs, gloo between CPU processes) and
bounds every wait; a message that does not arrive in time ends the exchange
with GlasmaError code TIMEOUT instead of hanging the rank.  `LocalTransport`
runs several slabs of one process on one device, copying each message into
the receiver's buffer (cudaMemcpyAsync through torch).  No kernel waits on
another rank: the exchange happens on the host between launches.
"""
from __future__ import annotations

import datetime
import math

from . import glasma as G


def slab_bounds(nz, nranks):
    """Contiguous z ranges [z0, z1) of nz slices over nranks ranks, sizes
    differing by at most one slice."""
    base, extra = divmod(int(nz), int(nranks))
    out, z = [], 0
    for r in range(nranks):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


class SlabRank:
    """Rank `rank` of `nranks`: a slab context and its message buffers."""

    def __init__(self, cfg, rank, nranks, rho=None, stream=None, device=None):
        import torch
        self.cfg = dict(cfg)
        self.rank, self.nranks = int(rank), int(nranks)
        z0, z1 = slab_bounds(cfg["nz"], nranks)[self.rank]
        self.h = G.glasma_slab_init(cfg, z0, z1, rho, stream)
        self.z0, self.z1 = z0, z1
        p = G.make_params(cfg)
        self.implicit = p.scheme == G.IMPLICIT
        self.tol, self.maxit = p.implicit_tol, p.implicit_max_iter
        self.precision = "fp32" if p.precision == G.FP32 else "fp64"
        dev = device if device is not None else torch.cuda.current_device()
        self.buf = {}
        for d in (+1, -1):
            if self.has(d):
                # send and receive buffers, 16-byte aligned by the allocator;
                # what arrives from direction d is the neighbour's message
                # in direction -d
                self.buf[("send", d)] = torch.empty(
                    G.glasma_slab_message_bytes(self.h, d), dtype=torch.uint8, device=dev)
                self.buf[("recv", d)] = torch.empty(
                    G.glasma_slab_message_bytes(self.h, -d), dtype=torch.uint8, device=dev)

    def has(self, d):
        """Is there a neighbouring rank in direction d (+1 above, -1 below)?"""
        return (self.rank + d) in range(self.nranks)

    def windows(self):
        info = G.glasma_get_info(self.h)
        return tuple(info.window_a), tuple(info.window_b)

    def pack(self):
        for d in (+1, -1):
            if self.has(d):
                G.glasma_slab_pack(self.h, d, self.buf[("send", d)].data_ptr())

    def unpack(self):
        # the message from the rank below is its dir +1 message
        for d in (+1, -1):
            if self.has(d):
                G.glasma_slab_unpack(self.h, d, self.buf[("recv", d)].data_ptr())

    def step(self):
        G.glasma_step(self.h, 1)

    def tmunu_rows(self):
        return G.glasma_tmunu(self.h)[0]


def implicit_step(ranks, fold):
    """One improved step of the ranks this process holds, their halos
    already exchanged: begin, sweeps until the stopping rule holds on the
    maxima folded over all ranks by fold([(dmax, emax), ...]) -> (dmax,
    emax), end.  Returns the number of sweeps."""
    for r in ranks:
        G.glasma_implicit_begin(r.h)
    r0 = ranks[0]
    dm, em = [], []
    converged = False
    for _ in range(r0.maxit):
        d, e = fold([G.glasma_implicit_sweep(r.h) for r in ranks])
        dm.append(d)
        em.append(e)
        if not math.isfinite(d):
            raise G.GlasmaError(-4, "implicit_step", "a sweep met a non-finite value")
        if G.glasma_implicit_converged(dm, em, r0.tol, r0.precision):
            converged = True
            break
    for r in ranks:
        G.glasma_implicit_end(r.h)
    if not converged:
        raise G.GlasmaError(-6, "implicit_step",
                            "no convergence within %d sweeps" % r0.maxit)
    return len(dm)


def _fold_max(pairs):
    return max(p[0] for p in pairs), max(p[1] for p in pairs)


def merge_windows(all_windows):
    """Union over ranks of ((zA0, WA), (zB0, WB)) windows (W = 0: none)."""
    out = []
    for N in range(2):
        spans = [w[N] for w in all_windows if w[N][1] > 0]
        if not spans:
            out.append((0, 0))
            continue
        a = min(s[0] for s in spans)
        b = max(s[0] + s[1] for s in spans)
        out.append((a, b - a))
    return tuple(out)


def total_energy(cfg, rows):
    """H from the gathered T^{mu nu} rows in z order, summed exactly as a
    single context sums them (eps slice by slice, then the cell volume)."""
    s = 0.0
    for v in rows[:, 0]:
        s += float(v)
    a_t, a_z = float(cfg.get("a_t", 1.0)), float(cfg.get("a_z", 1.0))
    return a_t * a_t * a_z * float(cfg["nx"] * cfg["ny"]) * s


class LocalTransport:
    """All slabs in one process on one device (one stream): messages are
    copied from each sender's buffer into its neighbour's."""

    def __init__(self, ranks):
        self.ranks = ranks

    def setup(self):
        w = merge_windows([r.windows() for r in self.ranks])
        for r in self.ranks:
            G.glasma_slab_set_windows(r.h, *w)

    def exchange(self):
        for r in self.ranks:
            r.pack()
        for k, r in enumerate(self.ranks):
            if r.has(-1):
                r.buf[("recv", -1)].copy_(self.ranks[k - 1].buf[("send", +1)])
            if r.has(+1):
                r.buf[("recv", +1)].copy_(self.ranks[k + 1].buf[("send", -1)])
        for r in self.ranks:
            r.unpack()

    def step(self):
        self.exchange()
        if self.ranks[0].implicit:
            return implicit_step(self.ranks, _fold_max)
        for r in self.ranks:
            r.step()

    def gather_rows(self):
        import numpy as np
        return np.concatenate([r.tmunu_rows() for r in self.ranks])


def exchange_messages(send, recv, rank, nranks, timeout_s=30.0, group=None):
    """Point-to-point halo exchange of one rank: send[d] goes to rank + d,
    recv[d] is filled from rank + d (d = +1, -1; tensors of equal size on
    both sides, CPU for gloo or CUDA for NCCL).  Every wait is bounded by
    timeout_s; a message that does not arrive raises GlasmaError TIMEOUT."""
    import torch.distributed as dist
    works = []
    for d in (+1, -1):
        peer = rank + d
        if 0 <= peer < nranks and d in send:
            works.append(dist.isend(send[d], peer, group=group))
    for d in (+1, -1):
        peer = rank + d
        if 0 <= peer < nranks and d in recv:
            works.append(dist.irecv(recv[d], peer, group=group))
    limit = datetime.timedelta(seconds=timeout_s)
    for w in works:
        try:
            ok = w.wait(timeout=limit)
        except RuntimeError as e:
            raise G.GlasmaError(-7, "exchange_messages",
                                "halo message not received within %.1f s: %s"
                                % (timeout_s, str(e).splitlines()[0])) from None
        if ok is False:
            raise G.GlasmaError(-7, "exchange_messages",
                                "halo message not received within %.1f s" % timeout_s)


class DistTransport:
    """One slab per process; messages through torch.distributed: device
    buffers with NCCL, staged through host memory with gloo."""

    def __init__(self, rank_obj, timeout_s=30.0, group=None):
        self.r = rank_obj
        self.timeout_s = timeout_s
        self.group = group

    def setup(self):
        import torch
        import torch.distributed as dist
        (a0, aw), (b0, bw) = self.r.windows()
        big = 1 << 30
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        # [min start A, -max end A, min start B, -max end B] over ranks with
        # a window (others contribute neutral values)
        v = torch.tensor([a0 if aw else big, -(a0 + aw) if aw else big,
                          b0 if bw else big, -(b0 + bw) if bw else big],
                         dtype=torch.int64, device=dev)
        dist.all_reduce(v, op=dist.ReduceOp.MIN, group=self.group)
        v = v.tolist()
        wa = (0, 0) if v[0] == big else (v[0], -v[1] - v[0])
        wb = (0, 0) if v[2] == big else (v[2], -v[3] - v[2])
        G.glasma_slab_set_windows(self.r.h, wa, wb)

    def exchange(self):
        import torch
        import torch.distributed as dist
        r = self.r
        r.pack()
        torch.cuda.synchronize()
        keys = [d for d in (+1, -1) if r.has(d)]
        if dist.get_backend(self.group) == "nccl":
            send = {d: r.buf[("send", d)] for d in keys}
            recv = {d: r.buf[("recv", d)] for d in keys}
        else:
            # gloo moves host tensors: the messages go through host memory
            send = {d: r.buf[("send", d)].cpu() for d in keys}
            recv = {d: torch.empty(r.buf[("recv", d)].shape, dtype=torch.uint8) for d in keys}
        exchange_messages(send, recv, r.rank, r.nranks, self.timeout_s,
                          self.group)
        for d in keys:
            if recv[d] is not r.buf[("recv", d)]:
                r.buf[("recv", d)].copy_(recv[d])
        r.unpack()

    def fold(self, pairs):
        """Max over all ranks of this rank's (dmax, emax)."""
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        v = torch.tensor(list(pairs[0]), dtype=torch.float64, device=dev)
        dist.all_reduce(v, op=dist.ReduceOp.MAX, group=self.group)
        return float(v[0]), float(v[1])

    def step(self):
        self.exchange()
        if self.r.implicit:
            return implicit_step([self.r], self.fold)
        self.r.step()
