"""Domain decomposition of a patch set over ranks and the cross-rank ghost
exchange plan.

The update shards by patches: each rank (one per GPU) owns a set of whole
patches and advances them with the stage kernels; the only data exchanged
between ranks are the ghost cells before every stage (the paper's
"FillBoundary", Sec. 4, which dominated its multi-GPU runs) and two scalar
reductions per step (the minimum timestep and the conservation sums).

* ``partition`` orders the patches along a Morton (Z-order) curve of their
  lower corners and cuts the curve into contiguous runs of nearly equal cell
  counts, so that each rank's patches are spatially compact.
* ``ghost_regions`` lists every ghost region of every patch with the interior
  region of the patch that owns its periodic image (the same geometry the
  library's copy descriptors encode).
* ``exchange_plan`` splits those regions into rank-local copies and, per peer
  rank, an ordered send list and an ordered receive list (the same order on
  both sides, so a packed buffer needs no headers).
* ``exchange`` packs, sends / receives with ``torch.distributed`` point-to-point
  operations (gloo for host arrays, NCCL for device arrays) and unpacks.

Device side: ``rank_layout`` places one rank's patches in that rank's own
field arrays; ``RankStepper`` advances a rank's shard (a library context made
by qk_init_shard) through one full update, as a generator that stops at the
two kinds of global synchronisation point (the signal-speed max and every
ghost exchange).  ``run_local`` drives several ranks in one process (each
halo buffer copied to the peer's receive buffer); ``run_distributed`` drives
one rank per process with ``torch.distributed`` (NCCL send / receive of the
packed device buffers, all-reduce for the max).  No kernel of one rank ever
waits on another rank: every synchronisation is between launches, on the host.
"""
from __future__ import annotations

import numpy as np


def _morton_key(x: int, y: int, z: int) -> int:
    key = 0
    for bit in range(21):
        key |= ((x >> bit) & 1) << (3 * bit)
        key |= ((y >> bit) & 1) << (3 * bit + 1)
        key |= ((z >> bit) & 1) << (3 * bit + 2)
    return key


def partition(layout, nranks: int) -> np.ndarray:
    """Owner rank of every patch: Morton order, contiguous runs of ~equal cells."""
    cells = np.prod(layout.n.astype(np.int64), axis=1)
    keys = [_morton_key(int(l[0]), int(l[1]), int(l[2])) for l in layout.lo]
    order = np.argsort(np.array(keys, dtype=np.uint64), kind="stable")
    owner = np.zeros(layout.nbox, dtype=np.int32)
    total = cells.sum()
    acc = 0
    for b in order:
        # rank = position of this patch's midpoint along the cumulative cells
        r = int(min(nranks - 1, (acc + cells[b] // 2) * nranks // total))
        owner[b] = r
        acc += cells[b]
    return owner


def ghost_regions(layout):
    """(dst_box, dst_lo, src_box, src_lo, ext) for every ghost region of every
    patch; dst_lo / src_lo are local cell coordinates including the ghost
    offset (0 = first ghost cell), ext the region extents (x, y, z)."""
    g = layout.ng
    dom = np.array(layout.dom_n, dtype=np.int64)
    lo = layout.lo.astype(np.int64)
    hi = lo + layout.n.astype(np.int64)
    out = []
    for b in range(layout.nbox):
        blo, bhi = lo[b], hi[b]
        for rz in range(3):
            for ry in range(3):
                for rx in range(3):
                    if (rx, ry, rz) == (1, 1, 1):
                        continue
                    r0 = np.empty(3, dtype=np.int64)
                    r1 = np.empty(3, dtype=np.int64)
                    for d, rs in enumerate((rx, ry, rz)):
                        if rs == 0:
                            r0[d], r1[d] = blo[d] - g, blo[d]
                        elif rs == 1:
                            r0[d], r1[d] = blo[d], bhi[d]
                        else:
                            r0[d], r1[d] = bhi[d], bhi[d] + g
                    a0 = np.floor_divide(r0, dom)
                    a1 = np.floor_divide(r1 - 1, dom)
                    for az in range(a0[2], a1[2] + 1):
                        for ay in range(a0[1], a1[1] + 1):
                            for ax in range(a0[0], a1[0] + 1):
                                sh = np.array([ax, ay, az]) * dom
                                w0 = np.maximum(r0 - sh, 0)
                                w1 = np.minimum(r1 - sh, dom)
                                if np.any(w0 >= w1):
                                    continue
                                i0 = np.maximum(w0[None, :], lo)
                                i1 = np.minimum(w1[None, :], hi)
                                hit = np.all(i0 < i1, axis=1)
                                for q in np.nonzero(hit)[0]:
                                    ext = i1[q] - i0[q]
                                    dst = i0[q] + sh - blo + g
                                    src = i0[q] - lo[q] + g
                                    out.append((b, tuple(int(v) for v in dst), int(q),
                                                tuple(int(v) for v in src),
                                                tuple(int(v) for v in ext)))
    return out


def exchange_plan(layout, owner: np.ndarray, regions=None):
    """Per rank: {'local': [...], 'send': {peer: [...]}, 'recv': {peer: [...]}}.
    Send and receive lists of a rank pair hold the same regions in the same
    order (sorted by destination patch, then destination corner)."""
    regions = ghost_regions(layout) if regions is None else regions
    nr = int(owner.max()) + 1 if len(owner) else 1
    plan = [{"local": [], "send": {}, "recv": {}} for _ in range(nr)]
    for reg in sorted(regions, key=lambda r: (r[0], r[1], r[2], r[3])):
        b, _, q, _, _ = reg
        rd, rs = int(owner[b]), int(owner[q])
        if rd == rs:
            plan[rd]["local"].append(reg)
        else:
            plan[rs]["send"].setdefault(rd, []).append(reg)
            plan[rd]["recv"].setdefault(rs, []).append(reg)
    return plan


def _view(layout, arr, b):
    return layout.full(arr, b)  # [z, y, x] including ghosts


def _src_slice(reg):
    _, _, _, s, e = reg
    return (slice(s[2], s[2] + e[2]), slice(s[1], s[1] + e[1]), slice(s[0], s[0] + e[0]))


def _dst_slice(reg):
    _, d, _, _, e = reg
    return (slice(d[2], d[2] + e[2]), slice(d[1], d[1] + e[1]), slice(d[0], d[0] + e[0]))


def apply_local(layout, fields, regions):
    """Copy the rank-local ghost regions (source and destination on this rank)."""
    for f in fields:
        for reg in regions:
            _view(layout, f, reg[0])[_dst_slice(reg)] = _view(layout, f, reg[2])[_src_slice(reg)]


def pack(layout, fields, regions) -> np.ndarray:
    parts = [_view(layout, f, reg[2])[_src_slice(reg)].ravel() for f in fields for reg in regions]
    return np.concatenate(parts) if parts else np.zeros(0, dtype=fields[0].dtype)


def unpack(layout, fields, regions, buf: np.ndarray) -> None:
    pos = 0
    for f in fields:
        for reg in regions:
            e = reg[4]
            n = e[0] * e[1] * e[2]
            _view(layout, f, reg[0])[_dst_slice(reg)] = buf[pos:pos + n].reshape(e[2], e[1], e[0])
            pos += n


def exchange(layout, fields, plan, rank: int) -> None:
    """Fill this rank's ghost cells: local copies, then one packed buffer per
    peer each way with non-blocking point-to-point operations."""
    import torch
    import torch.distributed as dist
    mine = plan[rank]
    apply_local(layout, fields, mine["local"])
    reqs, inbox = [], {}
    for peer, regs in sorted(mine["send"].items()):
        buf = torch.from_numpy(pack(layout, fields, regs))
        reqs.append(dist.isend(buf, peer))
    for peer, regs in sorted(mine["recv"].items()):
        n = sum(r[4][0] * r[4][1] * r[4][2] for r in regs) * len(fields)
        buf = torch.empty(n, dtype=torch.from_numpy(fields[0][:1]).dtype)
        inbox[peer] = buf
        reqs.append(dist.irecv(buf, peer))
    for r in reqs:
        r.wait()
    for peer, regs in sorted(mine["recv"].items()):
        unpack(layout, fields, regs, inbox[peer].numpy())


def global_max(value: float) -> float:
    """Max over ranks (the signal speed that sets the common timestep)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ device shards ---
def rank_layout(layout, owner: np.ndarray, rank: int, pad: int = 64):
    """The whole patch set, with this rank's patches packed into this rank's
    field arrays (others get offset 0: the library does not read them)."""
    from .inputs import Layout
    off = np.zeros(layout.nbox, dtype=np.int64)
    pos = 0
    for b in range(layout.nbox):
        if owner[b] == rank:
            off[b] = pos
            vol = int(np.prod(layout.n[b].astype(np.int64) + 2 * layout.ng))
            pos += (vol + pad - 1) // pad * pad
    return Layout(layout.lo.copy(), layout.n.copy(), off, layout.ng, tuple(layout.dom_n), int(pos))


class RankStepper:
    """One rank's part of a sharded update (Sec. 2.2 operator split, Sec. 4
    distribution by patches).  ``ctx`` is this rank's shard context; U / R its
    conserved hydro and radiation fields (torch CUDA tensors in the rank's
    layout).  ``step`` is a generator: it yields ("max", value) and expects the
    global max back, and yields ("halo", {peer: send buffer}, {peer: receive
    buffer}, event) after packing (event: recorded after the pack on the
    compute stream, or None), expecting the receive buffers filled on resume.

    With ``overlap``, each stage runs on the interior tiles right after the
    pack, before the yield (so that the transfer can proceed while they run),
    and on the boundary tiles after the unpack."""

    def __init__(self, ctx, U, R=None, overlap=False):
        import torch
        self.ctx, self.U, self.R = ctx, list(U), (list(R) if R is not None else None)
        self.overlap = overlap
        dt = U[0].dtype
        self.U1 = [torch.empty_like(u) for u in U]
        self.R1 = [torch.empty_like(r) for r in R] if R is not None else None
        self.peers = [p for p in range(ctx.nranks) if p != ctx.rank]
        self.cells = {p: ctx.halo_cells(p) for p in self.peers}
        # one send and one receive buffer per peer, sized for the widest fill (5 fields)
        nf = 5
        dev = U[0].device
        self.sbuf = {p: torch.empty(nf * max(1, s), dtype=dt, device=dev) for p, (s, _) in self.cells.items()}
        self.rbuf = {p: torch.empty(nf * max(1, r), dtype=dt, device=dev) for p, (_, r) in self.cells.items()}

    def _fill(self, fields, first, launch=None):
        """Full ghost fill of ``fields`` (state fields first, first+1, ...):
        rank-local copies and boundary values, then the halo; then the stage
        ``launch`` (split around the transfer when overlapping)."""
        import torch
        self.ctx.fill_ghosts(fields, first)
        nf = len(fields)
        sends, recvs = {}, {}
        for p in self.peers:
            s, r = self.cells[p]
            if s:
                sends[p] = self.sbuf[p][:nf * s]
                self.ctx.halo_pack(p, fields, sends[p], first)
            if r:
                recvs[p] = self.rbuf[p][:nf * r]
        event = None
        if fields[0].is_cuda:
            event = torch.cuda.Event()
            event.record()
        split = self.overlap and launch is not None
        if split:
            self.ctx.set_tile_part(1)
            launch()
        yield ("halo", sends, recvs, event)
        for p, buf in recvs.items():
            self.ctx.halo_unpack(p, fields, buf, first)
        if split:
            self.ctx.set_tile_part(2)
            launch()
            self.ctx.set_tile_part(0)
        elif launch is not None:
            launch()

    def step(self):
        ctx, U, R = self.ctx, self.U, self.R
        smax = yield ("max", ctx.signal_speed(U))
        dt, nsub, dtr, _ = ctx.set_timestep(smax)
        U1, R1 = self.U1, self.R1
        yield from self._fill(U, 0, lambda: ctx.hydro_stage(1, U, None, U1, dt))
        yield from self._fill(U1, 0, lambda: ctx.hydro_stage(2, U, U1, U, dt))
        if R is not None and not ctx.params.hydro_only:
            yield from self._fill(U[:1], 0)
            for _ in range(nsub):
                yield from self._fill(R, 5, lambda: ctx.rad_stage(1, R, None, R1, U[0], dtr))
                # stage 2 with the exchange in its epilogue (as qk_step runs it);
                # the exchange is per cell, so it follows each tile part
                yield from self._fill(R1, 5,
                                      lambda: ctx.rad_stage2_exchange(R, R1, R, U, dtr))
        return dt, nsub


def run_local(steppers):
    """Advance every rank of one process by one step, in lock-step: at each
    synchronisation point all ranks have issued their launches up to it, the
    host takes the max or copies each send buffer to the peer's receive
    buffer (device copies on the current stream), then all ranks resume."""
    gens = [s.step() for s in steppers]
    msgs = [next(g) for g in gens]
    result = [None] * len(gens)
    while True:
        kinds = {m[0] if m is not None else None for m in msgs}
        assert len(kinds) == 1, f"ranks out of step: {kinds}"
        kind = kinds.pop()
        if kind is None:
            return result
        if kind == "max":
            reply = [max(m[1] for m in msgs)] * len(gens)
        else:
            for r, m in enumerate(msgs):
                for p, buf in m[2].items():
                    buf.copy_(msgs[p][1][r])
            reply = [None] * len(gens)
        for r, g in enumerate(gens):
            try:
                msgs[r] = g.send(reply[r])
            except StopIteration as e:
                result[r] = e.value
                msgs[r] = None


def run_distributed(stepper, comm_stream=None):
    """Advance this process's rank by one step with torch.distributed: an
    all-reduce (MAX) for the signal speed and, for every ghost exchange, one
    batch of an isend / irecv pair per peer (device buffers: NCCL, one group;
    host buffers: gloo).  On
    the GPU the transfers are issued from ``comm_stream`` (created if None),
    which waits only for the pack, so that they run while the interior tiles
    of an overlapping stepper compute; waiting on the requests then orders the
    unpack on the compute stream after them."""
    import torch
    import torch.distributed as dist
    g = stepper.step()
    msg = next(g)
    cuda = stepper.U[0].is_cuda
    if cuda and comm_stream is None:
        comm_stream = torch.cuda.Stream()
    while True:
        if msg[0] == "max":
            t = torch.tensor([msg[1]], dtype=torch.float64, device=stepper.U[0].device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            reply = float(t.item())
        else:
            _, sends, recvs, event = msg

            def issue():
                # one batch (a NCCL group on the GPU): a send and a receive
                # between the same two ranks must not wait on each other
                ops = [dist.P2POp(dist.isend, buf, p) for p, buf in sorted(sends.items())]
                ops += [dist.P2POp(dist.irecv, buf, p) for p, buf in sorted(recvs.items())]
                return dist.batch_isend_irecv(ops) if ops else []

            if cuda:
                with torch.cuda.stream(comm_stream):
                    comm_stream.wait_event(event)
                    reqs = issue()
            else:
                reqs = issue()
            for q in reqs:
                q.wait()
            reply = None
        try:
            msg = g.send(reply)
        except StopIteration as e:
            return e.value
