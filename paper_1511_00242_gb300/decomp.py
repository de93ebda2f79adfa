"""Spatial decomposition of one mesh over ranks: 2-D blocks of cells with a
one-cell halo ring of all nine f_tilde fields, exchanged every step.

Each rank owns a block of cells [i0, i1) x [j0, j1) of the global mesh and
steps an extended block: its own cells plus one ring of halo cells on every
side that borders another block (or wraps around a periodic direction split
over several blocks).  The step of a cell reads only f_tilde of the cells
within one cell of it, edges and corners included (the cell stage is local;
the face reconstruction reads phi of both cells of a face and of their
neighbours along the face), plus the ghost values of physical boundaries,
which the extended block computes as the whole mesh does.  So after the halo
ring is refreshed from the neighbours, one step of the extended block gives
every owned cell exactly the value the single-mesh step gives; halo cells
themselves come out wrong (their far side is an arbitrary outflow boundary)
and are overwritten by the next exchange.  (Where a periodic direction is
split, the halo cell across the wrap takes its centre from the wrapped face
coordinate; it equals the single mesh's periodic ghost centre bit for bit
when the face coordinates are exact in binary, and to rounding otherwise.)

The exchange has two phases: columns of owned rows across W / E sides, then
rows of the full extended width (halo columns included) across S / N sides,
which carries the corner cells diagonally in two hops.  Transport is
pluggable: torch.distributed point-to-point (gloo on CPU tensors, NCCL on
device tensors), or direct copies between blocks held by one process.

Steppers hold a block's state and provide get / put of one line of cells of
all nine fields (see GpuStepper; the tests drive the FP64 CPU oracle with the
same interface).  The FP64 sums of mass and momentum over owned cells are
all-reduced across ranks.
"""
from __future__ import annotations

import math

import numpy as np

W_, E_, S_, N_ = 0, 1, 2, 3
INF = 1.0e300
_OUTFLOW = [("outflow", -INF, INF, 1.0, 0.0, 0.0)]


def _split(n: int, parts: int):
    """Nearly equal split of n cells into `parts` ranges, each >= 2 cells."""
    if parts < 1 or n < 2 * parts:
        raise ValueError(f"cannot split {n} cells into {parts} blocks of at least 2")
    edges = [round(k * n / parts) for k in range(parts + 1)]
    return list(zip(edges[:-1], edges[1:]))


def _periodic(side_segments) -> bool:
    return any(seg[0] == "periodic" for seg in side_segments)


class Block:
    """One rank's part of the mesh.

    i0, i1, j0, j1  owned cells of the global mesh
    halo[side]      True when that side borders another block (a halo ring
                    is held there); sides W, E, S, N = 0, 1, 2, 3
    nbr[side]       rank across that side (halo sides only)
    ox, oy          offset of the owned cells in the extended arrays
    nx, ny          owned cells; nxe, nye extended sizes
    case            the extended block as a problem (case dict)
    """

    def __init__(self, rank, bx, by, xr, yr, case, PX, PY):
        self.rank, self.bx, self.by = rank, bx, by
        (self.i0, self.i1), (self.j0, self.j1) = xr, yr
        gnx, gny = case["nx"], case["ny"]
        per_x, per_y = _periodic(case["bc"][W_]), _periodic(case["bc"][S_])
        self.halo = [False] * 4
        self.nbr = [None] * 4
        for side, (inner, wraps, other) in {
                W_: (self.i0 > 0, per_x and PX > 1, ((bx - 1) % PX, by)),
                E_: (self.i1 < gnx, per_x and PX > 1, ((bx + 1) % PX, by)),
                S_: (self.j0 > 0, per_y and PY > 1, (bx, (by - 1) % PY)),
                N_: (self.j1 < gny, per_y and PY > 1, (bx, (by + 1) % PY))}.items():
            if inner or wraps:
                self.halo[side] = True
                self.nbr[side] = other[1] * PX + other[0]
        self.nx, self.ny = self.i1 - self.i0, self.j1 - self.j0
        self.ox, self.oy = int(self.halo[W_]), int(self.halo[S_])
        self.nxe = self.nx + self.ox + int(self.halo[E_])
        self.nye = self.ny + self.oy + int(self.halo[N_])
        xf, yf = np.asarray(case["xf"], float), np.asarray(case["yf"], float)
        self.case = dict(case, nx=self.nxe, ny=self.nye,
                         xf=self._faces(xf, self.i0, self.i1, self.halo[W_], self.halo[E_]),
                         yf=self._faces(yf, self.j0, self.j1, self.halo[S_], self.halo[N_]),
                         bc=[_OUTFLOW if self.halo[s] else list(case["bc"][s]) for s in range(4)],
                         name=f"block {rank} of {case.get('name', 'mesh')}")
        # an unsplit periodic direction stays periodic; a split one is cut
        if per_x and PX > 1:
            for s in (W_, E_):
                if not self.halo[s]:
                    raise ValueError("periodic direction split without a wrap")

    @staticmethod
    def _faces(f, a, b, lo, hi):
        n = len(f) - 1
        out = list(f[a:b + 1])
        if lo:  # the cell west of a: cell a-1, or the last cell when wrapping
            out.insert(0, f[a - 1] if a > 0 else f[0] - (f[n] - f[n - 1]))
        if hi:
            out.append(f[b + 1] if b < n else f[n] + (f[1] - f[0]))
        return np.array(out)

    # owned cells of a global [.., ny, nx] array, and the extended view of it
    def owned(self, g):
        return g[..., self.j0:self.j1, self.i0:self.i1]

    def extended_from_global(self, g):
        """Extended-block values taken from a global array [..., ny, nx],
        halo cells included (periodic wraps by index)."""
        gny, gnx = g.shape[-2:]
        rows = np.arange(self.j0 - self.oy, self.j0 - self.oy + self.nye) % gny
        cols = np.arange(self.i0 - self.ox, self.i0 - self.ox + self.nxe) % gnx
        return np.ascontiguousarray(g[..., rows[:, None], cols[None, :]])

    def lines(self):
        """The transfers of one exchange, in order: (phase, side, axis, send
        index, receive index, lo, hi).  axis 0: a column (index along x) over
        rows lo..hi; axis 1: a row over columns lo..hi.  The send index is the
        owned line next to `side`, the receive index the halo line there."""
        out = []
        for side in (W_, E_):
            if self.halo[side]:
                send = self.ox if side == W_ else self.ox + self.nx - 1
                recv = 0 if side == W_ else self.nxe - 1
                out.append((0, side, 0, send, recv, self.oy, self.oy + self.ny))
        for side in (S_, N_):
            if self.halo[side]:
                send = self.oy if side == S_ else self.oy + self.ny - 1
                recv = 0 if side == S_ else self.nye - 1
                out.append((1, side, 1, send, recv, 0, self.nxe))
        return out


def plan(case, PX: int, PY: int):
    """Blocks of a PX x PY decomposition of `case` (a tensor mesh given by its
    face coordinates); rank = by * PX + bx."""
    if "xf" not in case or "yf" not in case:
        raise ValueError("the decomposition splits tensor meshes (face coordinates xf, yf) only")
    xs, ys = _split(case["nx"], PX), _split(case["ny"], PY)
    return [Block(by * PX + bx, bx, by, xs[bx], ys[by], case, PX, PY)
            for by in range(PY) for bx in range(PX)]


_OPP = {W_: E_, E_: W_, S_: N_, N_: S_}


def exchange_local(blocks, steppers):
    """Halo exchange between blocks held by one process (direct copies)."""
    for phase in (0, 1):
        moves = []
        for b in blocks:
            for ph, side, axis, send, recv, lo, hi in b.lines():
                if ph != phase:
                    continue
                nb = blocks[b.nbr[side]]
                # my halo line on `side` takes the neighbour's owned line on its opposite side
                for ph2, side2, _, send2, _, lo2, hi2 in nb.lines():
                    if ph2 == phase and side2 == _OPP[side] and nb.nbr[side2] == b.rank:
                        moves.append((b.rank, axis, recv, lo, hi, nb.rank, send2, lo2, hi2))
                        break
                else:
                    raise RuntimeError("neighbour has no matching line")
        data = [(dst, axis, recv, lo, hi, steppers[src].get(axis, send, lo2, hi2))
                for dst, axis, recv, lo, hi, src, send, lo2, hi2 in moves]
        for dst, axis, recv, lo, hi, d in data:
            steppers[dst].put(axis, recv, lo, hi, d)


def exchange_dist(block, stepper, dist, new_buffer):
    """Halo exchange of this rank's block over torch.distributed point-to-point
    messages (gloo or NCCL).  new_buffer(shape) returns a tensor to receive
    into (on the transport's device); stepper.get / put move lines between the
    block and such tensors.  Messages carry the receiver's side as tag."""
    for phase in (0, 1):
        ops, recvs = [], []
        for ph, side, axis, send, recv, lo, hi in block.lines():
            if ph != phase:
                continue
            buf = new_buffer((9, hi - lo))
            recvs.append((axis, recv, lo, hi, buf))
            ops.append(dist.P2POp(dist.irecv, buf, block.nbr[side], tag=side))
            ops.append(dist.P2POp(dist.isend, stepper.get(axis, send, lo, hi), block.nbr[side],
                                  tag=_OPP[side]))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        for axis, recv, lo, hi, buf in recvs:
            stepper.put(axis, recv, lo, hi, buf)


def allreduce_sums(local, dist, device="cpu"):
    """FP64 sum over ranks of this rank's (mass, x-momentum, y-momentum)."""
    import torch
    t = torch.tensor(np.asarray(local, dtype=np.float64), device=device)
    dist.all_reduce(t)
    return t.cpu().numpy()


class GpuStepper:
    """A block on the GPU: a Solver of the extended block, with lines of cells
    moved through libdvbe's pack / unpack kernels (device buffers of nine
    fields in the solver's storage precision).  torch provides the buffers."""

    def __init__(self, block, precision="f64", stream=None):
        import torch
        from . import Solver
        self.torch, self.block = torch, block
        self.s = Solver(block.case, precision=precision, stream=stream)
        self.dtype = {8: torch.float64, 4: torch.float32, 2: torch.float16}[self.s.device_state()[3]]

    def init_equilibrium_global(self, rho, ux, uy):
        b = self.block
        self.s.init_equilibrium(*(b.extended_from_global(a) for a in (rho, ux, uy)))

    def init_f_global(self, f):
        self.s.init_f(self.block.extended_from_global(f))

    def new_buffer(self, shape):
        return self.torch.empty(shape, dtype=self.dtype, device="cuda")

    def get(self, axis, index, lo, hi):
        buf = self.new_buffer((9, hi - lo))
        self.s.pack_line(axis, index, lo, hi, buf.data_ptr())
        return buf

    def put(self, axis, index, lo, hi, buf):
        self.s.unpack_line(axis, index, lo, hi, buf.data_ptr())

    def step(self, n=1):
        self.s.step(n)

    def owned_f(self):
        b = self.block
        return self.s.get_f()[:, b.oy:b.oy + b.ny, b.ox:b.ox + b.nx]

    def owned_sums(self):
        """FP64 (mass, momentum) over the owned cells, on the GPU."""
        return self.s.conserved_window(self.block.ox, self.block.oy, self.block.nx, self.block.ny)

    def close(self):
        self.s.close()


def run_local(case, PX, PY, fields, steps, precision="f64"):
    """The decomposed step on one GPU: PX x PY blocks, each its own Solver,
    halos exchanged in-process after every step.  Returns the global f_tilde
    assembled from the owned cells, and the summed conserved quantities."""
    blocks = plan(case, PX, PY)
    st = [GpuStepper(b, precision) for b in blocks]
    try:
        for s in st:
            s.init_equilibrium_global(*fields)
        for _ in range(steps):
            for s in st:
                s.step(1)
            exchange_local(blocks, st)
        f = np.zeros((9, case["ny"], case["nx"]))
        sums = np.zeros(3)
        for b, s in zip(blocks, st):
            f[:, b.j0:b.j1, b.i0:b.i1] = s.owned_f()
            sums += s.owned_sums()
        return f, sums
    finally:
        for s in st:
            s.close()
