"""Spatial decomposition on CPU: one mesh split into 2-D blocks with a
one-cell halo ring of all nine f_tilde fields exchanged every step, each
block stepped by the FP64 oracle, must reproduce the single-mesh oracle bit
for bit (the FV step of a cell reads only cells within one cell of it, edges
and corners included, Sec 2.2).  Run in one process with the in-process
exchange, and as gloo ranks (world sizes 2 and 4) with the point-to-point
exchange; the FP64 all-reduce of the owned cells' mass and momentum matches
the single mesh's sums.  The multi-GPU path uses the same plan and exchange
with the library's line pack / unpack kernels on device buffers (tested on
one GPU in test_gpu_decomposition)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402
from paper_1511_00242_gb300 import decomp  # noqa: E402


class OracleStepper:
    """A block held as a float64 array and stepped by the oracle."""

    def __init__(self, block, f_global):
        import torch
        self.torch, self.block = torch, block
        self.f = block.extended_from_global(f_global)

    def step(self, n=1):
        self.f = O.step(self.block.case, self.f, n)

    def get(self, axis, index, lo, hi):
        line = self.f[:, lo:hi, index] if axis == 0 else self.f[:, index, lo:hi]
        return self.torch.from_numpy(np.ascontiguousarray(line))

    def put(self, axis, index, lo, hi, buf):
        v = np.asarray(buf)
        if axis == 0:
            self.f[:, lo:hi, index] = v
        else:
            self.f[:, index, lo:hi] = v

    def owned(self):
        b = self.block
        return self.f[:, b.oy:b.oy + b.ny, b.ox:b.ox + b.nx]

    def owned_sums(self):
        b = self.block
        sub = dict(b.case, nx=b.nx, ny=b.ny, xf=b.case["xf"][b.ox:b.ox + b.nx + 1],
                   yf=b.case["yf"][b.oy:b.oy + b.ny + 1])
        return O.conserved(dict(sub, bc=W.periodic_bc()), np.ascontiguousarray(self.owned()))


def _dyadic_tg(n):
    """Doubly periodic box of spacing 1/16 (exact in binary), CFL 0.5."""
    case, fields = W.taylor_green_box(n)
    xf = W.uniform_faces(n, 0.0, n / 16.0)
    case = dict(case, xf=xf, yf=xf.copy(), dt=W.cfl_dt(xf, xf, 0.5))
    return case, fields


def _cases():
    """(case, fields) with every kind of side: walls (moving, diffuse),
    free stream, outflow, symmetry, periodic, on stretched meshes."""
    cav, _ = W.cavity(23, Re=200, scheme="dugks", stretch_beta=1.3)
    box = W.cavity_four_lids(26, 19, scheme="bkg", kind="diffuse")
    plate, _ = W.flat_plate(nx_up=6, nx_plate=14, ny=17, scheme="dugks", Re_L=2e3)
    tg, tgf = _dyadic_tg(20)
    # a periodic direction split over blocks: the halo cell's centre comes from
    # the wrapped face, which matches the single mesh's periodic ghost centre
    # bit for bit when the coordinates are exact in binary (spacing 1/16 here)
    couette, _ = W.couette(24, 16, U=0.05, nu=0.02, scheme="bkg", kind="diffuse")
    out = []
    for c in (cav, box, plate, tg, couette):
        fields, delta = W.random_state(c, 7, amp_neq=1e-3)
        out.append((c, fields, delta))
    return out


CASES = _cases()
STEPS = 12


def _single(case, fields, delta):
    return O.step(case, O.init_equilibrium(case, *fields) + delta, STEPS)


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("PX,PY", [(2, 1), (1, 3), (2, 2), (3, 2)])
def test_blocks_in_one_process_match_single_mesh(k, PX, PY):
    case, fields, delta = CASES[k]
    f0 = O.init_equilibrium(case, *fields) + delta
    blocks = decomp.plan(case, PX, PY)
    st = [OracleStepper(b, f0) for b in blocks]
    for _ in range(STEPS):
        for s in st:
            s.step(1)
        decomp.exchange_local(blocks, st)
    g = np.zeros_like(f0)
    sums = np.zeros(3)
    for b, s in zip(blocks, st):
        g[:, b.j0:b.j1, b.i0:b.i1] = s.owned()
        sums += s.owned_sums()
    ref = _single(case, fields, delta)
    np.testing.assert_array_equal(g, ref)
    np.testing.assert_allclose(sums, O.conserved(case, ref), rtol=1e-13, atol=1e-15)


def test_plan_covers_the_mesh_once():
    case = CASES[1][0]
    for PX, PY in ((1, 1), (2, 3), (4, 2)):
        cover = np.zeros((case["ny"], case["nx"]), int)
        for b in decomp.plan(case, PX, PY):
            cover[b.j0:b.j1, b.i0:b.i1] += 1
            assert b.nxe == b.nx + sum(b.halo[:2]) and b.nye == b.ny + sum(b.halo[2:])
        assert (cover == 1).all()
    with pytest.raises(ValueError):
        decomp.plan(case, 14, 1)  # blocks of fewer than 2 cells
    with pytest.raises(ValueError):  # quadrilateral meshes are not split
        decomp.plan(W.quad_from_faces(case), 2, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, PX, PY, k, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case, fields, delta = CASES[k]
        f0 = O.init_equilibrium(case, *fields) + delta
        block = decomp.plan(case, PX, PY)[rank]
        s = OracleStepper(block, f0)
        for _ in range(STEPS):
            s.step(1)
            decomp.exchange_dist(block, s, dist, lambda shape: torch.empty(shape, dtype=torch.float64))
        sums = decomp.allreduce_sums(s.owned_sums(), dist)
        ref = _single(case, fields, delta)
        ok = bool(np.array_equal(s.owned(), ref[:, block.j0:block.j1, block.i0:block.i1]))
        good_sums = bool(np.allclose(sums, O.conserved(case, ref), rtol=1e-13, atol=1e-15))
        q.put((rank, ok, good_sums))
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
@pytest.mark.parametrize("PX,PY,k", [(2, 1, 3), (1, 2, 2), (2, 2, 1), (2, 2, 3)])
def test_gloo_ranks_match_single_mesh(PX, PY, k):
    world, port = PX * PY, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, PX, PY, k, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in res), res
    assert all(s for _, _, s in res), res
