"""Spatial domain decomposition (the upwind common flux of paper Sec. 2.1, Eq. 9 is the only coupling
between elements): the mesh cut into slabs along x, each slab stepped on its own with the neighbours'
element layers exchanged before every RK stage, must reproduce the undivided run. CPU only: the slabs
are FP64 oracle problems with exchange faces, driven by the package's partition driver, in one process
and as gloo ranks."""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import partition as P
from paper_2308_06196_gb300 import workloads as W

torch = pytest.importorskip("torch")


def box(nelem=(5, 2, 2), p=2, nv=(6, 5, 6), tau=0.05, bc=None, bc_state=None, dim=3, limiter=False):
    lo = [0.0] * dim
    hi = [1.0 + 0.25 * d for d in range(dim)]
    c = dict(dim=dim, nelem=tuple(nelem[:dim]), lo=tuple(lo), hi=tuple(hi), p=p, nv=nv, vlo=(-4.0, -4.5, -4.0),
             vhi=(4.0, 4.0, 4.5), tau=tau)
    if bc is not None:
        c["bc"], c["bc_state"] = bc, bc_state
    c["limiter"] = limiter
    return c


def problem(c):
    k = W.mesh_kwargs(c)
    bc = None if "bc" not in c else np.asarray(c["bc"]).reshape(6)
    bs = None if "bc_state" not in c else np.asarray(c["bc_state"], dtype=float).reshape(6, 5)
    pr = orc.Problem(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"], bc=bc,
                     bc_state=bs)
    pr.set_limiter(c.get("limiter", False))
    return pr


def state(c, pr):
    X = pr.points()
    return W.smooth_prim(X, c["dim"], seed=7, amp=0.25)


def tube(nelem=7):
    """A 1-D x tube with Dirichlet ends of two different states and the limiter on."""
    bc = ((W.DIRICHLET, W.DIRICHLET), (W.PERIODIC, W.PERIODIC), (W.PERIODIC, W.PERIODIC))
    bs = (((1.0, 0.3, 0.0, 0.0, 1.0), (0.4, -0.2, 0.0, 0.0, 1.3)), ((0,) * 5, (0,) * 5), ((0,) * 5, (0,) * 5))
    return box(nelem=(nelem,), p=3, nv=(10, 6, 6), tau=0.02, bc=bc, bc_state=bs, dim=1, limiter=True)


class OracleSlab:
    """The partition driver's slab interface on an oracle problem (halos as CPU tensors in the oracle's
    [face element][node][velocity] order)."""

    def __init__(self, pr):
        self.pr = pr

    def halo_like(self, face):
        return torch.zeros(self.pr.pack_halo(face, 0).size, dtype=torch.float64)

    def pack_halo(self, face, stage):
        return torch.from_numpy(self.pr.pack_halo(face, stage).ravel().copy())

    def set_halo(self, face, t):
        self.pr.set_halo(face, t.numpy())

    def stage(self, dt, s):
        self.pr.stage(dt, s)


def slab_rows(c, sc):
    """Global point indices of slab sc's points, in the slab's own order."""
    ne, n1, dim = list(c["nelem"]) + [1] * (3 - c["dim"]), c["p"] + 1, c["dim"]
    nes = list(sc["nelem"]) + [1] * (3 - dim)
    npe = n1**dim
    e0 = sc["x_range"][0]
    rows = []
    for ez in range(nes[2]):
        for ey in range(nes[1]):
            for ex in range(nes[0]):
                eg = (e0 + ex) + ne[0] * (ey + ne[1] * ez)
                rows.extend(range(eg * npe, (eg + 1) * npe))
    return np.array(rows)


def whole(c, steps):
    pr = problem(c)
    pr.set_state(state(c, pr))
    dt = pr.dt(0.1)
    pr.step(dt, steps)
    return pr.get_f(), dt


def test_three_stages_make_one_step():
    # oracle_stage's three stages in order are oracle_step's arithmetic, bit for bit (limiter on)
    c = box(limiter=True)
    a, b = problem(c), problem(c)
    a.set_state(state(c, a))
    b.set_state(state(c, b))
    dt = a.dt(0.1)
    a.step(dt, 2)
    for _ in range(2):
        for s in range(3):
            b.stage(dt, s)
    assert np.array_equal(a.get_f(), b.get_f())


@pytest.mark.parametrize("case,world", [("box", 2), ("box", 3), ("tube", 3)])
def test_slabs_in_one_process_equal_the_whole(case, world):
    # the exchange done in place (each slab's packed layer handed to its neighbour's halo) before every
    # stage: the slabs' f equals the undivided run's, point for point
    c = box() if case == "box" else tube()
    steps = 3
    fw, dt = whole(c, steps)
    scs = [P.slab_config(c, r, world) for r in range(world)]
    slabs = []
    for sc in scs:
        pr = problem(sc)
        X = pr.points()
        pr.set_state(W.smooth_prim(X, c["dim"], seed=7, amp=0.25) if case == "box" else state(c, pr))
        slabs.append(pr)
    # the global state field must be the same function of the coordinates on every slab
    for pr, sc in zip(slabs, scs):
        assert np.allclose(pr.points(), problem(c).points()[slab_rows(c, sc)], atol=1e-14)
    for _ in range(steps):
        for s in range(3):
            packs = [(pr.pack_halo(P.LO, s), pr.pack_halo(P.HI, s)) for pr in slabs]
            for r, (pr, sc) in enumerate(zip(slabs, scs)):
                if sc["bc"][0][0] == P.EXCHANGE:
                    pr.set_halo(P.LO, packs[(r - 1) % world][1])
                if sc["bc"][0][1] == P.EXCHANGE:
                    pr.set_halo(P.HI, packs[(r + 1) % world][0])
            for pr in slabs:
                pr.stage(dt, s)
    for pr, sc in zip(slabs, scs):
        d = np.abs(pr.get_f() - fw[slab_rows(c, sc)]).max()
        assert d <= 1e-13 * np.abs(fw).max(), d


def test_missing_exchange_changes_the_result():
    # the halo matters: leaving a slab's halo at zero (no exchange) moves its boundary elements' f
    c = box()
    fw, dt = whole(c, 1)
    sc = P.slab_config(c, 0, 2)
    pr = problem(sc)
    pr.set_state(state(c, pr))
    pr.step(dt, 1)
    assert np.abs(pr.get_f() - fw[slab_rows(c, sc)]).max() > 1e-3 * np.abs(fw).max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, steps, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = box() if case == "box" else tube()
    sc = P.slab_config(c, rank, world)
    pr = problem(sc)
    pr.set_state(state(c, pr))
    dt = problem(c).dt(0.1)
    stepper = P.SlabStepper(OracleSlab(pr), rank, world, sc["bc"][0], dist)
    stepper.step(dt, steps)
    q.put((rank, pr.get_f()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("box", 2), ("tube", 3)])
def test_gloo_ranks_equal_the_whole(case, world):
    # one slab per gloo rank, the partition driver's point-to-point exchange before every stage; the
    # gathered f equals the undivided oracle run to round-off (1e-13 of max |f|)
    import torch.multiprocessing as mp

    steps = 3
    c = box() if case == "box" else tube()
    fw, _ = whole(c, steps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        sc = P.slab_config(c, r, world)
        d = np.abs(res[r] - fw[slab_rows(c, sc)]).max()
        assert d <= 1e-13 * np.abs(fw).max(), (r, d)


def test_slab_config_cuts_and_faces():
    c = W.config("mach5")
    cuts = [P.slab_range(128, r, 3) for r in range(3)]
    assert cuts == [(0, 43), (43, 86), (86, 128)]
    s0, s1, s2 = (P.slab_config(dict(c, bc=W.mach5_bc(c)[0]), r, 3) for r in range(3))
    assert s0["bc"][0] == (W.DIRICHLET, P.EXCHANGE) and s1["bc"][0] == (P.EXCHANGE, P.EXCHANGE)
    assert s2["bc"][0] == (P.EXCHANGE, W.DIRICHLET)
    assert s1["lo"][0] == pytest.approx(43 * 16.0 / 128) and s2["hi"][0] == pytest.approx(16.0)
    tg = W.config("taylor_green")
    a, b = P.slab_config(tg, 0, 2), P.slab_config(tg, 1, 2)
    assert a["bc"][0] == (P.EXCHANGE, P.EXCHANGE) and b["bc"][0] == (P.EXCHANGE, P.EXCHANGE)
    assert P.slab_config(tg, 0, 1)["bc"][0] == (W.PERIODIC, W.PERIODIC)
    with pytest.raises(ValueError):
        P.slab_config(dict(tg, nelem=(2, 16, 16)), 0, 3)
