"""Spatial domain decomposition on the GPU (paper Sec. 2.1, Eq. 9: the upwind common flux is the only
coupling between elements): slabs of one mesh as separate contexts with exchange x faces, stepped
stage by stage through the C ABI with the neighbours' element layers handed over before every stage
(bgk_halo_pack into device buffers, bgk_set_halo), must reproduce the undivided context's run. The
exchange here is done by the host on one GPU (no kernel waits for another); between GPUs the same
buffers go through the partition driver's point-to-point messages."""
import numpy as np
import pytest

from paper_2308_06196_gb300 import _build
from paper_2308_06196_gb300 import partition as P
from paper_2308_06196_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def solver(c, **kw):
    from paper_2308_06196_gb300.bgk import Solver

    k = W.mesh_kwargs(c)
    return Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                  bc=c.get("bc"), bc_state=c.get("bc_state"), limiter=c.get("limiter", False), vtiles_per_task=4,
                  **kw)


def rows(c, sc):
    ne, n1 = list(c["nelem"]), c["p"] + 1
    nes = list(sc["nelem"])
    e0, npe = sc["x_range"][0], n1**3
    out = []
    for ez in range(nes[2]):
        for ey in range(nes[1]):
            for ex in range(nes[0]):
                eg = (e0 + ex) + ne[0] * (ey + ne[1] * ez)
                out.extend(range(eg * npe, (eg + 1) * npe))
    return np.array(out)


def run_slabs(c, world, steps, prim_fn, dt):
    import torch

    scs = [P.slab_config(c, r, world) for r in range(world)]
    sl = [solver(sc) for sc in scs]
    for s in sl:
        s.set_state(prim_fn(s.points()))
    n = sl[0].halo_floats()
    packs = [(torch.empty(n, dtype=torch.float32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"))
             for _ in sl]
    for _ in range(steps):
        for st in range(3):
            for s, (lo, hi) in zip(sl, packs):
                s.halo_pack(st, lo, hi)
            for s in sl:
                s.synchronize()
            for r, (s, sc) in enumerate(zip(sl, scs)):
                if sc["bc"][0][0] == P.EXCHANGE:
                    s.set_halo(P.LO, packs[(r - 1) % world][1])
                if sc["bc"][0][1] == P.EXCHANGE:
                    s.set_halo(P.HI, packs[(r + 1) % world][0])
            for s in sl:
                s.stage(dt, st)
    out = [(s.get_f(), s.moments(), sc) for s, sc in zip(sl, scs)]
    for s in sl:
        s.close()
    return out


@pytest.mark.parametrize("case,world", [("periodic", 2), ("periodic", 3), ("dirichlet", 3)])
def test_gpu_slabs_equal_the_whole(case, world):
    _build.build()
    if case == "periodic":  # the Taylor-Green kernel configuration (p = 3, lean form) on a 5 x 2 x 2 box
        c = W.config("taylor_green", nelem=(5, 2, 2), hi=(1.0, 0.5, 0.5), nv=(8, 8, 8))

        def prim(x):
            return W.smooth_prim(x, 3, seed=3, amp=0.2)
    else:  # a Dirichlet duct at p = 2 with the limiter (general form), uneven slabs of 7 elements
        left, right = (1.0, 0.3, 0.0, 0.0, 1.0), (0.4, -0.2, 0.0, 0.0, 1.3)
        c = W.config("mach5", nelem=(7, 2, 2), hi=(7.0 / 8.0, 0.25, 0.25), nv=(12, 12, 12), vlo=(-6.0,) * 3,
                     vhi=(6.0,) * 3, tau=5e-3)
        c["bc"] = ((W.DIRICHLET, W.DIRICHLET), (W.PERIODIC, W.PERIODIC), (W.PERIODIC, W.PERIODIC))
        c["bc_state"] = ((left, right), ((0,) * 5, (0,) * 5), ((0,) * 5, (0,) * 5))

        def prim(x):  # the two end states meeting in the middle of the duct
            P = np.where((x[:, 0] < 7.0 / 16.0)[:, None], np.array(left), np.array(right))
            return np.ascontiguousarray(P)
    steps = 3
    s = solver(c)
    s.set_state(prim(s.points()))
    dt = s.dt(0.1)
    s.step(dt, steps)
    fw, Qw = s.get_f(), s.moments()
    s.close()
    for f, Q, sc in run_slabs(c, world, steps, prim, dt):
        r = rows(c, sc)
        assert np.abs(f - fw[r]).max() <= 1e-6 * np.abs(fw).max()
        assert np.abs(Q - Qw[r]).max() <= 1e-6 * np.abs(Qw).max()


def test_gpu_exchange_context_refuses_the_whole_step():
    from paper_2308_06196_gb300.bgk import BgkError

    _build.build()
    c = P.slab_config(W.config("taylor_green", nelem=(4, 2, 2), nv=(8, 8, 8)), 0, 2)
    s = solver(c)
    s.set_state(W.smooth_prim(s.points(), 3, seed=1))
    with pytest.raises(BgkError):
        s.step(s.dt(0.1), 1)
    s.close()
