"""The allocation-free entry point bgk_equilibrium_noalloc, for callers that cannot call cudaMalloc
(code inside another framework's memory pool or allocator hooks, or under a no-allocation policy
after start-up). It must give the same moments and conservative Maxwellian as the regular path
(a context's bgk_set_f followed by bgk_moments / bgk_equilibrium), on two calls in a row, using
only the library's fixed static scratch. This file is collected last on purpose: if it fails, a
run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_path_twice():
    import torch

    _build.build()
    from paper_2308_06196_gb300 import bgk

    # 3-D, 3 x 2 x 2 elements at p = 2 (108 points), 16^3 velocities (two 2048-velocity groups)
    dim, ne, p, n, L, tau = 3, [3, 2, 2], 2, 16, 5.0, 0.05
    pr = orc.Problem(dim, ne, [0.0] * 3, [1.0] * 3, p, (n,) * 3, (-L,) * 3, (L,) * 3, tau)
    s = bgk.Solver(dim, ne, [0.0] * 3, [1.0] * 3, p, (n,) * 3, (-L,) * 3, (L,) * 3, tau)
    xi, w = pr.xi, pr.w
    psi = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], 0.5 * (xi**2).sum(1)], 1)
    for call, seed in enumerate((31, 32)):
        pr.set_state(W.smooth_prim(pr.points(), dim, seed=seed))
        f = pr.get_f() * W.noise((pr.npts, pr.nvel), seed=seed + 100, amp=0.1)
        # regular path (allocating context)
        s.set_f(f)
        Q_ref, P_ref = s.moments(), s.equilibrium()
        # allocation-free path on caller-owned tensors
        f_dev = torch.tensor(f, dtype=torch.float32, device="cuda")
        Q_dev = torch.full((pr.npts, 5), float("nan"), dtype=torch.float64, device="cuda")
        P_dev = torch.full((pr.npts, 5), float("nan"), dtype=torch.float64, device="cuda")
        rc = bgk.equilibrium_noalloc(f_dev, (n,) * 3, (-L,) * 3, (L,) * 3, Q_dev, P_dev)
        assert rc == 0, f"call {call}: status {rc}"
        Q, P = Q_dev.cpu().numpy(), P_dev.cpu().numpy()
        # same quantities within the FP32 summation tolerance of the moments (both paths sum FP32
        # products of the same FP32 f, in different orders: ~1e-7 relative each)
        assert np.abs(Q - Q_ref).max() <= 5e-7 * np.abs(Q_ref).max(), call
        assert np.abs(P - P_ref).max() <= 5e-6 * np.abs(P_ref).max(), call
        # and the FP64 Newton property on its own output
        for q, pp in zip(Q[::7], P[::7]):
            g = pp[0] / (2 * np.pi * pp[4]) ** 1.5 * np.exp(-((xi - pp[1:4]) ** 2).sum(1) / (2 * pp[4]))
            assert np.all(np.abs((w * g) @ psi - q) <= 1e-12 * np.abs(q).max())


def test_noalloc_allocates_nothing():
    # the defining property: after a first call (the sizing point, which may load the library's module
    # and its static scratch on this device), further calls change neither the device's free memory
    # nor the torch allocator's total
    import torch

    _build.build()
    from paper_2308_06196_gb300 import bgk

    n, L = 12, 5.0
    pr = orc.Problem(1, [4], [0.0], [1.0], 2, (n,) * 3, (-L,) * 3, (L,) * 3, 0.05)
    pr.set_state(W.smooth_prim(pr.points(), 1, seed=51))
    f_dev = torch.tensor(pr.get_f(), dtype=torch.float32, device="cuda")
    Q_dev = torch.zeros((pr.npts, 5), dtype=torch.float64, device="cuda")
    P_dev = torch.zeros((pr.npts, 5), dtype=torch.float64, device="cuda")
    assert bgk.equilibrium_noalloc(f_dev, (n,) * 3, (-L,) * 3, (L,) * 3, Q_dev, P_dev) == 0
    Q0 = Q_dev.clone()
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        assert bgk.equilibrium_noalloc(f_dev, (n,) * 3, (-L,) * 3, (L,) * 3, Q_dev, P_dev) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(Q_dev, Q0)


def test_noalloc_rejects_oversized_request():
    import torch

    _build.build()
    from paper_2308_06196_gb300 import bgk

    # 24^3 velocities: 7 groups, (5 * 7 + 8) floats per point -> at most ~97k points in 16 MiB
    npts = 200_000
    f_dev = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    Q_dev = torch.zeros((1, 5), dtype=torch.float64, device="cuda")
    vg = bgk.make_vgrid((24, 24, 24), (-5.0,) * 3, (5.0,) * 3)
    import ctypes as C

    rc = bgk.lib().bgk_equilibrium_noalloc(C.c_void_p(f_dev.data_ptr()), npts, C.byref(vg),
                                           C.c_void_p(Q_dev.data_ptr()), C.c_void_p(Q_dev.data_ptr()), None)
    assert rc == bgk.BGK_EINVAL


def test_noalloc_planar_velocity_space():
    # m = 2 (n[2] = 1): 24^2 velocities on a 3-element p = 3 line, against the regular path and the
    # Newton property of the planar Maxwellian
    import torch

    _build.build()
    from paper_2308_06196_gb300 import bgk

    ne, p, n, L, tau = 3, 3, 24, 6.0, 0.05
    grid = ((n, n, 1), (-L, -L, 0.0), (L, L, 0.0))
    pr = orc.Problem(1, [ne], [0.0], [1.0], p, *grid, tau)
    s = bgk.Solver(1, [ne], [0.0], [1.0], p, *grid, tau)
    P0 = W.smooth_prim(pr.points(), 1, seed=41)
    P0[:, 3] = 0.0
    pr.set_state(P0)
    f = pr.get_f() * W.noise((pr.npts, pr.nvel), seed=42, amp=0.1)
    s.set_f(f)
    Q_ref, P_ref = s.moments(), s.equilibrium()
    f_dev = torch.tensor(f, dtype=torch.float32, device="cuda")
    Q_dev = torch.full((pr.npts, 5), float("nan"), dtype=torch.float64, device="cuda")
    P_dev = torch.full((pr.npts, 5), float("nan"), dtype=torch.float64, device="cuda")
    assert bgk.equilibrium_noalloc(f_dev, *grid, Q_dev, P_dev) == 0
    Q, P = Q_dev.cpu().numpy(), P_dev.cpu().numpy()
    assert np.all(Q[:, 3] == 0.0)
    assert np.abs(Q - Q_ref).max() <= 5e-7 * np.abs(Q_ref).max()
    assert np.abs(P - P_ref).max() <= 5e-6 * np.abs(P_ref).max()
    xi, w = pr.xi, pr.w
    psi = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], 0 * xi[:, 0], 0.5 * (xi[:, :2] ** 2).sum(1)], 1)
    for q, pp in zip(Q, P):
        g = pp[0] / (2 * np.pi * pp[4]) * np.exp(-((xi[:, :2] - pp[1:3]) ** 2).sum(1) / (2 * pp[4]))
        assert np.all(np.abs((w * g) @ psi - q) <= 1e-12 * np.abs(q).max())
