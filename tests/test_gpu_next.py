"""The widened rows on the GPU against the FP64 oracle: the Zhang-Shu positivity limiter (Sec. 2.1,
Eqs. 10-11) in the line kernel, the general hexahedral kernel and the plain all-FP64 form, the
non-conservative ablation (the continuous Maxwellian of the moments, Sec. 2.1, Eq. 13) and the
variable collision time tau = mu(theta) / P (Sec. 2, Eq. 5)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def make(dim, ne, p, N, L, tau, bc=None, bcs=None, limiter=False, continuous=False, **opts):
    from paper_2308_06196_gb300.bgk import Solver, MAXWELLIAN_CONTINUOUS, MAXWELLIAN_CONSERVATIVE

    lo, hi = [0.0] * dim, [1.0] * dim
    s = Solver(dim, ne, lo, hi, p, (N,) * 3, (-L,) * 3, (L,) * 3, tau, bc=bc, bc_state=bcs, limiter=limiter,
               maxwellian=MAXWELLIAN_CONTINUOUS if continuous else MAXWELLIAN_CONSERVATIVE, **opts)
    pr = orc.Problem(dim, ne, lo, hi, p, (N,) * 3, (-L,) * 3, (L,) * 3, tau,
                     bc=None if bc is None else np.asarray(bc).reshape(6),
                     bc_state=None if bcs is None else np.asarray(bcs, dtype=float).reshape(30))
    pr.set_limiter(limiter)
    pr.set_maxwellian(continuous)
    return s, pr


def tube(left=(1.0, 1.0), right=(0.125, 0.8)):
    bc = [[W.DIRICHLET, W.DIRICHLET], [0, 0], [0, 0]]
    bcs = np.zeros((3, 2, 5))
    bcs[0, 0] = [left[0], 0, 0, 0, left[1]]
    bcs[0, 1] = [right[0], 0, 0, 0, right[1]]
    return bc, bcs


def positivity_ratio(f, p, dim, nvel):
    _, w = orc.gauss_legendre(p + 1)
    Wn = w if dim == 1 else np.einsum("i,j,k->kji", w, w, w).ravel()
    fe = f.reshape(-1, len(Wn), nvel)
    mean = np.einsum("i,eik->ek", Wn, fe) / Wn.sum()
    pos = mean > 1e-12 * f.max()
    return (fe.min(axis=1)[pos] / mean[pos]).min()


def test_limiter_line_kernel_sod():
    bc, bcs = tube()
    s, pr = make(1, [12], 3, 12, 8.0, 1e-3, bc, bcs, limiter=True, chunks=1)
    prim = W.prim_sod(pr.points(), (1.0, 1.0), (0.125, 0.8))
    s.set_state(prim)
    pr.set_state(prim)
    dt = pr.dt(0.1)
    s.step(dt, 10)
    pr.step(dt, 10)
    f = s.get_f()
    assert rel(s.moments(), pr.moments()) < 1e-5
    assert rel(f, pr.get_f()) < 1e-5
    # positive wherever the element mean is (FP32 round-off of the contraction)
    assert positivity_ratio(f, 3, 1, s.nvel) >= -1e-5


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
def test_limiter_hexahedra_tube(precision, tol):
    # the tube along x on a 4 x 2 x 2 hexahedral mesh, Dirichlet x-ends and periodic y, z: the
    # general kernel's cross-layer limiter (FP32-split) and the FP64 form's limiter pass
    bc, bcs = tube()
    s, pr = make(3, [4, 2, 2], 2, 8, 6.0, 2e-3, bc, bcs, limiter=True, precision=precision)
    prim = W.prim_sod(pr.points(), (1.0, 1.0), (0.125, 0.8))
    s.set_state(prim)
    pr.set_state(prim)
    dt = pr.dt(0.1)
    s.step(dt, 5)
    pr.step(dt, 5)
    assert rel(s.moments(), pr.moments()) < tol
    assert rel(s.get_f(), pr.get_f()) < tol


def test_continuous_maxwellian_ablation_line():
    # periodic line, coarse velocity grid: the ablation's moments drift (the conservation error the
    # paper attributes to the sampled Maxwellian), and the GPU follows the oracle's drift
    s, pr = make(1, [8], 3, 10, 10.0, 1e-2, continuous=True)
    prim = W.smooth_prim(pr.points(), 1, seed=6, amp=0.3)
    s.set_state(prim)
    pr.set_state(prim)
    _, w = orc.gauss_legendre(4)

    def tot(Q):
        return (Q.reshape(8, 4, 5) * w[None, :, None]).sum((0, 1))

    T0 = tot(pr.moments())
    dt = pr.dt(0.1)
    s.step(dt, 20)
    pr.step(dt, 20)
    d_orc, d_gpu = tot(pr.moments()) - T0, tot(s.moments()) - T0
    assert np.abs(d_orc).max() > 1e-4 * np.abs(T0).max()  # far above round-off
    assert np.abs(d_gpu - d_orc).max() <= 1e-3 * np.abs(d_orc).max() + 1e-6 * np.abs(T0).max()
    assert rel(s.moments(), pr.moments()) < 1e-5


def test_batch_with_limiter_equals_members_alone():
    from paper_2308_06196_gb300.bgk import Batch, Solver

    ms = W.sod_members(members=4, seed=21, elements=(6, 14), nvs=(12,), rho=(0.05, 1.0))

    def build():
        out = []
        for m in ms:
            k = W.mesh_kwargs(m)
            x = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                       bc=m["bc"], bc_state=m["bc_state"], chunks=1, limiter=True)
            x.set_state(W.prim_sod(x.points(), m["left"], m["right"]))
            out.append(x)
        return out

    alone, batched = build(), build()
    dts = [x.dt(0.1) for x in alone]
    for x, dt in zip(alone, dts):
        x.step(dt, 5)
    b = Batch(batched)
    b.step(dts, 5)
    b.synchronize()
    for q, (xa, xb) in enumerate(zip(alone, batched)):
        assert rel(xb.moments(), xa.moments()) <= 1e-6, q
    b.close()


def test_variable_tau_line_and_hexahedra():
    # tau = mu(theta) / P varies along a Sod tube: line kernel (FP32-split), general hexahedral kernel
    # (FP32-split) and the FP64 form against the oracle
    bc, bcs = tube()
    for dim, ne, p, N, precision, tol in ((1, [10], 3, 12, 0, 1e-5), (3, [4, 2, 2], 2, 8, 0, 1e-5),
                                          (3, [4, 2, 2], 2, 8, 1, 1e-10)):
        extra = dict(chunks=1) if dim == 1 else {}
        s, pr = make(dim, ne, p, N, 7.0, 1.0, bc, bcs, precision=precision, mu_ref=2e-3, mu_omega=0.81, **extra)
        pr.set_viscosity(2e-3, 0.81)
        prim = W.prim_sod(pr.points(), (1.0, 1.0), (0.125, 0.8))
        s.set_state(prim)
        pr.set_state(prim)
        dt = min(pr.dt(0.1), s.dt(0.1))
        assert dt < 1.0  # the state's smallest tau, not the unused constant
        s.step(dt, 6)
        pr.step(dt, 6)
        assert rel(s.moments(), pr.moments()) < tol, (dim, precision)
        assert rel(s.get_f(), pr.get_f()) < tol, (dim, precision)


@pytest.mark.parametrize("p", [2, 3])
def test_variable_tau_with_body_force(p):
    # a per-point collision time and the body-force source together (the general hexahedral kernels):
    # the Maxwellian's weight is the node's own b dt / tau plus the force polynomial, against the oracle
    bc, bcs = tube()
    force = (0.3, 0.1, 0.0)
    s, _ = make(3, [4, 2, 2], p, 8, 7.0, 1.0, bc, bcs, mu_ref=2e-3, mu_omega=0.81, body_force=force)
    pr = orc.Problem(3, [4, 2, 2], [0.0] * 3, [1.0] * 3, p, (8,) * 3, (-7.0,) * 3, (7.0,) * 3, 1.0,
                     bc=np.asarray(bc).reshape(6), bc_state=np.asarray(bcs, dtype=float).reshape(30), force=force)
    pr.set_viscosity(2e-3, 0.81)
    prim = W.prim_sod(pr.points(), (1.0, 1.0), (0.125, 0.8))
    s.set_state(prim)
    pr.set_state(prim)
    dt = min(pr.dt(0.1), s.dt(0.1))
    s.step(dt, 6)
    pr.step(dt, 6)
    assert rel(s.moments(), pr.moments()) < 1e-5
    assert rel(s.get_f(), pr.get_f()) < 1e-5


@pytest.mark.parametrize("p", [2, 3])
def test_general_kernel_matches_lean_and_oracle(p):
    # a positive smooth periodic state: the limiter never acts, so the general kernel (limiter on)
    # must give the lean kernel's result; both against the oracle
    s_lean, pr = make(3, [3, 3, 3], p, 12, 5.0, 2e-3)
    s_gen, _ = make(3, [3, 3, 3], p, 12, 5.0, 2e-3, limiter=True)
    prim = W.smooth_prim(pr.points(), 3, seed=9, amp=0.2)
    for x in (s_lean, s_gen, pr):
        x.set_state(prim)
    dt = pr.dt(0.1)
    s_lean.step(dt, 3)
    s_gen.step(dt, 3)
    pr.step(dt, 3)
    assert rel(s_gen.moments(), s_lean.moments()) < 1e-6
    assert rel(s_gen.moments(), pr.moments()) < 1e-5
    assert rel(s_gen.get_f(), pr.get_f()) < 1e-5
