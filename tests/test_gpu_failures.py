"""Failure detection through the C ABI, all on the host or in data (nothing faults or hangs the device):
non-physical states met on the device are reported (BGK_EDOMAIN, sticky), invalid descriptors are
rejected (BGK_EINVAL) and a configuration larger than the free device memory is refused before any
allocation (BGK_ENOMEM). Checkpoint and resume through bgk_get_f / bgk_set_f continue the run to FP32
rounding."""
import numpy as np
import pytest

from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def line(**kw):
    """A small line problem; keywords override the mesh / grid arguments, the rest go to the options."""
    from paper_2308_06196_gb300.bgk import Solver

    args = dict(dim=1, nelem=[4], lo=[0.0], hi=[1.0], p=2, nv=(8, 8, 8), vlo=(-4.0,) * 3, vhi=(4.0,) * 3, tau=0.05)
    opts = {k: kw.pop(k) for k in list(kw) if k not in args}
    args.update(kw)
    return Solver(args["dim"], args["nelem"], args["lo"], args["hi"], args["p"], args["nv"], args["vlo"],
                  args["vhi"], args["tau"], **opts)


@pytest.mark.parametrize("bad", ["nan_rho", "neg_theta"])
def test_non_physical_state_is_reported_and_sticky(bad):
    from paper_2308_06196_gb300.bgk import BGK_EDOMAIN, BgkError

    s = line()
    prim = W.smooth_prim(s.points(), 1, seed=1)
    if bad == "nan_rho":
        prim[3, 0] = np.nan
    else:
        prim[5, 4] = -0.5
    with pytest.raises(BgkError) as err:
        s.set_state(prim)
    assert err.value.code == BGK_EDOMAIN
    with pytest.raises(BgkError) as err:  # the status stays with the context
        s.step(1e-3, 1)
    assert err.value.code == BGK_EDOMAIN


def test_negative_density_from_f_is_reported():
    from paper_2308_06196_gb300.bgk import BGK_EDOMAIN, BgkError

    s = line()
    s.set_state(W.smooth_prim(s.points(), 1, seed=2))
    f = s.get_f()
    f[2] = -np.abs(f[2])  # one point with a negative density
    with pytest.raises(BgkError) as err:
        s.set_f(f)
        s.synchronize()
    assert err.value.code == BGK_EDOMAIN


@pytest.mark.parametrize("kw", [dict(p=0), dict(p=9), dict(dim=0, nelem=[], lo=[], hi=[]),
                                dict(tau=0.0), dict(tau=float("nan")), dict(nv=(1, 8, 8)),
                                dict(vlo=(4.0, -4.0, -4.0)),
                                dict(bc=[[1, 1], [0, 0], [0, 0]], bc_state=np.zeros((3, 2, 5)))])
def test_invalid_descriptors_are_rejected(kw):
    from paper_2308_06196_gb300.bgk import BGK_EINVAL, BgkError

    with pytest.raises(BgkError) as err:
        line(**kw)
    assert err.value.code == BGK_EINVAL


def test_configuration_beyond_device_memory_is_refused_before_allocating():
    from paper_2308_06196_gb300.bgk import BGK_ENOMEM, BgkError, Solver

    # 64^3 hexahedra at p = 3 with 48^3 velocities: 1.8e12 degrees of freedom, about 7 TB in FP32
    with pytest.raises(BgkError) as err:
        Solver(3, [64, 64, 64], [0.0] * 3, [1.0] * 3, 3, (48, 48, 48), (-6.0,) * 3, (6.0,) * 3, 0.01)
    assert err.value.code == BGK_ENOMEM


def test_checkpoint_and_resume():
    from paper_2308_06196_gb300.bgk import Solver

    k = dict(dim=3, nelem=[3, 2, 2], lo=[0.0] * 3, hi=[1.0] * 3, p=2, nv=(8, 8, 8), vlo=(-4.0,) * 3, vhi=(4.0,) * 3,
             tau=0.02)

    def make():
        return Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])

    a, b = make(), make()
    prim = W.smooth_prim(a.points(), 3, seed=4)
    a.set_state(prim)
    b.set_state(prim)
    dt = a.dt(0.1)
    a.step(dt, 10)  # uninterrupted
    b.step(dt, 4)
    ckpt = b.get_f()  # checkpoint
    b.close()
    c = make()
    c.set_f(ckpt)  # resume in a fresh context
    c.step(dt, 6)
    Qa, Qc = a.moments(), c.moments()
    # the resumed run starts its first Newton solve cold (the warm start is not part of the checkpoint)
    assert np.abs(Qc - Qa).max() <= 1e-6 * np.abs(Qa).max()
