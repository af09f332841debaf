"""Batched line-element problems (bgk_batch_*): many independent Sod shock tubes of uneven size,
degree and velocity grid stepped by one persistent stage launch and one Newton launch per RK stage.
The batch must give each member the result it gets alone (same kernels' arithmetic, scheduled
together), and that result must match the FP64 oracle within the FP32-split tolerance."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_06196_gb300 import _build, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def solver(m, **opts):
    from paper_2308_06196_gb300.bgk import Solver

    k = W.mesh_kwargs(m)
    opts.setdefault("chunks", 1)
    return Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                  bc=m["bc"], bc_state=m["bc_state"], **opts)


def oracle_problem(m):
    k = W.mesh_kwargs(m)
    return orc.Problem(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                       bc=np.asarray(m["bc"]).reshape(6), bc_state=np.asarray(m["bc_state"], dtype=float).reshape(30))


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def setup(members, **opts):
    ss = []
    for m in members:
        s = solver(m, **opts)
        s.set_state(W.prim_sod(s.points(), m["left"], m["right"]))
        ss.append(s)
    return ss


def small_ensemble(n=9, seed=5, elements=(5, 21), nvs=(12, 16)):
    return W.sod_members(members=n, seed=seed, elements=elements, nvs=nvs)


def test_batch_equals_members_alone():
    from paper_2308_06196_gb300.bgk import Batch

    ms = small_ensemble()
    alone, batched = setup(ms), setup(ms)
    dts = [s.dt(0.1) for s in alone]
    for s, dt in zip(alone, dts):
        s.step(dt, 4)
    b = Batch(batched)
    b.step(dts, 4)
    b.synchronize()
    for q, (sa, sb) in enumerate(zip(alone, batched)):
        # the same stage and Newton arithmetic per member; only the launch differs
        assert rel(sb.moments(), sa.moments()) <= 1e-6, q
        assert rel(sb.get_f(), sa.get_f()) <= 1e-6, q
    b.close()


def test_batch_matches_oracle_100_steps():
    # stiff members (dt = tau: every stage relaxes fully towards the Maxwellian) over 100 steps, the
    # FP32-split tolerance of 1e-5 relative in the moments
    from paper_2308_06196_gb300.bgk import Batch

    ms = small_ensemble(n=4, seed=11, elements=(6, 12), nvs=(12,))
    ms += W.sod_members(members=2, seed=12, elements=(6, 10), nvs=(12,), tau=(1e-4, 1e-3))
    ss = setup(ms)
    prs = []
    for m in ms:
        pr = oracle_problem(m)
        pr.set_state(W.prim_sod(pr.points(), m["left"], m["right"]))
        prs.append(pr)
    dts = [pr.dt(0.1) for pr in prs]
    b = Batch(ss)
    b.step(dts, 100)
    b.synchronize()
    for pr, dt in zip(prs, dts):
        pr.step(dt, 100)
    for q, (s, pr) in enumerate(zip(ss, prs)):
        assert rel(s.moments(), pr.moments()) < 1e-5, q
        assert rel(s.get_f(), pr.get_f()) < 1e-5, q


def test_batch_uniform_members_stay_uniform():
    # equal Dirichlet states on both ends and a uniform initial state: nothing may change
    from paper_2308_06196_gb300.bgk import Batch

    ms = small_ensemble(n=5, seed=2)
    for m in ms:
        m["right"] = m["left"]
        st = np.asarray(m["bc_state"], dtype=float)
        st[0, 1] = st[0, 0]
        m["bc_state"] = st
    ss = setup(ms)
    Q0 = [s.moments() for s in ss]
    b = Batch(ss)
    b.step([s.dt(0.1) for s in ss], 60)
    b.synchronize()
    for q, s in enumerate(ss):
        # FP32 storage: a few rounding units, without drift (unbiased 2^x, exact moment weights,
        # exactly summing stage coefficients)
        assert rel(s.moments(), Q0[q]) < 1e-6, q


def test_batch_autotune_keeps_results():
    from paper_2308_06196_gb300.bgk import Batch

    ms = small_ensemble(n=6, seed=8, elements=(8, 40), nvs=(12, 16, 24))
    ref, tuned = setup(ms), setup(ms)
    dts = [s.dt(0.1) for s in ref]
    b0 = Batch(ref)
    b0.step(dts, 3)
    b0.synchronize()
    b1 = Batch(tuned)
    b1.autotune()
    b1.step(dts, 3)
    b1.synchronize()
    for q, (s0, s1) in enumerate(zip(ref, tuned)):
        # another task length only regroups the FP32 partial moment sums
        assert rel(s1.moments(), s0.moments()) < 2e-6, q
    b0.close()
    b1.close()


def test_batch_rejects_unsuitable_members():
    from paper_2308_06196_gb300.bgk import Batch, BgkError

    ms = small_ensemble(n=2)
    ok = setup(ms)
    with pytest.raises(BgkError):
        Batch([ok[0], ok[0]])  # a member twice
    multi = setup(ms[:1], chunks=0)  # octant chunks: stage buffers shared between chunks
    with pytest.raises(BgkError):
        Batch([ok[1], multi[0]])


def test_full_sod_ensemble_sampled_members():
    # the full 256-member ensemble in one batch (the measured workload): two steps, then four sampled
    # members against the same members stepped alone
    from paper_2308_06196_gb300.bgk import Batch

    ms = W.sod_members(**W.config("sod_ensemble"))
    ss = setup(ms)
    b = Batch(ss)
    b.autotune()
    dts = [s.dt(0.1) for s in ss]
    b.step(dts, 2)
    b.synchronize()
    for q in (0, 17, 128, 255):
        alone = setup([ms[q]])[0]
        alone.step(dts[q], 2)
        # the autotuned task length may differ from the member's own: regrouped FP32 partials only
        assert rel(ss[q].moments(), alone.moments()) < 2e-6, q
        assert np.all(np.isfinite(ss[q].moments()))
        alone.close()
    b.close()
