"""Seeded synthetic workloads shaped like the paper's flows (the paper's datasets are not used).

This module holds only problem definitions and input fields: meshes, velocity grids, relaxation
times and the primitive state (rho, u, v, w, T) at given node coordinates, plus seeded random
perturbations. None of the method's arithmetic (Maxwellians, moments, FR operators) is here, so
both the CUDA library and the CPU oracle can take their inputs from it.
"""
from __future__ import annotations

import math

import numpy as np

PERIODIC, DIRICHLET, WALL = 0, 1, 2
TWO_PI = 2.0 * math.pi

# Workloads. Each entry: mesh (dim, nelem, lo, hi, bc, bc_state), degree p, velocity grid (nv, vlo,
# vhi), relaxation time tau, CFL number for the explicit step and the number of steps.
CONFIGS = {
    # 1-D periodic line, 32 elements at p = 3, 16^3 velocities on [-6, 6]^3: correctness workload
    "periodic1d": dict(dim=1, nelem=(32,), lo=(0.0,), hi=(1.0,), p=3, nv=(16, 16, 16),
                       vlo=(-6.0,) * 3, vhi=(6.0,) * 3, tau=0.01, cfl=0.1, steps=100),
    # 3-D Taylor-Green-type flow on [0, 2 pi]^3, 16^3 hexahedra at p = 3, 24^3 velocities on [-5, 5]^3
    "taylor_green": dict(dim=3, nelem=(16, 16, 16), lo=(0.0,) * 3, hi=(TWO_PI,) * 3, p=3, nv=(24, 24, 24),
                         vlo=(-5.0,) * 3, vhi=(5.0,) * 3, tau=1e-3, cfl=0.1, steps=50),
    # rarefied channel between two diffuse isothermal walls (y = 0, 1; T_w = 1), periodic in x and z,
    # 32 x 16 x 4 hexahedra at p = 2, 32^3 velocities on [-6, 6]^3, body force 0.01 in x, Kn = 0.1
    # (tau = Kn H / sqrt(pi theta_w / 2), the BGK mean free path with H = 1, theta_w = 1)
    "channel": dict(dim=3, nelem=(32, 16, 4), lo=(0.0,) * 3, hi=(2.0, 1.0, 0.25), p=2, nv=(32, 32, 32),
                    vlo=(-6.0,) * 3, vhi=(6.0,) * 3, tau=0.1 / math.sqrt(math.pi / 2.0), cfl=0.1, steps=50,
                    bc=((PERIODIC, PERIODIC), (WALL, WALL), (PERIODIC, PERIODIC)),
                    bc_state=(((0,) * 5, (0,) * 5), ((0, 0, 0, 0, 1.0), (0, 0, 0, 0, 1.0)), ((0,) * 5, (0,) * 5)),
                    force=(0.01, 0.0, 0.0)),
    # Mach-5 normal shock in a square duct: 128 x 8 x 8 hexahedra at p = 2 on [0, 16] x [0, 1]^2 (cubic
    # elements), periodic y and z, Dirichlet x-ends with the upstream / downstream states, 48^3
    # velocities on [-14, 14]^3, tau = 5e-4; the step at x = 8. The positivity limiter is on: without
    # it the p = 2 solution undershoots at the shock and some point's moments stop admitting a
    # Maxwellian within a few steps (in FP32 and FP64 alike)
    "mach5": dict(dim=3, nelem=(128, 8, 8), lo=(0.0,) * 3, hi=(16.0, 1.0, 1.0), p=2, nv=(48, 48, 48),
                  vlo=(-14.0,) * 3, vhi=(14.0,) * 3, tau=5e-4, cfl=0.1, steps=20, mach=5.0, limiter=True),
    # ensemble of independent 1-D Sod shock tubes on [0, 1] (interface at x = 1/2, gas at rest, Dirichlet
    # ends), drawn from one seed: elements U{16..128}, p U{2, 3}, velocity grid N^3 on [-8, 8]^3 with
    # N in {12, 16, 24, 32}, (rho, T) of each side U[0.125, 1] x U[0.8, 1.25], tau log-uniform [1e-4, 1e-1]
    # transverse shear wave on a periodic line in the two-dimensional velocity space (m = 2: velocity grid
    # N^2, the third axis one node): 65,536 elements at p = 3, 32^2 velocities on [-7, 7]^2, tau = 1e-3;
    # u_y = 0.1 sin(2 pi x) decays by shear viscosity (1.1 GB per FP32 f array, larger than L2)
    "planar_shear": dict(dim=1, nelem=(65536,), lo=(0.0,), hi=(1.0,), p=3, nv=(32, 32, 1), vlo=(-7.0, -7.0, 0.0),
                         vhi=(7.0, 7.0, 0.0), tau=1e-3, cfl=0.1, steps=20, amp=0.1),
    # planar Taylor-Green vortex on quadrilaterals (dim = 2) in the two-dimensional velocity space: [0, 2 pi]^2,
    # 128^2 elements at p = 3 (262,144 points), 32^2 velocities on [-7, 7]^2, Ma 0.1, tau = 1e-3
    "planar_tg": dict(dim=2, nelem=(128, 128), lo=(0.0, 0.0), hi=(TWO_PI, TWO_PI), p=3, nv=(32, 32, 1),
                      vlo=(-7.0, -7.0, 0.0), vhi=(7.0, 7.0, 0.0), tau=1e-3, cfl=0.1, steps=20, mach=0.1),
    "sod_ensemble": dict(members=256, seed=0, elements=(16, 128), degrees=(2, 3), nvs=(12, 16, 24, 32), vmax=8.0,
                         rho=(0.125, 1.0), temp=(0.8, 1.25), tau=(1e-4, 1e-1), cfl=0.1, steps=20),
}


def config(name: str, **override) -> dict:
    c = dict(CONFIGS[name])
    c.update(override)
    return c


def mesh_kwargs(c: dict) -> dict:
    """Arguments common to the CUDA binding's Solver and the oracle's Problem."""
    return dict(dim=c["dim"], nelem=list(c["nelem"]), lo=list(c["lo"]), hi=list(c["hi"]), p=c["p"],
                nv=tuple(c["nv"]), vlo=tuple(c["vlo"]), vhi=tuple(c["vhi"]), tau=c["tau"])


def prim_periodic1d(x: np.ndarray) -> np.ndarray:
    """rho = 1 + 0.1 sin(2 pi x), u = 0, T = 1 (nondimensional, R = 1)."""
    n = len(x)
    P = np.zeros((n, 5))
    P[:, 0] = 1.0 + 0.1 * np.sin(TWO_PI * x[:, 0])
    P[:, 4] = 1.0
    return P


def prim_taylor_green(x: np.ndarray, mach: float = 0.1, gamma: float = 5.0 / 3.0) -> np.ndarray:
    """Taylor-Green vortex: rho = 1, U0 = Ma sqrt(gamma T0) with T0 = 1,
    u = U0 sin x cos y cos z, v = -U0 cos x sin y cos z, w = 0,
    p = 1 + rho U0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2), T = p / rho."""
    U0 = mach * math.sqrt(gamma)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    P = np.zeros((len(x), 5))
    P[:, 0] = 1.0
    P[:, 1] = U0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    P[:, 2] = -U0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    pres = 1.0 + U0 * U0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    P[:, 4] = pres / P[:, 0]
    return P


def prim_shear(x: np.ndarray, amp: float = 0.1) -> np.ndarray:
    """rho = 1, T = 1, u = 0, v = amp sin(2 pi x): a transverse shear wave along x."""
    P = np.zeros((len(x), 5))
    P[:, 0] = 1.0
    P[:, 2] = amp * np.sin(TWO_PI * x[:, 0])
    P[:, 4] = 1.0
    return P


def prim_planar_tg(x: np.ndarray, mach: float = 0.1, gamma: float = 2.0) -> np.ndarray:
    """Planar Taylor-Green vortex (gamma = 2 for the two-dimensional velocity space): rho = 1,
    U0 = Ma sqrt(gamma), u = U0 sin x cos y, v = -U0 cos x sin y, p = 1 + U0^2 / 4 (cos 2x + cos 2y), T = p."""
    U0 = mach * math.sqrt(gamma)
    X, Y = x[:, 0], x[:, 1]
    P = np.zeros((len(x), 5))
    P[:, 0] = 1.0
    P[:, 1] = U0 * np.sin(X) * np.cos(Y)
    P[:, 2] = -U0 * np.cos(X) * np.sin(Y)
    P[:, 4] = 1.0 + U0 * U0 / 4.0 * (np.cos(2 * X) + np.cos(2 * Y))
    return P


def prim_channel(x: np.ndarray) -> np.ndarray:
    """Gas at rest, rho = 1, T = 1."""
    P = np.zeros((len(x), 5))
    P[:, 0] = 1.0
    P[:, 4] = 1.0
    return P


def sod_members(members: int = 256, seed: int = 0, elements=(16, 128), degrees=(2, 3), nvs=(12, 16, 24, 32),
                vmax: float = 8.0, rho=(0.125, 1.0), temp=(0.8, 1.25), tau=(1e-4, 1e-1), **_) -> list:
    """The seeded Sod ensemble: one dict per member with the Solver/Problem arguments (mesh_kwargs
    form plus bc, bc_state) and its left/right states. Draw order per member: E, p, N, rho_L, T_L,
    rho_R, T_R, log10 tau."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(members):
        E = int(rng.integers(elements[0], elements[1] + 1))
        p = int(rng.integers(degrees[0], degrees[1] + 1))
        N = int(nvs[int(rng.integers(0, len(nvs)))])
        rl, tl = rng.uniform(*rho), rng.uniform(*temp)
        rr, tr = rng.uniform(*rho), rng.uniform(*temp)
        t = 10.0 ** rng.uniform(math.log10(tau[0]), math.log10(tau[1]))
        out.append(dict(dim=1, nelem=(E,), lo=(0.0,), hi=(1.0,), p=p, nv=(N, N, N), vlo=(-vmax,) * 3,
                        vhi=(vmax,) * 3, tau=float(t),
                        bc=((DIRICHLET, DIRICHLET), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC)),
                        bc_state=(((rl, 0.0, 0.0, 0.0, tl), (rr, 0.0, 0.0, 0.0, tr)), ((0,) * 5, (0,) * 5),
                                  ((0,) * 5, (0,) * 5)),
                        left=(rl, tl), right=(rr, tr)))
    return out


def rankine_hugoniot(mach: float, gamma: float = 5.0 / 3.0):
    """Upstream (rho, u, T) = (1, M sqrt(gamma), 1) and the downstream state of the normal shock that is
    steady in this frame: rho2 = (gamma+1) M^2 / ((gamma-1) M^2 + 2), p2 = 1 + 2 gamma (M^2 - 1) / (gamma+1),
    u2 = u1 / rho2, T2 = p2 / rho2 (R = 1)."""
    u1 = mach * math.sqrt(gamma)
    r2 = (gamma + 1.0) * mach**2 / ((gamma - 1.0) * mach**2 + 2.0)
    p2 = 1.0 + 2.0 * gamma * (mach**2 - 1.0) / (gamma + 1.0)
    return (1.0, u1, 1.0), (r2, u1 / r2, p2 / r2)


def mach5_bc(c: dict):
    """Boundary kinds and states of the duct: Dirichlet x-ends (upstream, downstream), periodic y, z."""
    (r1, u1, t1), (r2, u2, t2) = rankine_hugoniot(c["mach"])
    bc = ((DIRICHLET, DIRICHLET), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC))
    bcs = (((r1, u1, 0.0, 0.0, t1), (r2, u2, 0.0, 0.0, t2)), ((0,) * 5, (0,) * 5), ((0,) * 5, (0,) * 5))
    return bc, bcs


def prim_mach5(x: np.ndarray, c: dict) -> np.ndarray:
    """The Rankine-Hugoniot step at the middle of the duct."""
    (r1, u1, t1), (r2, u2, t2) = rankine_hugoniot(c["mach"])
    xm = 0.5 * (c["lo"][0] + c["hi"][0])
    up = x[:, 0] < xm
    P = np.zeros((len(x), 5))
    P[:, 0] = np.where(up, r1, r2)
    P[:, 1] = np.where(up, u1, u2)
    P[:, 4] = np.where(up, t1, t2)
    return P


def prim_sod(x: np.ndarray, left, right) -> np.ndarray:
    """Gas at rest with (rho, T) = left for x < 1/2 and right otherwise."""
    P = np.zeros((len(x), 5))
    L = x[:, 0] < 0.5
    P[:, 0] = np.where(L, left[0], right[0])
    P[:, 4] = np.where(L, left[1], right[1])
    return P


PRIM = {"periodic1d": prim_periodic1d, "taylor_green": prim_taylor_green, "channel": prim_channel}


def prim_field(name: str, x: np.ndarray) -> np.ndarray:
    return PRIM[name](x)


def smooth_prim(x: np.ndarray, dim: int, seed: int = 0, amp: float = 0.2) -> np.ndarray:
    """A seeded smooth periodic primitive field on the unit box (random low Fourier modes),
    rho and T bounded away from 0, |U| <= amp."""
    rng = np.random.default_rng(seed)
    n = len(x)
    P = np.zeros((n, 5))

    def field():
        f = np.zeros(n)
        for _ in range(3):
            k = rng.integers(-2, 3, size=3)
            k[dim:] = 0
            ph = rng.uniform(0, TWO_PI)
            f += rng.uniform(-1, 1) * np.cos(TWO_PI * (x @ k) + ph)
        return f / 3.0

    P[:, 0] = 1.0 + amp * field()
    for d in range(3):
        P[:, 1 + d] = amp * field()
    P[:, 4] = 1.0 + amp * field()
    return P


def curved_nodes(x: np.ndarray, lo, hi, nelem, eps: float = 0.1, kind: str = "bump") -> np.ndarray:
    """Physical coordinates of the solution nodes of a curvilinear hexahedral mesh, from the affine node
    coordinates x [n, 3] of the box [lo, hi] with nelem elements per direction.

    kind = "bump": X = x + eps (h_x b(y), h_y b(z), h_z b(x)) with b = 4 t (1 - t) of the element-local
    coordinate t in [0, 1] of the other direction: quadratic in every element (exact at p >= 2),
    continuous and periodic, faces curved, volume kept.
    kind = "sine": X = x + eps (h_x s(y), h_y s(z), h_z s(x)) with s = sin(2 pi (t - lo) / L) over the
    whole box: smooth and periodic but not polynomial per element."""
    lo, hi, ne = np.asarray(lo, float), np.asarray(hi, float), np.asarray(nelem)
    h = (hi - lo) / ne
    X = np.array(x, dtype=float, copy=True)

    def disp(d):
        t = (x[:, d] - lo[d]) / h[d]
        if kind == "bump":
            tl = t - np.floor(t)
            return 4.0 * tl * (1.0 - tl)
        return np.sin(TWO_PI * (x[:, d] - lo[d]) / (hi[d] - lo[d]))

    for d in range(3):
        X[:, d] += eps * h[d] * disp((d + 1) % 3)
    return X


def _proper_rotations():
    """The 24 rotations of the cube as (P, F): local axis k runs along structured axis P[k], reversed
    when F[k]; determinant sign(P) (-1)^(number of flips) = +1."""
    import itertools

    out = []
    for P in itertools.permutations(range(3)):
        sgn = 1
        for i in range(3):
            for j in range(i + 1, 3):
                if P[i] > P[j]:
                    sgn = -sgn
        for F in itertools.product((0, 1), repeat=3):
            if sgn * (-1) ** sum(F) == 1:
                out.append((P, F))
    return out


def unstructured_box(ne, p: int, bc=None, seed: int = 0, shuffle: bool = True) -> dict:
    """A structured ne[0] x ne[1] x ne[2] hexahedral grid relabelled as an unstructured mesh: elements in
    a seeded random order (or the grid's own order with shuffle=False, as a locality-ordered mesh would
    have), each with a seeded random rotation of its local axes. Returns
      node_map [E*NP]: (structured point index) of every new point (new element-major, local x fastest),
      nbr, nface, orient [E, 6]: the connectivity tables of oracle_set_connectivity / bgk_set_connectivity
    (bc[d][side] of the structured grid: 0 periodic, else a boundary face with the structured face's
    ghost). Pure index bookkeeping: coordinates and states are carried over by node_map."""
    rng = np.random.default_rng(seed)
    ne = tuple(int(v) for v in ne)
    E, n1 = ne[0] * ne[1] * ne[2], p + 1
    NP = n1 ** 3
    perm = rng.permutation(E) if shuffle else np.arange(E)  # structured element -> new element
    inv = np.argsort(perm)                 # new element -> structured element
    rots = _proper_rotations()
    rot = [rots[int(rng.integers(0, 24))] for _ in range(E)]  # per new element
    bc = bc if bc is not None else ((0, 0), (0, 0), (0, 0))

    def struct_ec(e):
        return [e % ne[0], (e // ne[0]) % ne[1], e // (ne[0] * ne[1])]

    def to_struct(loc, r):
        P, F = r
        T = [0, 0, 0]
        for k in range(3):
            T[P[k]] = (n1 - 1 - loc[k]) if F[k] else loc[k]
        return T

    def to_local(T, r):
        P, F = r
        return [(n1 - 1 - T[P[k]]) if F[k] else T[P[k]] for k in range(3)]

    node_map = np.zeros(E * NP, dtype=np.int64)
    for en in range(E):
        es = int(inv[en])
        for i in range(NP):
            loc = [i % n1, (i // n1) % n1, i // (n1 * n1)]
            T = to_struct(loc, rot[en])
            node_map[en * NP + i] = es * NP + T[0] + n1 * (T[1] + n1 * T[2])
    nbr = np.zeros((E, 6), dtype=np.int32)
    nface = np.zeros((E, 6), dtype=np.int32)
    orient = np.zeros((E, 6), dtype=np.int32)
    for en in range(E):
        es = int(inv[en])
        P, F = rot[en]
        for d in range(3):
            o1, o2 = [q for q in range(3) if q != d]
            for side in range(2):
                D, S = P[d], side ^ F[d]
                ec = struct_ec(es)
                ec[D] += 1 if S else -1
                if ec[D] < 0 or ec[D] >= ne[D]:
                    if bc[D][S] != 0:
                        nbr[en, 2 * d + side] = -1 - (2 * D + S)
                        continue
                    ec[D] %= ne[D]
                ns = ec[0] + ne[0] * (ec[1] + ne[1] * ec[2])
                nn = int(perm[ns])
                Pn, Fn = rot[nn]
                dn = list(Pn).index(D)
                sn = (1 - S) ^ Fn[dn]
                q1, q2 = [q for q in range(3) if q != dn]
                pairs = []
                for a in range(n1):
                    for b in range(n1):
                        loc = [0, 0, 0]
                        loc[d], loc[o1], loc[o2] = side * (n1 - 1), a, b
                        T = to_struct(loc, rot[en])
                        T[D] = n1 - 1 - T[D]
                        ln = to_local(T, rot[nn])
                        pairs.append(((a, b), (ln[q1], ln[q2])))
                code = None
                for c in range(8):
                    ok = True
                    for (a, b), (a2, b2) in pairs:
                        x, y = (b, a) if c & 1 else (a, b)
                        if c & 2:
                            x = n1 - 1 - x
                        if c & 4:
                            y = n1 - 1 - y
                        if (x, y) != (a2, b2):
                            ok = False
                            break
                    if ok:
                        code = c
                        break
                assert code is not None
                nbr[en, 2 * d + side] = nn
                nface[en, 2 * d + side] = 2 * dn + sn
                orient[en, 2 * d + side] = code
    return dict(node_map=node_map, nbr=nbr, nface=nface, orient=orient, perm=perm)


def noise(shape, seed: int = 0, amp: float = 0.05) -> np.ndarray:
    """Seeded multiplicative perturbation factors 1 + amp * U(-1, 1)."""
    rng = np.random.default_rng(seed)
    return 1.0 + amp * rng.uniform(-1.0, 1.0, size=shape)
