// k_stage.cu -- the fused SSP-RK3 stage kernel of the Boltzmann-BGK hot path (FP32-split form).
//
// One warp task = one element x a run of G velocity tiles (32 velocities of one sign octant each).
// Lane l owns velocity l of the tile and keeps all (p+1)^dim nodes of its element in registers.
// Per tile the warp
//   1. loads f_s of its element (coalesced 128-byte lines, one per node),
//   2. adds the FR advection residual direction by direction (Sec. 2.1, Eqs. 7-9): for the upwind
//      side of each line it reads the neighbour element's line (same tile) and interpolates the
//      neighbour's trace at the shared face; the interior trace is folded into the merged operator,
//   3. evaluates the conservative Maxwellian g = exp2(b0 + b.xi + b4 |xi|^2) of every node from the
//      per-point exponent that the Newton kernel wrote (Sec. 2.1, text after Eq. 13), applies the BGK
//      relaxation (Eq. 3) and the Shu-Osher combination of the stage (Sec. 2.2), stores f_{s+1},
//   4. transposes f_{s+1} through shared memory and sums w_k psi_k f over the 32 velocities of the
//      tile for every node (Eq. 2 with Eq. 12), accumulating one FP32 partial per node and moment.
// At the end of the task it writes the partial moments of its element; the Newton kernel sums the
// partials of all tasks exactly (double-float) before solving for the next stage's Maxwellian.
//
// The stage never reads what another task of the same launch writes: it reads f_s (source), f^n,
// the BGK exponent table and the ghost table, and writes only its own part of the destination and
// of the partial-moment table. The destination may alias f^n (the last stage updates f^n in place).
#include "bgk_common.cuh"

namespace bgk {

template <int N1, int DIM>
struct Geo {
    static constexpr int NP = (DIM == 1) ? N1 : N1 * N1 * N1;
    static constexpr int NL = (DIM == 1) ? 1 : N1 * N1;  // lines per direction
    // node index of position j along direction d on line ln (ln enumerates the other two indices)
    static __device__ __forceinline__ constexpr int node(int d, int ln, int j)
    {
        if (DIM == 1)
            return j;
        const int u = ln % N1, v = ln / N1;
        return d == 0 ? j + N1 * (u + N1 * v) : (d == 1 ? u + N1 * (j + N1 * v) : u + N1 * (v + N1 * j));
    }
};

// fused multiply-add on two packed FP32 lanes (sm_100+): d = a * b + c, element-wise
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float sum2(unsigned long long v)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}

// Upwind neighbour of element (ec) in direction d: returns its index, or -1 when the face is a
// non-periodic domain boundary (then the ghost table supplies the upwind value).
__device__ __forceinline__ int upwind_neighbour(const Mesh &m, const int ec[3], int d, bool left)
{
    int c[3] = {ec[0], ec[1], ec[2]};
    c[d] += left ? -1 : 1;
    if (c[d] < 0 || c[d] >= m.ne[d]) {
        if (m.bc[2 * d + (left ? 0 : 1)] != 0)
            return -1;
        c[d] = (c[d] + m.ne[d]) % m.ne[d];
    }
    return c[0] + m.ne[0] * (c[1] + m.ne[1] * c[2]);
}

// Raw values of the upwind neighbour along every line of direction D (one coalesced 128-byte load
// per node; all NL * N1 loads of a direction are issued together so their latency overlaps).
template <int N1, int DIM, int D>
__device__ __forceinline__ void load_lines(float (&v)[Geo<N1, DIM>::NL][N1], const float *__restrict__ nb)
{
    using Gm = Geo<N1, DIM>;
#pragma unroll
    for (int ln = 0; ln < Gm::NL; ln++)
#pragma unroll
        for (int j = 0; j < N1; j++)
            v[ln][j] = __ldg(nb + Gm::node(D, ln, j) * kWarp);
}

// Upwind trace of every line: the neighbour's interpolant at the shared face, in the difference form
// t = v_0 + sum_j l_j (v_j - v_0), exact for a constant state. A left neighbour is evaluated at its
// +1 end (lp), a right neighbour at its -1 end (lm).
template <int N1, int NL>
__device__ __forceinline__ void reduce_trace(float (&T)[NL], const float (&v)[NL][N1], const Ops &op, bool left)
{
#pragma unroll
    for (int ln = 0; ln < NL; ln++) {
        float t = 0.f;
#pragma unroll
        for (int j = 1; j < N1; j++)
            t = fmaf(left ? op.lp[j] : op.lm[j], v[ln][j] - v[ln][0], t);
        T[ln] = v[ln][0] + t;
    }
}

// Advection of all lines of one direction given the upwind traces T, inflow from the left
// (LEFT, xi_d > 0) or the right. acc += cd * (derivative along d), cd = -(2/h_d) xi_d b dt:
//   d_i = sum_{j != R} Dm[i][j] (f_j - f_R) + g[i] (T - f_R),  R = the inflow end of the line,
// Dm = D - g (x) l the derivative matrix with the interior trace folded in (exact zero for constants).
template <int N1, int DIM, int D, bool LEFT>
__device__ __forceinline__ void apply_dir(float (&acc)[Geo<N1, DIM>::NP], const float (&f)[Geo<N1, DIM>::NP],
                                          const float (&T)[Geo<N1, DIM>::NL], const Ops &op, float cd)
{
    using Gm = Geo<N1, DIM>;
    constexpr int P = N1 - 1;
    constexpr int R = LEFT ? 0 : P;
#pragma unroll
    for (int ln = 0; ln < Gm::NL; ln++) {
        const float fr = f[Gm::node(D, ln, R)];
        const float Tc = cd * (T[ln] - fr);
        float Gv[N1];
#pragma unroll
        for (int j = 0; j < N1; j++)
            Gv[j] = cd * (f[Gm::node(D, ln, j)] - fr);
#pragma unroll
        for (int i = 0; i < N1; i++) {
            float s = acc[Gm::node(D, ln, i)];
#pragma unroll
            for (int j = 0; j < N1; j++) {
                if (j == R)
                    continue;
                s = fmaf(LEFT ? op.DL[i][j] : op.DR[i][j], Gv[j], s);
            }
            acc[Gm::node(D, ln, i)] = fmaf(LEFT ? op.gl[i] : op.gr[i], Tc, s);
        }
    }
}

template <int N1, int DIM, int D>
__device__ __forceinline__ void apply(float (&acc)[Geo<N1, DIM>::NP], const float (&f)[Geo<N1, DIM>::NP],
                                      const float (&T)[Geo<N1, DIM>::NL], const StageArgs &A, float xid, bool left)
{
    const float cd = -A.mesh.inv_h2[D] * xid * (A.b * A.dt);
    if (left)
        apply_dir<N1, DIM, D, true>(acc, f, T, A.ops, cd);
    else
        apply_dir<N1, DIM, D, false>(acc, f, T, A.ops, cd);
}

// Issue the neighbour loads of direction D (or fill the ghost value on a non-periodic boundary).
template <int N1, int DIM, int D>
__device__ __forceinline__ bool fetch_dir(float (&v)[Geo<N1, DIM>::NL][N1], float &ghost, const StageArgs &A,
                                          const int ec[3], int vl, int slot, bool left)
{
    const int en = upwind_neighbour(A.mesh, ec, D, left);
    if (en >= 0) {
        load_lines<N1, DIM, D>(v, A.src + fidx(vl, en, 0, threadIdx.x & 31, A.mesh.nelem, Geo<N1, DIM>::NP));
        return true;
    }
    ghost = __ldg(A.ghost + (2 * D + (left ? 0 : 1)) * A.nslots + slot);
    return false;
}

template <int N1, int NL>
__device__ __forceinline__ void traces(float (&T)[NL], const float (&v)[NL][N1], bool have, float ghost,
                                       const Ops &op, bool left)
{
    if (have) {
        reduce_trace<N1, NL>(T, v, op, left);
    } else {
#pragma unroll
        for (int ln = 0; ln < NL; ln++)
            T[ln] = ghost;
    }
}

template <int NP>
struct StageSmem {
    static constexpr int NPL = (NP + 31) / 32;  // moment nodes per lane
    float wf[kWarpsPerCta][NP][36];              // [node][velocity] transposed stage output (x w psi later)
    float wpsi[kWarpsPerCta][5][32];
    float macc[kWarpsPerCta][5][NPL * 32];       // per-task moment accumulators
    float par[kWarpsPerCta][NP][kParamStride];   // BGK exponents of the element's points
};

// MODE 0: full stage. MODE 1: moments of src only (no advection, no store).
// CTAs per SM the register budget is sized for: the p = 3 hexahedron keeps 2 x 64 values per lane.
template <int NP>
struct MinCtas {
    static constexpr int value = NP > 32 ? 2 : 3;
};

template <int N1, int DIM, int MODE>
__global__ void __launch_bounds__(kWarp *kWarpsPerCta, MinCtas<Geo<N1, DIM>::NP>::value) k_stage(const StageArgs A)
{
    using Gm = Geo<N1, DIM>;
    constexpr int NP = Gm::NP;
    using Sm = StageSmem<NP>;
    constexpr int NPL = Sm::NPL;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int E = A.mesh.nelem;
    const int nEB = (E + kWarpsPerCta - 1) / kWarpsPerCta;
    const int gl = blockIdx.x / nEB;
    const int e = (blockIdx.x % nEB) * kWarpsPerCta + wid;
    if (e >= E)
        return;  // whole warp; the kernel uses warp-level synchronisation only
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    int ec[3];
    ec[0] = e % A.mesh.ne[0];
    ec[1] = (e / A.mesh.ne[0]) % A.mesh.ne[1];
    ec[2] = e / (A.mesh.ne[0] * A.mesh.ne[1]);

    if (MODE == 0) {
        const float4 *src4 = reinterpret_cast<const float4 *>(A.param + (int64_t)e * NP * kParamStride);
        float4 *dst4 = reinterpret_cast<float4 *>(&sm.par[wid][0][0]);
        for (int q = lane; q < NP * kParamStride / 4; q += kWarp)
            dst4[q] = __ldg(src4 + q);
    }
#pragma unroll
    for (int q = 0; q < NPL; q++)
#pragma unroll
        for (int c = 0; c < 5; c++)
            sm.macc[wid][c][q * 32 + lane] = 0.f;

    const float kb = A.b * (1.f - A.dt * A.inv_tau);
    // f: f_s of the current tile; acc: f^n of the current tile (or 0), prefetched one tile ahead
    float f[NP], acc[NP];
    {
        const int64_t b0 = fidx(vl0, e, 0, lane, E, NP);
#pragma unroll
        for (int i = 0; i < NP; i++)
            f[i] = __ldg(A.src + b0 + i * kWarp);
        if (MODE == 0) {
#pragma unroll
            for (int i = 0; i < NP; i++)
                acc[i] = A.fn ? __ldcs(A.fn + b0 + i * kWarp) : 0.f;
        }
    }
    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const float x0 = __ldg(A.xi + slot), x1 = __ldg(A.xi + A.nslots + slot), x2 = __ldg(A.xi + 2 * A.nslots + slot);
#pragma unroll
        for (int c = 0; c < 5; c++)
            sm.wpsi[wid][c][lane] = __ldg(A.wpsi + ((int64_t)vt * 5 + c) * kWarp + lane);
        const int64_t base = fidx(vl, e, 0, lane, E, NP);

        if (MODE == 0) {
            // acc = an f^n + b (1 - dt/tau) f_s, then the advection of every direction
#pragma unroll
            for (int i = 0; i < NP; i++)
                acc[i] = fmaf(A.an, acc[i], kb * f[i]);
            const bool l0 = x0 >= 0.f, l1 = x1 >= 0.f, l2 = x2 >= 0.f;
            float v[Gm::NL][N1], T[Gm::NL], gh = 0.f;
            bool have = fetch_dir<N1, DIM, 0>(v, gh, A, ec, vl, slot, l0);
            traces<N1, Gm::NL>(T, v, have, gh, A.ops, l0);
            if constexpr (DIM > 1) {
                apply<N1, DIM, 0>(acc, f, T, A, x0, l0);
                have = fetch_dir<N1, DIM, 1>(v, gh, A, ec, vl, slot, l1);
                traces<N1, Gm::NL>(T, v, have, gh, A.ops, l1);
                apply<N1, DIM, 1>(acc, f, T, A, x1, l1);
                have = fetch_dir<N1, DIM, 2>(v, gh, A, ec, vl, slot, l2);
                traces<N1, Gm::NL>(T, v, have, gh, A.ops, l2);
                apply<N1, DIM, 2>(acc, f, T, A, x2, l2);
            } else {
                apply<N1, DIM, 0>(acc, f, T, A, x0, l0);
            }
            // BGK source towards the conservative Maxwellian (cg g) and the store of f_{s+1}
            const float cg = A.b * A.dt * A.inv_tau * __ldg(A.gmask + slot);
            const float xs = x0 * x0 + x1 * x1 + x2 * x2;
            float *dst = A.dst + base;
#pragma unroll
            for (int i = 0; i < NP; i++) {
                const float4 pb = *reinterpret_cast<const float4 *>(&sm.par[wid][i][0]);
                const float b4 = sm.par[wid][i][4];
                const float ex = fmaf(b4, xs, fmaf(pb.w, x2, fmaf(pb.z, x1, fmaf(pb.y, x0, pb.x))));
                const float o = fmaf(cg, exp2f(ex), acc[i]);
                __stcs(dst + i * kWarp, o);
                sm.wf[wid][i][lane] = o;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NP; i++)
                sm.wf[wid][i][lane] = f[i];
        }
        __syncwarp();
        // prefetch the next tile (its latency overlaps the moment sums below)
        if (vl + 1 < vl1) {
            const int64_t b1 = fidx(vl + 1, e, 0, lane, E, NP);
#pragma unroll
            for (int i = 0; i < NP; i++)
                f[i] = __ldg(A.src + b1 + i * kWarp);
            if (MODE == 0) {
#pragma unroll
                for (int i = 0; i < NP; i++)
                    acc[i] = A.fn ? __ldcs(A.fn + b1 + i * kWarp) : 0.f;
            }
        }

        // moments of the 32 velocities of this tile, node = lane + 32 q, pairs over k
#pragma unroll
        for (int q = 0; q < NPL; q++) {
            const int nd = lane + 32 * q;
            if (nd < NP) {
                unsigned long long m[5];
#pragma unroll
                for (int c = 0; c < 5; c++)
                    m[c] = 0ull;
#pragma unroll
                for (int k = 0; k < 32; k += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(&sm.wf[wid][nd][k]);
                    const unsigned long long v01 = pack2(v.x, v.y), v23 = pack2(v.z, v.w);
#pragma unroll
                    for (int c = 0; c < 5; c++) {
                        const float4 w = *reinterpret_cast<const float4 *>(&sm.wpsi[wid][c][k]);
                        m[c] = ffma2(pack2(w.x, w.y), v01, m[c]);
                        m[c] = ffma2(pack2(w.z, w.w), v23, m[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < 5; c++)
                    sm.macc[wid][c][nd] += sum2(m[c]);
            }
        }
        __syncwarp();
    }

    // partial moments of this task: partial[group][c][point]
    const int grp = A.group0 + gl;
#pragma unroll
    for (int q = 0; q < NPL; q++) {
        const int nd = lane + 32 * q;
        if (nd < NP)
#pragma unroll
            for (int c = 0; c < 5; c++)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)e * NP + nd] = sm.macc[wid][c][nd];
    }
}

// ------------------------------------------------------------------------------------------------
// Hexahedra: one CTA per (element, run of G tiles), one warp per z-layer of the element's nodes.
// Lane l owns velocity l of the tile. A warp keeps its layer's N1^2 values (f_s, the accumulator and
// the x/y neighbour lines) in registers, so x and y derivatives are register-local; the z-lines cross
// the layers and are read from a shared copy of the element tile. The z-upwind traces are split
// over the warps (warp w interpolates the z-lines with iy = w) and shared the same way.
// ------------------------------------------------------------------------------------------------
template <int N1>
struct Stage3Smem {
    static constexpr int NP = N1 * N1 * N1;
    float tile[NP][kWarp];        // f_s of the element, [node][lane]
    float zc[NP][kWarp];          // z-derivative sums, [node][lane]
    float wf[N1][16][36];         // per warp: its layer's stage output, [node][velocity] (16 rows)
    float par[NP][kParamStride];  // BGK exponents of the element's points
    float wpsi[5][kWarp];         // w psi of the tile's velocities
};

// The 1-D line computation shared by the three directions: for the line values fl (inflow end R,
// upwind trace T) returns s_i = sum_{j != R} Dm[i][j] (f_j - f_R) + g_i (T - f_R) for all nodes i
// (Dm = D - g (x) l, the derivative with the interior trace folded in; d f_i/dt gains cd * s_i).
template <int N1, bool LEFT>
__device__ __forceinline__ void line_sums(float (&s)[N1], const float (&fl)[N1], float T, const Ops &op)
{
    constexpr int R = LEFT ? 0 : N1 - 1;
    const float fr = fl[R];
    const float tr = T - fr;
    float G[N1];
#pragma unroll
    for (int j = 0; j < N1; j++)
        G[j] = fl[j] - fr;
#pragma unroll
    for (int i = 0; i < N1; i++) {
        float v = (LEFT ? op.gl[i] : op.gr[i]) * tr;
#pragma unroll
        for (int j = 0; j < N1; j++)
            if (j != R)
                v = fmaf(LEFT ? op.DL[i][j] : op.DR[i][j], G[j], v);
        s[i] = v;
    }
}

// Upwind trace of one neighbour line v (difference form, exact for a constant state): a left
// neighbour is evaluated at its +1 end (lp), a right neighbour at its -1 end (lm).
template <int N1, bool LEFT>
__device__ __forceinline__ float trace_line(const float (&v)[N1], const Ops &op)
{
    float t = 0.f;
#pragma unroll
    for (int j = 1; j < N1; j++)
        t = fmaf(LEFT ? op.lp[j] : op.lm[j], v[j] - v[0], t);
    return v[0] + t;
}

template <int N1, int MODE>
__global__ void __launch_bounds__(kWarp *N1, (N1 >= 4 ? 4 : (N1 == 3 ? 6 : 8))) k_stage3(const StageArgs A)
{
    constexpr int NQ = N1 * N1;      // nodes per layer
    constexpr int NP = NQ * N1;
    constexpr int NT = kWarp * N1;   // threads
    using Sm = Stage3Smem<N1>;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;  // w: this warp's z-layer and y-slice
    const int E = A.mesh.nelem;
    const int gl = blockIdx.x / E;
    const int e = blockIdx.x % E;
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    int ec[3];
    ec[0] = e % A.mesh.ne[0];
    ec[1] = (e / A.mesh.ne[0]) % A.mesh.ne[1];
    ec[2] = e / (A.mesh.ne[0] * A.mesh.ne[1]);

    if (MODE == 0) {
        const float4 *src4 = reinterpret_cast<const float4 *>(A.param + (int64_t)e * NP * kParamStride);
        float4 *dst4 = reinterpret_cast<float4 *>(&sm.par[0][0]);
        for (int q = tid; q < NP * kParamStride / 4; q += NT)
            dst4[q] = __ldg(src4 + q);
    }
    // moment sums: lane = (node pair np = lane / 4: layer nodes np and np + 8) x (velocity eighth
    // kg = lane % 4: velocities 8 kg .. 8 kg + 7 of every tile); FP32 pairs over even/odd velocities,
    // accumulated over the whole task and combined across the 4 lanes of a pair at the end
    const int np = lane >> 2, kg = lane & 3;
    unsigned long long ms[2][5];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int c = 0; c < 5; c++)
            ms[h][c] = 0ull;
    const float kb = A.b * (1.f - A.dt * A.inv_tau);
    const float bdt = A.b * A.dt;

    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const float x0 = __ldg(A.xi + slot), x1 = __ldg(A.xi + A.nslots + slot), x2 = __ldg(A.xi + 2 * A.nslots + slot);
        const float *tileg = A.src + fidx(vl, e, 0, lane, E, NP);
        float f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++)
            f[q] = __ldg(tileg + (q + NQ * w) * kWarp);
        float o[NQ];
        if (MODE == 0) {
            const bool l0 = x0 >= 0.f, l1 = x1 >= 0.f, l2 = x2 >= 0.f;
            float acc[NQ];
            if (A.fn) {
                const float *fng = A.fn + fidx(vl, e, 0, lane, E, NP);
#pragma unroll
                for (int q = 0; q < NQ; q++)
                    acc[q] = __ldcs(fng + (q + NQ * w) * kWarp);
            } else {
#pragma unroll
                for (int q = 0; q < NQ; q++)
                    acc[q] = 0.f;
            }
            // upwind neighbour values: x-lines and y-lines of layer w, z-lines of slice iy = w
            float vx[N1][N1], vy[N1][N1], vz[N1][N1];
            const int enx = upwind_neighbour(A.mesh, ec, 0, l0);
            const int eny = upwind_neighbour(A.mesh, ec, 1, l1);
            const int enz = upwind_neighbour(A.mesh, ec, 2, l2);
            if (enx >= 0) {
                const float *nb = A.src + fidx(vl, enx, 0, lane, E, NP);
#pragma unroll
                for (int iy = 0; iy < N1; iy++)
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        vx[iy][j] = __ldg(nb + (j + N1 * iy + NQ * w) * kWarp);
            }
            if (eny >= 0) {
                const float *nb = A.src + fidx(vl, eny, 0, lane, E, NP);
#pragma unroll
                for (int ix = 0; ix < N1; ix++)
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        vy[ix][j] = __ldg(nb + (ix + N1 * j + NQ * w) * kWarp);
            }
            if (enz >= 0) {
                const float *nb = A.src + fidx(vl, enz, 0, lane, E, NP);
#pragma unroll
                for (int ix = 0; ix < N1; ix++)
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        vz[ix][j] = __ldg(nb + (ix + N1 * w + NQ * j) * kWarp);
            }
#pragma unroll
            for (int q = 0; q < NQ; q++)
                sm.tile[q + NQ * w][lane] = f[q];
            // acc = an f^n + b (1 - dt/tau) f_s, then x and y lines from registers
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = fmaf(A.an, acc[q], kb * f[q]);
            const float cx = -A.mesh.inv_h2[0] * x0 * bdt, cy = -A.mesh.inv_h2[1] * x1 * bdt,
                        cz = -A.mesh.inv_h2[2] * x2 * bdt;
            const float gx = enx >= 0 ? 0.f : __ldg(A.ghost + (l0 ? 0 : 1) * A.nslots + slot);
            const float gy = eny >= 0 ? 0.f : __ldg(A.ghost + (2 + (l1 ? 0 : 1)) * A.nslots + slot);
            const float gz = enz >= 0 ? 0.f : __ldg(A.ghost + (4 + (l2 ? 0 : 1)) * A.nslots + slot);
#pragma unroll
            for (int iy = 0; iy < N1; iy++) {
                float fl[N1], sv[N1];
#pragma unroll
                for (int j = 0; j < N1; j++)
                    fl[j] = f[j + N1 * iy];
                if (l0)
                    line_sums<N1, true>(sv, fl, enx >= 0 ? trace_line<N1, true>(vx[iy], A.ops) : gx, A.ops);
                else
                    line_sums<N1, false>(sv, fl, enx >= 0 ? trace_line<N1, false>(vx[iy], A.ops) : gx, A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    acc[j + N1 * iy] = fmaf(cx, sv[j], acc[j + N1 * iy]);
            }
#pragma unroll
            for (int ix = 0; ix < N1; ix++) {
                float fl[N1], sv[N1];
#pragma unroll
                for (int j = 0; j < N1; j++)
                    fl[j] = f[ix + N1 * j];
                if (l1)
                    line_sums<N1, true>(sv, fl, eny >= 0 ? trace_line<N1, true>(vy[ix], A.ops) : gy, A.ops);
                else
                    line_sums<N1, false>(sv, fl, eny >= 0 ? trace_line<N1, false>(vy[ix], A.ops) : gy, A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    acc[ix + N1 * j] = fmaf(cy, sv[j], acc[ix + N1 * j]);
            }
            __syncthreads();  // B1: the element tile is complete
            if (w == 0) {
#pragma unroll
                for (int c = 0; c < 5; c++)
                    sm.wpsi[c][lane] = __ldg(A.wpsi + ((int64_t)vt * 5 + c) * kWarp + lane);
            }
            // z-lines of slice iy = w (all layers), from the shared tile; results to zc
#pragma unroll
            for (int ix = 0; ix < N1; ix++) {
                const int q = ix + N1 * w;
                float fl[N1], sv[N1];
#pragma unroll
                for (int j = 0; j < N1; j++)
                    fl[j] = sm.tile[q + NQ * j][lane];
                if (l2)
                    line_sums<N1, true>(sv, fl, enz >= 0 ? trace_line<N1, true>(vz[ix], A.ops) : gz, A.ops);
                else
                    line_sums<N1, false>(sv, fl, enz >= 0 ? trace_line<N1, false>(vz[ix], A.ops) : gz, A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    sm.zc[q + NQ * j][lane] = sv[j];
            }
            __syncthreads();  // B2: z-sums complete
            // BGK source towards the conservative Maxwellian, Shu-Osher combination, store
            const float cg = bdt * A.inv_tau * __ldg(A.gmask + slot);
            const float xs = x0 * x0 + x1 * x1 + x2 * x2;
            float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                const int i = q + NQ * w;
                const float4 pb = *reinterpret_cast<const float4 *>(&sm.par[i][0]);
                const float b4 = sm.par[i][4];
                const float ex = fmaf(b4, xs, fmaf(pb.w, x2, fmaf(pb.z, x1, fmaf(pb.y, x0, pb.x))));
                const float a = fmaf(cz, sm.zc[i][lane], acc[q]);
                o[q] = fmaf(cg, exp2f(ex), a);
                __stcs(dst + i * kWarp, o[q]);
            }
        } else {
            __syncthreads();  // B1 (same barrier sequence in both modes)
            if (w == 0) {
#pragma unroll
                for (int c = 0; c < 5; c++)
                    sm.wpsi[c][lane] = __ldg(A.wpsi + ((int64_t)vt * 5 + c) * kWarp + lane);
            }
            __syncthreads();  // B2
#pragma unroll
            for (int q = 0; q < NQ; q++)
                o[q] = f[q];
        }
        // moments of this layer's nodes (Eq. 2 with Eq. 12) of the stored values
#pragma unroll
        for (int q = 0; q < NQ; q++)
            sm.wf[w][q][lane] = o[q];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k += 4) {
            const int kk = 8 * kg + k;
            unsigned long long wv[5][2];
#pragma unroll
            for (int c = 0; c < 5; c++) {
                const float4 w4 = *reinterpret_cast<const float4 *>(&sm.wpsi[c][kk]);
                wv[c][0] = pack2(w4.x, w4.y);
                wv[c][1] = pack2(w4.z, w4.w);
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const float4 v = *reinterpret_cast<const float4 *>(&sm.wf[w][np + 8 * h][kk]);
                const unsigned long long v01 = pack2(v.x, v.y), v23 = pack2(v.z, v.w);
#pragma unroll
                for (int c = 0; c < 5; c++) {
                    ms[h][c] = ffma2(wv[c][0], v01, ms[h][c]);
                    ms[h][c] = ffma2(wv[c][1], v23, ms[h][c]);
                }
            }
        }
        __syncwarp();
    }
    // partial moments of this task: combine the 4 velocity eighths of every node pair
    const int grp = A.group0 + gl;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int q = np + 8 * h;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            float x = sum2(ms[h][c]);
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (kg == 0 && q < NQ)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)e * NP + q + NQ * w] = x;
        }
    }
}

template <int N1, int DIM>
static cudaError_t prepare_nd()
{
    if constexpr (DIM == 3) {
        const int smem3 = (int)sizeof(Stage3Smem<N1>);
        cudaError_t err = cudaFuncSetAttribute(k_stage3<N1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_stage3<N1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
        return err;
    } else {
        const int smem = (int)sizeof(StageSmem<Geo<N1, DIM>::NP>);
        cudaError_t err = cudaFuncSetAttribute(k_stage<N1, DIM, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_stage<N1, DIM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        return err;
    }
}

template <int N1, int DIM>
static cudaError_t launch_nd(const StageArgs &A, int mode, cudaStream_t s)
{
    if constexpr (DIM == 3) {
        const int ngroups3 = (A.nvt + A.G - 1) / A.G;
        const int smem3 = (int)sizeof(Stage3Smem<N1>);
        dim3 grid3(A.mesh.nelem * ngroups3), block3(kWarp * N1);
        if (mode == 0)
            k_stage3<N1, 0><<<grid3, block3, smem3, s>>>(A);
        else
            k_stage3<N1, 1><<<grid3, block3, smem3, s>>>(A);
        return cudaGetLastError();
    } else {
        const int nEB = (A.mesh.nelem + kWarpsPerCta - 1) / kWarpsPerCta;
        const int ngroups = (A.nvt + A.G - 1) / A.G;
        dim3 grid(nEB * ngroups), block(kWarp * kWarpsPerCta);
        const int smem = (int)sizeof(StageSmem<Geo<N1, DIM>::NP>);
        if (mode == 0)
            k_stage<N1, DIM, 0><<<grid, block, smem, s>>>(A);
        else
            k_stage<N1, DIM, 1><<<grid, block, smem, s>>>(A);
        return cudaGetLastError();
    }
}

#define BGK_DISPATCH(FN, ...)                                                        \
    if (dim == 3) {                                                                  \
        switch (p) {                                                                 \
        case 1: return FN<2, 3>(__VA_ARGS__);                                        \
        case 2: return FN<3, 3>(__VA_ARGS__);                                        \
        case 3: return FN<4, 3>(__VA_ARGS__);                                        \
        }                                                                            \
    } else if (dim == 1) {                                                           \
        switch (p) {                                                                 \
        case 1: return FN<2, 1>(__VA_ARGS__);                                        \
        case 2: return FN<3, 1>(__VA_ARGS__);                                        \
        case 3: return FN<4, 1>(__VA_ARGS__);                                        \
        case 4: return FN<5, 1>(__VA_ARGS__);                                        \
        case 5: return FN<6, 1>(__VA_ARGS__);                                        \
        }                                                                            \
    }                                                                                \
    return cudaErrorInvalidValue;

// Set the shared-memory attributes of the stage kernels of one (dim, p); call before any capture.
cudaError_t prepare_stage(int dim, int p) { BGK_DISPATCH(prepare_nd) }

// Launch one stage (mode 0) or a moments-only pass (mode 1) over one velocity chunk.
cudaError_t launch_stage(const StageArgs &A, int p, int mode, cudaStream_t s)
{
    const int dim = A.mesh.dim;
    BGK_DISPATCH(launch_nd, A, mode, s)
}

}  // namespace bgk
