// k_stage3c.cuh -- the fused SSP-RK3 stage kernel of curvilinear hexahedra on the structured element
// grid (FP32-split form), every operand staged in shared memory by bulk asynchronous copies as in
// k_stage3s.cuh; instantiated per degree in k_stage3_p*.cu.
#pragma once
#include <type_traits>

#include "k_stage3s.cuh"

#ifndef BGK_STAGE3C_MINCTAS_P3
#define BGK_STAGE3C_MINCTAS_P3 4
#endif

namespace bgk {

// ------------------------------------------------------------------------------------------------
// Curvilinear hexahedra, structured element grid (Sec. 2.1, Eqs. 6-9 on the mapped element): the
// reference-space flux u f with u = Ja^d . xi at every node, and the upwind common flux of every face
// point from the sign of the shared face normal's N . xi per lane. The layout and the copy schedule are
// k_stage3s's: one CTA per (element, run of G velocity tiles), one warp per z-layer, lane = velocity of
// the tile; the warp's f_s layer double-buffered, three rotating slots per warp for f^n and the upwind
// neighbours' layers, the velocity tables double-buffered by warp 0. The staged neighbour of direction
// d is the one on the side the tile's sign octant makes upwind (the low side where xi_d >= 0): a face
// normal of a curved element is close to its axis, so that side's face is the inflow face of nearly
// every lane. A lane whose flow enters through the other face (a normal tilted against a small xi_d)
// reads that neighbour's trace from global memory; where no lane of the warp does, nothing is read.
// ------------------------------------------------------------------------------------------------
template <int N1, int GEN>
struct Stage3cSmem {
    static constexpr int NP = N1 * N1 * N1, NQ = N1 * N1;
    float fs[2][NP][kWarp];
    float sl[N1][3][NQ][kWarp];
    float tab[2][kTabRows][kWarp];
    float par[N1][(NQ + 1) / 2][kParamStride][2];  // BGK exponents by layer and node pair (see k_stage3s)
    float fpar[GEN ? NP : 1][GEN ? kParamStride : 4];
    float lim[GEN ? 2 : 1][GEN ? N1 : 1][GEN ? kWarp : 4];
    float4 met[NP][3];      // metric rows Ja^d; .w of row 0 = -b dt / J (the line sums' factor), of row 1 = W J
    // where N1 is even, the rows of direction d again by the node pairs of two adjacent lines (see
    // pair_row): (x_a, x_b, y_a, y_b), (z_a, z_b, s_a, s_b) with s = -b dt / J
    float4 metp[N1 % 2 == 0 ? 3 : 1][N1 % 2 == 0 ? NP / 2 : 1][2];
    float4 fnm[3][2][NQ];   // shared face normals (direction, low/high side, face point)
    // where N1 is even, again by face-point pairs (fp, fp + 1) of the paired lines: (x_a, x_b, y_a, y_b),
    // (z_a, z_b, 0, 0)
    float4 fnmp[N1 % 2 == 0 ? 3 : 1][2][N1 % 2 == 0 ? NQ / 2 : 1][2];
    float iwj;              // 1 / sum_i W_i J_i
    unsigned long long bar[N1][5];
    unsigned long long tbar[2];
};

// The reference-space line of direction d at one lane: node values fl, fluxes u fl, the exterior
// traces tL / tR used where the face normal's flow enters (uL > 0 at the low face, uR < 0 at the high
// face), the element's own trace of f elsewhere (as curv_line in k_stage3.cuh).
template <int N1>
__device__ __forceinline__ void curv_line_c(float (&sv)[N1], const float (&fl)[N1], const float (&u)[N1], float uL,
                                            float uR, float tL, float tR, const Ops &op)
{
    float F[N1], oL = 0.f, oR = 0.f;
#pragma unroll
    for (int j = 0; j < N1; j++) {
        F[j] = u[j] * fl[j];
        oL = fmaf(op.lm[j], fl[j], oL);
        oR = fmaf(op.lp[j], fl[j], oR);
    }
    const float FIL = uL * (uL > 0.f ? tL : oL);
    const float FIR = uR * (uR < 0.f ? tR : oR);
#pragma unroll
    for (int i = 0; i < N1; i++) {
        float a = fmaf(op.gl[i], FIL, op.gr[i] * FIR);
#pragma unroll
        for (int j = 0; j < N1; j++)
            a = fmaf(op.DM[i][j], F[j], a);
        sv[i] = a;
    }
}

// Node pairs of the paired lines of direction d (N1 even): lines 2 lp and 2 lp + 1 of a warp, node j:
// the pair's first node a (its partner a + N1 for d = 0, a + 1 otherwise) and its slot in metp[d].
template <int N1>
__host__ __device__ constexpr int pair_row(int d, int a)
{
    return d == 0 ? a % N1 + N1 * ((a / N1) % N1 / 2) + (N1 * N1 / 2) * (a / (N1 * N1))
                  : (a % N1) / 2 + (N1 / 2) * (a / N1);
}

// GEN = 0: every face periodic, no body force, no limiter, constant tau and one velocity spacing on all
// axes (the lean form of k_stage3s); GEN = 1: Dirichlet and diffuse-wall ghosts, the force source, the
// limiter, variable tau and per-axis spacings.
template <int N1, int GEN>
__global__ void __launch_bounds__(kWarp *N1, (N1 >= 4 ? BGK_STAGE3C_MINCTAS_P3 : (N1 == 3 ? 6 : 8))) k_stage3c(const StageArgs A)
{
    constexpr int NQ = N1 * N1;
    constexpr int NP = NQ * N1;
    constexpr int NT = kWarp * N1;
    constexpr uint32_t kRow = kWarp * sizeof(float);
    using Sm = Stage3cSmem<N1, GEN>;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int E = A.mesh.nelem;
    const int gl = blockIdx.x / E;
    const int e = blockIdx.x % E;
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    int ec[3];
    ec[0] = e % A.mesh.ne[0];
    ec[1] = (e / A.mesh.ne[0]) % A.mesh.ne[1];
    ec[2] = e / (A.mesh.ne[0] * A.mesh.ne[1]);
    const float bdt = A.b * A.dt;

    // the element's BGK exponents, body-force polynomials, metric rows and face normals
    {
        constexpr int NH = (NQ + 1) / 2;
        const float *src = A.param + (int64_t)e * NP * kParamStride;
        for (int q = tid; q < N1 * NH * 2 * kParamStride; q += NT) {
            const int c = q % kParamStride, sl = (q / kParamStride) & 1, h = (q / (2 * kParamStride)) % NH;
            const int lw = q / (2 * kParamStride * NH);
            const int node = lw * NQ + min(2 * h + sl, NQ - 1);
            sm.par[lw][h][c][sl] = __ldg(src + node * kParamStride + c);
        }
        if (GEN && A.fpar) {
            const float4 *f4 = reinterpret_cast<const float4 *>(A.fpar + (int64_t)e * NP * kParamStride);
            float4 *d4 = reinterpret_cast<float4 *>(&sm.fpar[0][0]);
            for (int q = tid; q < NP * kParamStride / 4; q += NT)
                d4[q] = __ldg(f4 + q);
        }
        for (int q = tid; q < NP * 3; q += NT) {
            float4 m = __ldg(A.met + (int64_t)e * NP * 3 + q);
            if (q % 3 == 0)
                m.w = -bdt * m.w;  // rounded as the product the unstaged kernel forms at every use
            (&sm.met[0][0])[q] = m;
        }
        if constexpr (N1 % 2 == 0) {
            for (int q = tid; q < 3 * NP; q += NT) {  // q = d NP + node a; the pair's first nodes only
                const int d = q / NP, a = q % NP;
                const bool first = d == 0 ? ((a / N1) % N1) % 2 == 0 : (a % N1) % 2 == 0;
                if (!first)
                    continue;
                const int bn = a + (d == 0 ? N1 : 1);
                const float4 ma = __ldg(A.met + ((int64_t)e * NP + a) * 3 + d);
                const float4 mb = __ldg(A.met + ((int64_t)e * NP + bn) * 3 + d);
                const float sa = -bdt * __ldg(A.met + ((int64_t)e * NP + a) * 3).w;
                const float sb = -bdt * __ldg(A.met + ((int64_t)e * NP + bn) * 3).w;
                sm.metp[d][pair_row<N1>(d, a)][0] = make_float4(ma.x, mb.x, ma.y, mb.y);
                sm.metp[d][pair_row<N1>(d, a)][1] = make_float4(ma.z, mb.z, sa, sb);
            }
        }
        for (int q = tid; q < 6 * NQ; q += NT)
            (&sm.fnm[0][0][0])[q] = __ldg(A.fnm + (int64_t)e * 6 * NQ + q);
        if constexpr (N1 % 2 == 0) {
            for (int q = tid; q < 3 * NQ; q += NT) {  // q = (d, side) NQ / 2 + pair
                const int ds = q / (NQ / 2), pr = q % (NQ / 2);
                const float4 na = __ldg(A.fnm + (int64_t)e * 6 * NQ + ds * NQ + 2 * pr);
                const float4 nb = __ldg(A.fnm + (int64_t)e * 6 * NQ + ds * NQ + 2 * pr + 1);
                sm.fnmp[ds / 2][ds % 2][pr][0] = make_float4(na.x, nb.x, na.y, nb.y);
                sm.fnmp[ds / 2][ds % 2][pr][1] = make_float4(na.z, nb.z, 0.f, 0.f);
            }
        }
        if (tid == 0)
            sm.iwj = __ldg(A.iwj + e);
    }
    const uint32_t bar0 = smem_u32(&sm.bar[w][0]), tbar0 = smem_u32(&sm.tbar[0]);
    auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    auto tbar = [&](int b) { return tbar0 + 8u * (uint32_t)b; };
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 5; i++)
            mbar_init(bar(i), 1);
        if (w == 0) {
            mbar_init(tbar(0), 1);
            mbar_init(tbar(1), 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const bool has_fn = A.fn != nullptr;
    // the staged (octant-upwind) neighbour of every direction of tile vl, -1 on a Dirichlet or wall face
    auto nbrs_oct = [&](int oct, int (&en)[3]) {
#pragma unroll
        for (int d = 0; d < 3; d++)
            en[d] = upwind_neighbour(A.mesh, ec, d, ((oct >> d) & 1) != 0);
    };
    auto nbrs = [&](int vl, int (&en)[3]) {
        const int oct = (int)__ldg(A.toct + A.vt0 + vl);
#pragma unroll
        for (int d = 0; d < 3; d++)
            en[d] = upwind_neighbour(A.mesh, ec, d, ((oct >> d) & 1) != 0);
    };
    // role lanes as in k_stage3s: lane 0 the f_s layer, RZ .. RZ + N1 - 1 the z-neighbour's row groups,
    // RFN the f^n layer, RX / RY the x- / y-neighbour's layer w, RT of warp 0 the velocity table
    constexpr int RZ = 1, RFN = N1 + 1, RX = N1 + 2, RY = N1 + 3, RT = N1 + 4;
    const int64_t tstride = (int64_t)E * NP * kWarp;
    auto role_src = [&](const int (&en)[3]) -> const float * {
        if (lane == 0)
            return A.src + fidx(0, e, NQ * w, 0, E, NP);
        if (lane >= RZ && lane < RZ + N1)
            return en[2] >= 0 ? A.src + fidx(0, en[2], N1 * w + NQ * (lane - RZ), 0, E, NP) : nullptr;
        if (lane == RFN)
            return A.fn ? A.fn + fidx(0, e, NQ * w, 0, E, NP) : nullptr;
        if (lane == RX)
            return en[0] >= 0 ? A.src + fidx(0, en[0], NQ * w, 0, E, NP) : nullptr;
        if (lane == RY)
            return en[1] >= 0 ? A.src + fidx(0, en[1], NQ * w, 0, E, NP) : nullptr;
        return nullptr;
    };
    const uint32_t fs0 = smem_u32(&sm.fs[0][NQ * w][0]), sl0 = smem_u32(&sm.sl[w][0][0][0]);
    constexpr uint32_t kFsBuf = NP * kRow, kSlot = NQ * kRow;
    auto issue_layer = [&](const float *csrc, int vl, int k) {
        const uint32_t bb = bar(2 + k);
        mbar_arrive_expect_tx(bb, csrc ? kSlot : 0);
        if (csrc)
            bulk_g2s(sl0 + k * kSlot, csrc + vl * tstride, kSlot, bb);
    };

    int en[3];
    nbrs(vl0, en);
    const float *csrc = role_src(en);
    // the neighbours and the role lanes' sources are recomputed only where the octant changes from one
    // tile to the next (the velocities are ordered by octant, so within a chunk almost never)
    int octc = (int)__ldg(A.toct + A.vt0 + vl0);
    const float *fsrc = A.src + fidx(0, e, NQ * w, 0, E, NP);  // lane 0's source (the same every tile)
    if (lane == 0) {
        mbar_arrive_expect_tx(bar(0), kSlot);
        bulk_g2s(fs0, fsrc + vl0 * tstride, kSlot, bar(0));
        if (w == 0) {
            mbar_arrive_expect_tx(tbar(0), kTabRows * kRow);
            bulk_g2s(smem_u32(&sm.tab[0][0][0]), A.vtab + (int64_t)(A.vt0 + vl0) * kTabRows * kWarp,
                     kTabRows * kRow, tbar(0));
        }
    }
    if (lane == RFN && has_fn)
        issue_layer(csrc, vl0, 0);
    if (lane == RX)
        issue_layer(csrc, vl0, 1);
    if (lane == RY)
        issue_layer(csrc, vl0, 2);
    uint32_t ph = 0;
    auto wait = [&](int i) {
        mbar_wait(bar(i), (ph >> i) & 1, A.err);
        ph ^= 1u << i;
    };

    const int np = lane >> 2, kg = lane & 3;
    constexpr int NHR = NQ > 8 ? 2 : 1;
    float msum[NHR][5];
#pragma unroll
    for (int h = 0; h < NHR; h++)
#pragma unroll
        for (int c = 0; c < 5; c++)
            msum[h][c] = 0.f;
    const float kb = A.kb;

    int ka = 0;
    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const int b = (vl - vl0) & 1;
        const int kx = ka == 2 ? 0 : ka + 1, ky = ka == 0 ? 2 : ka - 1;
        int enn[3] = {en[0], en[1], en[2]};
        const bool more = vl + 1 < vl1;
        const int octn = more ? (int)__ldg(A.toct + vt + 1) : octc;
        const bool turn = octn != octc;  // the next tile lies in another octant
        if (turn)
            nbrs_oct(octn, enn);
        __syncwarp();
        if (lane == 0 && more) {
            fence_proxy_async();
            mbar_arrive_expect_tx(bar(b ^ 1), kSlot);
            bulk_g2s(fs0 + (b ^ 1) * kFsBuf, fsrc + (vl + 1) * tstride, kSlot, bar(b ^ 1));
        }
        const int oct = octc;
        const bool l0 = (oct & 1) != 0, l1 = (oct & 2) != 0, l2 = (oct & 4) != 0;
        const int enx = en[0], eny = en[1], enz = en[2];

        wait(b);
        mbar_wait(tbar(b), (ph >> (5 + b)) & 1, A.err);
        ph ^= 1u << (5 + b);
        const float m0 = sm.tab[b][0][lane], m1 = sm.tab[b][1][lane], m2 = sm.tab[b][2][lane];
        const float x0 = fmaf(A.vs[0], m0, A.vc[0]), x1 = fmaf(A.vs[1], m1, A.vc[1]), x2 = fmaf(A.vs[2], m2, A.vc[2]);
        float acc[NQ];
        if (has_fn) {
            wait(2 + ka);
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = sm.sl[w][ka][q][lane];
        } else {
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = 0.f;
        }
        // slot ka is consumed: the z-neighbour's slice lands there
        __syncwarp();
        if (lane >= RZ && lane < RZ + N1) {
            const float *zs = csrc;
            const uint32_t bb = bar(2 + ka);
            fence_proxy_async();
            if (lane == RZ)
                mbar_arrive_expect_tx(bb, zs ? kSlot : 0);
            if (zs)
                bulk_g2s(sl0 + ka * kSlot + (lane - RZ) * N1 * kRow, zs + vl * tstride, N1 * kRow, bb);
        }
        // (launch-uniform feature tests sit outside the unrolled node loops, which stay one basic block)
        if (GEN && A.vtau) {
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = fmaf(A.an, acc[q],
                              __fsub_rn(A.b, __fmul_rn(bdt, sm.par[w][q / 2][6][q % 2])) * sm.fs[b][q + NQ * w][lane]);
        } else {
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = fmaf(A.an, acc[q], kb * sm.fs[b][q + NQ * w][lane]);
        }
        // The lines of direction d through this warp's nodes: x- and y-lines of layer w (their sums
        // go to acc), z-lines of slice w (their sums overwrite the rows they read, after B1). Line ln
        // has face point fp = ln + N1 w on both faces. lo: the tile's octant stages the low-side
        // neighbour (slot ks); es: that neighbour, < 0 on a boundary face (its ghost value instead).
        // Lanes whose flow enters through the other face take that face's exterior trace, read for all
        // lines of the direction at once and only where some lane of the warp needs it.
        auto lines = [&](auto dc, int ks, bool lo, int es) {
            constexpr int d = decltype(dc)::value;
            auto node = [&](int ln, int j) {  // element node j of line ln
                return d == 0 ? j + N1 * ln + NQ * w : (d == 1 ? ln + N1 * j + NQ * w : ln + N1 * w + NQ * j);
            };
            auto srow = [&](int ln, int j) { return d == 0 ? j + N1 * ln : ln + N1 * j; };  // row in slot ks
            float cS[N1], cF[N1];  // trace weights of the staged and of the other side's neighbour
#pragma unroll
            for (int j = 0; j < N1; j++) {
                cS[j] = lo ? A.ops.lp[j] : A.ops.lm[j];
                cF[j] = lo ? A.ops.lm[j] : A.ops.lp[j];
            }
            auto trace = [&](const float(&v)[N1], const float(&c)[N1]) {  // trace_line with weights c
                float t = 0.f;
#pragma unroll
                for (int j = 1; j < N1; j++)
                    t = fmaf(c[j], v[j] - v[0], t);
                return v[0] + t;
            };
            float uL[N1], uR[N1], tF[N1];
            bool far = false;
            if constexpr (N1 % 2 == 0) {  // two face points at a time (the same operations per half)
                const unsigned long long X0 = pack2(x0, x0), X1 = pack2(x1, x1), X2 = pack2(x2, x2);
#pragma unroll
                for (int ln = 0; ln < N1; ln += 2) {
                    const int pr = (ln + N1 * w) / 2;
                    float u2[2][2];
#pragma unroll
                    for (int sd = 0; sd < 2; sd++) {
                        const float4 n0 = sm.fnmp[d][sd][pr][0], n1 = sm.fnmp[d][sd][pr][1];
                        unpack2(ffma2(pack2(n1.x, n1.y), X2, ffma2(pack2(n0.z, n0.w), X1, fmul2(pack2(n0.x, n0.y), X0))),
                                u2[sd][0], u2[sd][1]);
                    }
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        uL[ln + h] = u2[0][h];
                        uR[ln + h] = u2[1][h];
                        tF[ln + h] = 0.f;
                        far = far || (lo ? uR[ln + h] < 0.f : uL[ln + h] > 0.f);
                    }
                }
            } else {
#pragma unroll
                for (int ln = 0; ln < N1; ln++) {
                    const int fp = ln + N1 * w;
                    const float4 nL = sm.fnm[d][0][fp], nR = sm.fnm[d][1][fp];
                    uL[ln] = fmaf(nL.z, x2, fmaf(nL.y, x1, nL.x * x0));
                    uR[ln] = fmaf(nR.z, x2, fmaf(nR.y, x1, nR.x * x0));
                    tF[ln] = 0.f;
                    far = far || (lo ? uR[ln] < 0.f : uL[ln] > 0.f);
                }
            }
            if (__any_sync(0xffffffffu, far)) {
                const int g = 2 * d + (lo ? 1 : 0);
                const int eo = upwind_neighbour(A.mesh, ec, d, !lo);
                if (!GEN || eo >= 0) {
                    const float *nb = A.src + fidx(vl, eo, 0, lane, E, NP);
                    float v[N1][N1];
#pragma unroll
                    for (int ln = 0; ln < N1; ln++) {
                        const bool need = lo ? uR[ln] < 0.f : uL[ln] > 0.f;
#pragma unroll
                        for (int j = 0; j < N1; j++)
                            v[ln][j] = need ? __ldg(nb + node(ln, j) * kWarp) : 0.f;
                    }
#pragma unroll
                    for (int ln = 0; ln < N1; ln++)
                        tF[ln] = trace(v[ln], cF);
                } else {
                    // (the wall test is outside the loops: no load is formed from a pointer that may be null)
                    const float gv = __ldg(A.ghost + (int64_t)g * A.nslots + slot);
                    if (A.mesh.bc[g] == 2) {
                        const float *rw = A.rhow + ((int64_t)g * A.nfmax + face_elem(A.mesh, ec, d)) * NQ + N1 * w;
#pragma unroll
                        for (int ln = 0; ln < N1; ln++)
                            tF[ln] = gv * __ldg(rw + ln);
                    } else {
#pragma unroll
                        for (int ln = 0; ln < N1; ln++)
                            tF[ln] = gv;
                    }
                }
            }
            float gS[N1];  // the staged side's ghost value of every line on a boundary face
#pragma unroll
            for (int ln = 0; ln < N1; ln++)
                gS[ln] = 0.f;
            if (GEN && es < 0) {
                const int g = 2 * d + (lo ? 0 : 1);
                const float gv = __ldg(A.ghost + (int64_t)g * A.nslots + slot);
                if (A.mesh.bc[g] == 2) {
                    const float *rw = A.rhow + ((int64_t)g * A.nfmax + face_elem(A.mesh, ec, d)) * NQ + N1 * w;
#pragma unroll
                    for (int ln = 0; ln < N1; ln++)
                        gS[ln] = gv * __ldg(rw + ln);
                } else {
#pragma unroll
                    for (int ln = 0; ln < N1; ln++)
                        gS[ln] = gv;
                }
            }
            if constexpr (N1 % 2 == 0) {
                // two adjacent lines at a time on packed FP32 pairs: the same operations, in the same
                // order, as curv_line_c on each line (bit-identical results)
                const unsigned long long X0 = pack2(x0, x0), X1 = pack2(x1, x1), X2 = pack2(x2, x2);
#pragma unroll
                for (int ln = 0; ln < N1; ln += 2) {
                    unsigned long long fl[N1], F[N1], v[N1], sp[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        fl[j] = pack2(sm.fs[b][node(ln, j)][lane], sm.fs[b][node(ln + 1, j)][lane]);
                        v[j] = pack2(sm.sl[w][ks][srow(ln, j)][lane], sm.sl[w][ks][srow(ln + 1, j)][lane]);
                        const float4 *mp = &sm.metp[d][pair_row<N1>(d, node(ln, j))][0];
                        const float4 p0 = mp[0], p1 = mp[1];
                        const unsigned long long u =
                            ffma2(pack2(p1.x, p1.y), X2, ffma2(pack2(p0.z, p0.w), X1, fmul2(pack2(p0.x, p0.y), X0)));
                        F[j] = fmul2(u, fl[j]);
                        sp[j] = pack2(p1.z, p1.w);
                    }
                    // the staged side's trace of both lines, and their own traces
                    unsigned long long t = 0ull, oL = 0ull, oR = 0ull;
#pragma unroll
                    for (int j = 1; j < N1; j++)
                        t = ffma2(dup2(cS[j]), fsub2(v[j], v[0]), t);
                    t = fadd2(v[0], t);
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        oL = ffma2(dup2(A.ops.lm[j]), fl[j], oL);
                        oR = ffma2(dup2(A.ops.lp[j]), fl[j], oR);
                    }
                    float tS2[2], oL2[2], oR2[2], FI[2][2];
                    unpack2(t, tS2[0], tS2[1]);
                    unpack2(oL, oL2[0], oL2[1]);
                    unpack2(oR, oR2[0], oR2[1]);
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const float tS = !GEN || es >= 0 ? tS2[h] : gS[ln + h];
                        const float tL = lo ? tS : tF[ln + h], tR = lo ? tF[ln + h] : tS;
                        FI[0][h] = uL[ln + h] * (uL[ln + h] > 0.f ? tL : oL2[h]);
                        FI[1][h] = uR[ln + h] * (uR[ln + h] < 0.f ? tR : oR2[h]);
                    }
                    const unsigned long long FIL = pack2(FI[0][0], FI[0][1]), FIR = pack2(FI[1][0], FI[1][1]);
#pragma unroll
                    for (int i = 0; i < N1; i++) {
                        unsigned long long a = ffma2(dup2(A.ops.gl[i]), FIL, fmul2(dup2(A.ops.gr[i]), FIR));
#pragma unroll
                        for (int j = 0; j < N1; j++)
                            a = ffma2(dup2(A.ops.DM[i][j]), F[j], a);
                        float sa, sb;
                        unpack2(a, sa, sb);
                        if (d < 2) {
                            float ca, cb;
                            unpack2(sp[i], ca, cb);
                            acc[node(ln, i) - NQ * w] = fmaf(ca, sa, acc[node(ln, i) - NQ * w]);
                            acc[node(ln + 1, i) - NQ * w] = fmaf(cb, sb, acc[node(ln + 1, i) - NQ * w]);
                        } else {
                            sm.fs[b][node(ln, i)][lane] = sa;
                            sm.fs[b][node(ln + 1, i)][lane] = sb;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int ln = 0; ln < N1; ln++) {
                    float fl[N1], u[N1], sv[N1], v[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        fl[j] = sm.fs[b][node(ln, j)][lane];
                        v[j] = sm.sl[w][ks][srow(ln, j)][lane];
                        const float4 m = sm.met[node(ln, j)][d];
                        u[j] = fmaf(m.z, x2, fmaf(m.y, x1, m.x * x0));
                    }
                    const float tS = !GEN || es >= 0 ? trace(v, cS) : gS[ln];
                    curv_line_c<N1>(sv, fl, u, uL[ln], uR[ln], lo ? tS : tF[ln], lo ? tF[ln] : tS, A.ops);
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        if (d < 2)
                            acc[node(ln, j) - NQ * w] = fmaf(sm.met[node(ln, j)][0].w, sv[j], acc[node(ln, j) - NQ * w]);
                        else
                            sm.fs[b][node(ln, j)][lane] = sv[j];
                    }
                }
            }
        };
        wait(2 + kx);
        lines(std::integral_constant<int, 0>{}, kx, l0, enx);
        wait(2 + ky);
        lines(std::integral_constant<int, 1>{}, ky, l1, eny);
        // slots kx and ky are consumed: the next tile's f^n and x-neighbour layer land there
        __syncwarp();
        if (more && ((lane == RFN && has_fn) || lane == RX)) {
            fence_proxy_async();
            issue_layer(lane == RX && turn ? role_src(enn) : csrc, vl + 1, lane == RX ? ky : kx);
        }
        __syncthreads();  // B1: every layer of the element tile has landed
        // z-lines of slice iy = w (all layers) from the shared tile
        wait(2 + ka);
        lines(std::integral_constant<int, 2>{}, ka, l2, enz);
        // slot ka is consumed: the next tile's y-neighbour layer lands there; warp 0 also brings the next
        // tile's velocity table into the other table buffer (every warp is past B1)
        __syncwarp();
        if (more && (lane == RY || (w == 0 && lane == RT))) {
            fence_proxy_async();
            if (lane == RY) {
                issue_layer(turn ? role_src(enn) : csrc, vl + 1, ka);
            } else {
                mbar_arrive_expect_tx(tbar(b ^ 1), kTabRows * kRow);
                bulk_g2s(smem_u32(&sm.tab[b ^ 1][0][0]), A.vtab + (int64_t)(vt + 1) * kTabRows * kWarp,
                         kTabRows * kRow, tbar(b ^ 1));
            }
        }
        __syncthreads();  // B2: z-sums complete
#pragma unroll
        for (int q = 0; q < NQ; q++)
            acc[q] = fmaf(sm.met[q + NQ * w][0].w, sm.fs[b][q + NQ * w][lane], acc[q]);
        __syncwarp();  // the z-sums of this layer are read before its rows take the stage output
        const float gm = sm.tab[b][3][lane] != 0.f ? 1.f : 0.f;
        const float cg = A.kg * gm, cf = bdt * gm;
        const float xs = x0 * x0 + x1 * x1 + x2 * x2;
        const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
        const bool iso = !GEN || A.viso;
        const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
        const unsigned long long U0 = iso ? pack2(mms, mms) : pack2(mm0, mm0);
        const unsigned long long U1 = iso ? U0 : pack2(mm1, mm1);
        const unsigned long long U2 = iso ? 0ull : pack2(mm2, mm2);
        float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
        float lsum = 0.f, lmin = 3.4e38f;
        auto bgk_src = [&](auto vtau_c, auto force_c, auto lim_c) {
            constexpr bool VT = decltype(vtau_c)::value, FP = decltype(force_c)::value;
            constexpr bool LIM = decltype(lim_c)::value;
#pragma unroll
            for (int h = 0; h < (NQ + 1) / 2; h++) {
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[w][h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];
                const unsigned long long lin =
                    ffma2(pack2(p23.z, p23.w), M2,
                          ffma2(pack2(p23.x, p23.y), M1, ffma2(pack2(p01.z, p01.w), M0, pack2(p01.x, p01.y))));
                const unsigned long long ex =
                    GEN ? ffma2(pack2(p45.x, p45.y), U0,
                                ffma2(pack2(p45.z, p45.w), U1, ffma2(pack2(p67.x, p67.y), U2, lin)))
                        : ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U0, lin));
                float g[2];
                exp2_fp32x2(ex, pack2(p67.z, p67.w), g[0], g[1]);
#pragma unroll
                for (int sl = 0; sl < 2; sl++) {
                    const int q = 2 * h + sl;
                    if (q >= NQ)
                        break;
                    const int i = q + NQ * w;
                    const float a = acc[q];
                    float gc = cg;
                    if constexpr (VT) {
                        const float itau = sl == 0 ? p67.x : p67.y;
                        gc = __fsub_rn(A.b, __fsub_rn(A.b, __fmul_rn(bdt, itau))) * gm;
                    }
                    if constexpr (FP) {
                        const float4 fq = *reinterpret_cast<const float4 *>(&sm.fpar[i][0]);
                        const float qv =
                            fmaf(sm.fpar[i][4], xs, fmaf(fq.w, x2, fmaf(fq.z, x1, fmaf(fq.y, x0, fq.x))));
                        gc = fmaf(cf, qv, gc);  // on top of the node's own Maxwellian weight
                    }
                    const float o = fmaf(gc, g[sl], a);
                    if constexpr (LIM) {
                        lsum = fmaf(sm.met[i][1].w, o, lsum);
                        lmin = fminf(lmin, o);
                    } else {
                        __stcs(dst + i * kWarp, o);
                    }
                    sm.fs[b][q + NQ * w][lane ^ (4 * (q & 7))] = o;
                }
            }
        };
        using T_ = std::true_type;
        using F_ = std::false_type;
        if constexpr (GEN) {
            if (A.limiter) {
                if (A.fpar)
                    A.vtau ? bgk_src(T_{}, T_{}, T_{}) : bgk_src(F_{}, T_{}, T_{});
                else
                    A.vtau ? bgk_src(T_{}, F_{}, T_{}) : bgk_src(F_{}, F_{}, T_{});
            } else {
                if (A.fpar)
                    A.vtau ? bgk_src(T_{}, T_{}, F_{}) : bgk_src(F_{}, T_{}, F_{});
                else
                    A.vtau ? bgk_src(T_{}, F_{}, F_{}) : bgk_src(F_{}, F_{}, F_{});
            }
        } else {
            bgk_src(F_{}, F_{}, F_{});
        }
        if (GEN && A.limiter) {
            // Zhang-Shu (Sec. 2.1, Eqs. 10-11) over the physical element: weights W J over their sum
            sm.lim[0][w][lane] = lsum;
            sm.lim[1][w][lane] = lmin;
            __syncthreads();  // B3
            float mean = 0.f, mn = sm.lim[1][0][lane];
#pragma unroll
            for (int lw = 0; lw < N1; lw++) {
                mean += sm.lim[0][lw][lane];
                mn = fminf(mn, sm.lim[1][lw][lane]);
            }
            mean *= sm.iwj;
            const float beta = mn < 0.f ? fminf(fabsf(mean / (mean - mn)), 1.f) : 1.f;
            if (mn < 0.f) {
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    float &slot_o = sm.fs[b][q + NQ * w][lane ^ (4 * (q & 7))];
                    slot_o = fmaf(beta, slot_o - mean, mean);
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; q++)
                __stcs(dst + (q + NQ * w) * kWarp, sm.fs[b][q + NQ * w][lane ^ (4 * (q & 7))]);
        }
        // moments of this layer's nodes (Eq. 2 with Eq. 12) of the stored values
        __syncwarp();
        unsigned long long pm[2][5];
#pragma unroll
        for (int h = 0; h < NHR; h++)
#pragma unroll
            for (int c = 0; c < 5; c++)
                pm[h][c] = 0ull;
#pragma unroll
        for (int k = 0; k < 8; k += 4) {
            const int kk = 8 * kg + k;
            unsigned long long wv[5][2];
            {
                const float4 W4 = *reinterpret_cast<const float4 *>(&sm.tab[b][3][kk]);
                const float4 E4 = *reinterpret_cast<const float4 *>(&sm.tab[b][4][kk]);
                wv[0][0] = pack2(W4.x, W4.y);
                wv[0][1] = pack2(W4.z, W4.w);
                wv[4][0] = pack2(E4.x, E4.y);
                wv[4][1] = pack2(E4.z, E4.w);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const float4 M4 = *reinterpret_cast<const float4 *>(&sm.tab[b][d][kk]);
                    wv[1 + d][0] = fmul2(pack2(W4.x, W4.y), pack2(M4.x, M4.y));
                    wv[1 + d][1] = fmul2(pack2(W4.z, W4.w), pack2(M4.z, M4.w));
                }
            }
#pragma unroll
            for (int h = 0; h < NHR; h++) {
                const int row = min(np + 8 * h, NQ - 1);
                const float4 v = *reinterpret_cast<const float4 *>(&sm.fs[b][row + NQ * w][kk ^ (4 * (row & 7))]);
                const unsigned long long v01 = pack2(v.x, v.y), v23 = pack2(v.z, v.w);
#pragma unroll
                for (int c = 0; c < 5; c++) {
                    pm[h][c] = ffma2(wv[c][0], v01, pm[h][c]);
                    pm[h][c] = ffma2(wv[c][1], v23, pm[h][c]);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < NHR; h++)
#pragma unroll
            for (int c = 0; c < 5; c++)
                msum[h][c] += sum2(pm[h][c]);
#pragma unroll
        for (int d = 0; d < 3; d++)
            en[d] = enn[d];
        if (turn) {
            csrc = role_src(en);
            octc = octn;
        }
        ka = ka == 2 ? 0 : ka + 1;
    }
    const int grp = A.group0 + gl;
#pragma unroll
    for (int h = 0; h < NHR; h++) {
        const int q = np + 8 * h;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            float x = msum[h][c];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (kg == 0 && q < NQ)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)e * NP + q + NQ * w] = x;
        }
    }
}

template <int N1>
cudaError_t prepare3c()
{
    cudaError_t e = cudaFuncSetAttribute(k_stage3c<N1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Stage3cSmem<N1, 0>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stage3c<N1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(Stage3cSmem<N1, 1>));
    return e;
}

template <int N1, int GEN>
cudaError_t launch3c(const StageArgs &A, cudaStream_t s)
{
    const int ngroups = (A.nvt + A.G - 1) / A.G;
    k_stage3c<N1, GEN><<<A.mesh.nelem * ngroups, kWarp * N1, sizeof(Stage3cSmem<N1, GEN>), s>>>(A);
    return cudaGetLastError();
}

}  // namespace bgk
