// k_stage3.cuh -- the fused SSP-RK3 stage kernel of curvilinear hexahedra with unstructured
// connectivity (FP32-split form), the moments-only pass of every hexahedral mesh, and the dispatch of
// the hexahedral stage kernels: affine hexahedra step in k_stage3s.cuh (k_stage3w.cuh at p <= 2),
// curvilinear hexahedra on the structured element grid in k_stage3c.cuh. Instantiated per degree in
// k_stage3_p*.cu.
#pragma once
#include "k_stage3c.cuh"
#include "k_stage3s.cuh"
#include "k_stage3w.cuh"
#include "stage_common.cuh"

// Resident CTAs per SM the register allocation is sized for (p = 3 moments-only pass / p = 3 with
// the curvilinear advection / p = 2). The register file is split over the SM's four schedulers, so a
// CTA of 3 warps (p = 2) at 80 registers packs 8 per SM (24 warps).
#ifndef BGK_STAGE3_MINCTAS_P3
#define BGK_STAGE3_MINCTAS_P3 5
#endif
#ifndef BGK_STAGE3_MINCTAS_P3_GEN
#define BGK_STAGE3_MINCTAS_P3_GEN 4
#endif
#ifndef BGK_STAGE3_MINCTAS_P2
#define BGK_STAGE3_MINCTAS_P2 8
#endif

namespace bgk {

// ------------------------------------------------------------------------------------------------
// Curvilinear hexahedra with unstructured connectivity: one CTA per (element, run of G tiles), one warp
// per z-layer of the element's nodes, lane l = velocity l of the tile. A warp keeps its layer's values
// (f_s and the accumulator) in registers, so the r- and s-lines are register-local; the t-lines cross
// the layers and are read from a shared copy of the element tile, their sums shared the same way.
// Exterior traces are loaded per lane where the face flow enters (N . xi decides per lane and face
// point): a neighbour's line through a face point may run along any of its axes, so its rows are not
// one contiguous layer to stage.
// ------------------------------------------------------------------------------------------------
template <int N1, int GEN>
struct Stage3Smem {
    static constexpr int NP = N1 * N1 * N1;
    float tile[2][NP][kWarp];     // f_s of the element, [node][lane], double-buffered (cp.async)
    float fnb[NP][kWarp];         // f^n of the element (each warp its own layer), refilled after use
    float zc[NP][kWarp];          // z-derivative sums, [node][lane]
    float msum[N1][10][kWarp];    // per warp and lane: running moment sums of its 2 nodes x 5 moments
    // BGK exponents of the element's points by layer and node pair, [layer][pair][param][node of the
    // pair], so that one 16-byte load gives two parameters of both nodes (odd layers repeat the last node)
    float par[N1][(N1 * N1 + 1) / 2][kParamStride][2];
    float fpar[GEN ? NP : 1][kParamStride];  // body-force polynomials of the element's points (general form)
    float lim[GEN ? 2 : 1][GEN ? N1 : 1][kWarp];  // positivity limiter: per-layer weighted sums and minima
    float wpsi[5][kWarp];         // w psi of the tile's velocities
};

// Curvilinear hexahedra: the element's metric rows and face normals (see StageArgs), placed after the
// stage's shared memory at a 16-byte boundary.
template <int N1>
struct CurvSmem {
    float4 met[N1 * N1 * N1][3];
    // where N1 is even, the rows of direction d again by the node pairs of two adjacent lines (pair_row):
    // (x_a, x_b, y_a, y_b), (z_a, z_b, s_a, s_b) with s = -b dt / J
    float4 metp[N1 % 2 == 0 ? 3 : 1][N1 % 2 == 0 ? N1 * N1 * N1 / 2 : 1][2];
    float4 fnm[3][2][N1 * N1];
    int4 ftab[6];                          // unstructured connectivity of the element (see StageArgs)
    unsigned char fbase[6][N1 * N1];
    float iwj;
};

template <int N1, int GEN, int CURV>
constexpr int stage3_smem_bytes()
{
    return CURV ? (int)((sizeof(Stage3Smem<N1, GEN>) + 15) / 16 * 16 + sizeof(CurvSmem<N1>))
                : (int)sizeof(Stage3Smem<N1, GEN>);
}

// Curvilinear line of direction d (Sec. 2.1, Eqs. 7-9 on the mapped element): with the nodal fluxes
// F_j = u_j f_j (u_j = Ja^d . xi at node j), s_i = (D F)_i + gl'_i (F^I_L - F_L) + gr'_i (F^I_R - F_R)
// = sum_j DM_ij F_j + gl'_i F^I_L + gr'_i F^I_R, where F_L, F_R are the interpolated traces of F (folded
// into DM = D - gl' (x) lm - gr' (x) lp) and F^I the upwind common fluxes of the face normals' u_L, u_R
// (Eq. 9): the exterior trace tL / tR where the face flow enters the element, the element's own trace
// of f where it leaves.
template <int N1>
__device__ __forceinline__ void curv_line(float (&sv)[N1], const float (&fl)[N1], const float (&u)[N1], float uL,
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

// OCT in 0..7: every tile of the launch lies in that sign octant (bit d set: xi_d >= 0, the upwind
// neighbour in direction d is on the low side); OCT = 8: the octant is read per tile.
// GEN = 0: every face periodic, no body force and one velocity spacing on all axes (the lean form;
// the Maxwellian exponent needs only the sum of the squared grid indices); GEN = 1: Dirichlet and
// diffuse-wall faces, the body-force source and per-axis spacings.
// CURV = 2 (OCT = 8; lean or general form): curvilinear hexahedra with unstructured connectivity, the
// reference-space flux (Ja^d . xi) f and per-lane upwinding at every face point from the shared face
// normal, the element's neighbours, their shared faces and face-point orientations from its
// connectivity row (curvilinear hexahedra on the structured element grid step in k_stage3c.cuh).
template <int N1, int MODE, int OCT, int GEN, int CURV = 0>
__global__ void __launch_bounds__(kWarp *N1, (N1 >= 4 ? (GEN || CURV ? BGK_STAGE3_MINCTAS_P3_GEN : BGK_STAGE3_MINCTAS_P3)
                                               : (N1 == 3 ? BGK_STAGE3_MINCTAS_P2 : 8))) k_stage3(const StageArgs A)
{
    static_assert(MODE == 1 || CURV == 2, "affine hexahedra step in k_stage3s, structured curvilinear ones in k_stage3c");
    constexpr int NQ = N1 * N1;      // nodes per layer
    constexpr int NP = NQ * N1;
    constexpr int NT = kWarp * N1;   // threads
    using Sm = Stage3Smem<N1, GEN>;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);
    CurvSmem<N1> &cs = *reinterpret_cast<CurvSmem<N1> *>(smraw + (sizeof(Sm) + 15) / 16 * 16);  // CURV only

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

    if constexpr (MODE == 0) {
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
        if constexpr (CURV) {
            for (int q = tid; q < NP * 3; q += NT)
                (&cs.met[0][0])[q] = __ldg(A.met + (int64_t)e * NP * 3 + q);
            if constexpr (N1 % 2 == 0) {
                const float bdt0 = A.b * A.dt;
                for (int q = tid; q < 3 * NP; q += NT) {  // q = d NP + node a; the pairs' first nodes only
                    const int d = q / NP, a = q % NP;
                    const bool first = d == 0 ? ((a / N1) % N1) % 2 == 0 : (a % N1) % 2 == 0;
                    if (!first)
                        continue;
                    const int bn = a + (d == 0 ? N1 : 1);
                    const float4 ma = __ldg(A.met + ((int64_t)e * NP + a) * 3 + d);
                    const float4 mb = __ldg(A.met + ((int64_t)e * NP + bn) * 3 + d);
                    const float sa = -bdt0 * __ldg(A.met + ((int64_t)e * NP + a) * 3).w;
                    const float sb = -bdt0 * __ldg(A.met + ((int64_t)e * NP + bn) * 3).w;
                    cs.metp[d][pair_row<N1>(d, a)][0] = make_float4(ma.x, mb.x, ma.y, mb.y);
                    cs.metp[d][pair_row<N1>(d, a)][1] = make_float4(ma.z, mb.z, sa, sb);
                }
            }
            for (int q = tid; q < 6 * NQ; q += NT)
                (&cs.fnm[0][0][0])[q] = __ldg(A.fnm + (int64_t)e * 6 * NQ + q);
            if (tid == 0)
                cs.iwj = __ldg(A.iwj + e);
            {
                if (tid < 6)
                    cs.ftab[tid] = __ldg(A.ftab + (int64_t)e * 6 + tid);
                for (int q = tid; q < 6 * NQ; q += NT)
                    (&cs.fbase[0][0])[q] = __ldg(A.fbase + (int64_t)e * 6 * NQ + q);
            }
        }
        // the general form reads 1/tau of its layer (variable collision time), and the curvilinear lines
        // the metric, normals and connectivity, before the first tile's B1, from rows other warps loaded
        if (GEN || CURV)
            __syncthreads();
    }
    // moment sums: lane = (node pair np = lane / 4: layer nodes np and np + 8) x (velocity eighth
    // kg = lane % 4: velocities 8 kg .. 8 kg + 7 of every tile); FP32 pairs over even/odd velocities
    // per tile, added to running sums in shared memory (no registers held across the tile), combined
    // across the 4 lanes of a pair at the end. The stage output of the warp's layer is transposed
    // through the layer's own rows of the tile buffer, free once the z-lines have read them (B2), with
    // the 4-float column groups of row q rotated by q mod 8 (conflict-free writes and reads).
    const int np = lane >> 2, kg = lane & 3;
    // the second half of the rows (np + 8) exists only for layers of more than 8 nodes. Every row is
    // summed in the same order, so equal rows give bit-equal moments (a y/z-homogeneous state stays so).
    constexpr int NHR = NQ > 8 ? 2 : 1;
#pragma unroll
    for (int m = 0; m < 10; m++)
        sm.msum[w][m][lane] = 0.f;
    const float kb = A.kb;
    const float bdt = A.b * A.dt;
    // Exterior traces through face (d, side) of the connectivity row for the N1 lines of this warp whose
    // face points are fp0 + ln, where the lane's flow enters (need[ln]), 0 elsewhere: the neighbour's
    // interpolant at the shared face (its line through the face point: first node and stride from the
    // row), or the face's ghost value (times the wall density of the point on a wall). The loads of all
    // lines are in flight together, and nothing is read where no lane of the warp needs a value.
    auto exteriors = [&](int vl, int slot, int d, int side, int fp0, const bool(&need)[N1], float(&t)[N1]) {
        bool any = false;
#pragma unroll
        for (int ln = 0; ln < N1; ln++) {
            t[ln] = 0.f;
            any = any || need[ln];
        }
        if (!__any_sync(0xffffffffu, any))
            return;
        const int4 tb = cs.ftab[2 * d + side];
        if (tb.x < 0) {
            const float gv = __ldg(A.ghost + (int64_t)(-1 - tb.x) * A.nslots + slot);
            if (tb.w >= 0) {  // a wall face (the test outside the loop: no load from an invalid address)
#pragma unroll
                for (int ln = 0; ln < N1; ln++)
                    t[ln] = gv * __ldg(A.rhowu + (int64_t)tb.w * NQ + fp0 + ln);
            } else {
#pragma unroll
                for (int ln = 0; ln < N1; ln++)
                    t[ln] = gv;
            }
            return;
        }
        const float *nb = A.src + fidx(vl, tb.x, 0, lane, E, NP);
        float v[N1][N1];
#pragma unroll
        for (int ln = 0; ln < N1; ln++) {
            const int base = cs.fbase[2 * d + side][fp0 + ln];
#pragma unroll
            for (int j = 0; j < N1; j++)
                v[ln][j] = need[ln] ? __ldg(nb + (base + j * tb.y) * kWarp) : 0.f;
        }
#pragma unroll
        for (int ln = 0; ln < N1; ln++)
            t[ln] = tb.z ? trace_line<N1, true>(v[ln], A.ops) : trace_line<N1, false>(v[ln], A.ops);
    };

    // asynchronous copy of this warp's layer of f_s (and f^n) of tile vl into buffer b: NQ rows of
    // 128 bytes, contiguous in global and shared memory
    const bool has_fn = MODE == 0 && A.fn != nullptr;
    constexpr int NCH = NQ * kWarp / 4;  // 16-byte chunks of one layer
    auto prefetch = [&](int vl, int b) {
        const float4 *gs = reinterpret_cast<const float4 *>(A.src + fidx(vl, e, NQ * w, 0, E, NP));
        float4 *ss = reinterpret_cast<float4 *>(&sm.tile[b][NQ * w][0]);
#pragma unroll
        for (int m = lane; m < NCH; m += kWarp)
            cp_async16(ss + m, gs + m);
        cp_commit();
    };
    // f^n of this warp's layer: one buffer, refilled for the next tile once this tile has read it
    auto prefetch_fn = [&](int vl) {
        if (has_fn) {
            const float4 *gf = reinterpret_cast<const float4 *>(A.fn + fidx(vl, e, NQ * w, 0, E, NP));
            float4 *sf = reinterpret_cast<float4 *>(&sm.fnb[NQ * w][0]);
#pragma unroll
            for (int m = lane; m < NCH; m += kWarp)
                cp_async16(sf + m, gf + m);
        }
        cp_commit();
    };
    prefetch(vl0, 0);
    prefetch_fn(vl0);
    // the tile's grid indices and padding mask, loaded one tile ahead into registers
    float mi_n[3], gm_n = 0.f;
    auto load_rows = [&](int vt) {
        const int sl = vt * kWarp + lane;
#pragma unroll
        for (int d = 0; d < 3; d++)
            mi_n[d] = __ldg(A.mi + d * A.nslots + sl);
        gm_n = __ldg(A.gmask + sl);
    };
    if (vl0 < vl1)
        load_rows(A.vt0 + vl0);

    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const int b = (vl - vl0) & 1;
        const float m0 = mi_n[0], m1 = mi_n[1], m2 = mi_n[2], gm_c = gm_n;
        if (vl + 1 < vl1)
            load_rows(vt + 1);
        // the other buffer was last read before the previous tile's B2, which every warp has passed;
        // pending groups: tile vl, f^n vl (issued last tile), then tile vl + 1
        if (vl + 1 < vl1) {
            prefetch(vl + 1, b ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncwarp();
        const float x0 = fmaf(A.vs[0], m0, A.vc[0]), x1 = fmaf(A.vs[1], m1, A.vc[1]), x2 = fmaf(A.vs[2], m2, A.vc[2]);
        float f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++)
            f[q] = sm.tile[b][q + NQ * w][lane];
        if constexpr (MODE == 0) {
            float acc[NQ];
            if (has_fn) {
#pragma unroll
                for (int q = 0; q < NQ; q++)
                    acc[q] = sm.fnb[q + NQ * w][lane];
            } else {
#pragma unroll
                for (int q = 0; q < NQ; q++)
                    acc[q] = 0.f;
            }
            __syncwarp();  // every lane has read its f^n rows before they are refilled
            if (vl + 1 < vl1)
                prefetch_fn(vl + 1);
            else
                cp_commit();  // keep the group count per tile fixed
            const float cz = -A.mesh.inv_h2[2] * x2 * bdt;
            if constexpr (CURV) {
                // curvilinear: kb f_s as above, then the x- and y-lines of layer w with the metric
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    float kbq = kb;
                    if (GEN && A.vtau)
                        kbq = __fsub_rn(A.b, __fmul_rn(bdt, sm.par[w][q / 2][6][q % 2]));
                    acc[q] = fmaf(A.an, acc[q], kbq * f[q]);
                }
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    // face-normal speeds of the warp's lines, then the exterior traces where the flow enters
                    float uLs[N1], uRs[N1], tLs[N1], tRs[N1];
                    bool inL[N1], inR[N1];
#pragma unroll
                    for (int ln = 0; ln < N1; ln++) {
                        const float4 nL = cs.fnm[d][0][ln + N1 * w], nR = cs.fnm[d][1][ln + N1 * w];
                        uLs[ln] = fmaf(nL.z, x2, fmaf(nL.y, x1, nL.x * x0));
                        uRs[ln] = fmaf(nR.z, x2, fmaf(nR.y, x1, nR.x * x0));
                        inL[ln] = uLs[ln] > 0.f;
                        inR[ln] = uRs[ln] < 0.f;
                    }
                    exteriors(vl, slot, d, 0, N1 * w, inL, tLs);
                    exteriors(vl, slot, d, 1, N1 * w, inR, tRs);
                    if constexpr (N1 % 2 == 0) {
                        // two adjacent lines on packed FP32 pairs, each half curv_line's operations in
                        // its order (bit-identical results)
                        const unsigned long long X0 = pack2(x0, x0), X1 = pack2(x1, x1), X2 = pack2(x2, x2);
#pragma unroll
                        for (int ln = 0; ln < N1; ln += 2) {
                            unsigned long long fl[N1], F[N1], sp[N1];
                            int qa[N1], qb[N1];
#pragma unroll
                            for (int j = 0; j < N1; j++) {
                                qa[j] = d == 0 ? j + N1 * ln : ln + N1 * j;
                                qb[j] = qa[j] + (d == 0 ? N1 : 1);
                                fl[j] = pack2(f[qa[j]], f[qb[j]]);
                                const float4 *mp = &cs.metp[d][pair_row<N1>(d, qa[j] + NQ * w)][0];
                                const float4 p0 = mp[0], p1 = mp[1];
                                const unsigned long long u =
                                    ffma2(pack2(p1.x, p1.y), X2, ffma2(pack2(p0.z, p0.w), X1, fmul2(pack2(p0.x, p0.y), X0)));
                                F[j] = fmul2(u, fl[j]);
                                sp[j] = pack2(p1.z, p1.w);
                            }
                            unsigned long long oL = 0ull, oR = 0ull;
#pragma unroll
                            for (int j = 0; j < N1; j++) {
                                oL = ffma2(dup2(A.ops.lm[j]), fl[j], oL);
                                oR = ffma2(dup2(A.ops.lp[j]), fl[j], oR);
                            }
                            float oL2[2], oR2[2], FI[2][2];
                            unpack2(oL, oL2[0], oL2[1]);
                            unpack2(oR, oR2[0], oR2[1]);
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                FI[0][h] = uLs[ln + h] * (uLs[ln + h] > 0.f ? tLs[ln + h] : oL2[h]);
                                FI[1][h] = uRs[ln + h] * (uRs[ln + h] < 0.f ? tRs[ln + h] : oR2[h]);
                            }
                            const unsigned long long FIL = pack2(FI[0][0], FI[0][1]), FIR = pack2(FI[1][0], FI[1][1]);
#pragma unroll
                            for (int i = 0; i < N1; i++) {
                                unsigned long long a = ffma2(dup2(A.ops.gl[i]), FIL, fmul2(dup2(A.ops.gr[i]), FIR));
#pragma unroll
                                for (int j = 0; j < N1; j++)
                                    a = ffma2(dup2(A.ops.DM[i][j]), F[j], a);
                                float sa, sb, ca, cb;
                                unpack2(a, sa, sb);
                                unpack2(sp[i], ca, cb);
                                acc[qa[i]] = fmaf(ca, sa, acc[qa[i]]);
                                acc[qb[i]] = fmaf(cb, sb, acc[qb[i]]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int ln = 0; ln < N1; ln++) {
                            float fl[N1], u[N1], sv[N1];
                            int nd[N1], qi[N1];  // element node and in-layer node (compile-time) of the line
#pragma unroll
                            for (int j = 0; j < N1; j++) {
                                qi[j] = d == 0 ? j + N1 * ln : ln + N1 * j;
                                nd[j] = qi[j] + NQ * w;
                                fl[j] = f[qi[j]];
                                const float4 m = cs.met[nd[j]][d];
                                u[j] = fmaf(m.z, x2, fmaf(m.y, x1, m.x * x0));
                            }
                            curv_line<N1>(sv, fl, u, uLs[ln], uRs[ln], tLs[ln], tRs[ln], A.ops);
#pragma unroll
                            for (int j = 0; j < N1; j++)
                                acc[qi[j]] = fmaf(-bdt * cs.met[nd[j]][0].w, sv[j], acc[qi[j]]);
                        }
                    }
                }
                __syncthreads();  // B1: the element tile is complete
                if (w == 0) {
#pragma unroll
                    for (int c = 0; c < 5; c++)
                        sm.wpsi[c][lane] = __ldg(A.wpsi + ((int64_t)vt * 5 + c) * kWarp + lane);
                }
                // z-lines of slice iy = w (all layers) from the shared tile; unscaled sums to zc
                float uLs[N1], uRs[N1], tLs[N1], tRs[N1];
                bool inL[N1], inR[N1];
#pragma unroll
                for (int ln = 0; ln < N1; ln++) {
                    const float4 nL = cs.fnm[2][0][ln + N1 * w], nR = cs.fnm[2][1][ln + N1 * w];
                    uLs[ln] = fmaf(nL.z, x2, fmaf(nL.y, x1, nL.x * x0));
                    uRs[ln] = fmaf(nR.z, x2, fmaf(nR.y, x1, nR.x * x0));
                    inL[ln] = uLs[ln] > 0.f;
                    inR[ln] = uRs[ln] < 0.f;
                }
                exteriors(vl, slot, 2, 0, N1 * w, inL, tLs);
                exteriors(vl, slot, 2, 1, N1 * w, inR, tRs);
                if constexpr (N1 % 2 == 0) {  // paired z-lines (as the x- and y-lines above)
                    const unsigned long long X0 = pack2(x0, x0), X1 = pack2(x1, x1), X2 = pack2(x2, x2);
#pragma unroll
                    for (int ln = 0; ln < N1; ln += 2) {
                        unsigned long long fl[N1], F[N1];
#pragma unroll
                        for (int j = 0; j < N1; j++) {
                            const int nd = ln + N1 * w + NQ * j;
                            fl[j] = pack2(sm.tile[b][nd][lane], sm.tile[b][nd + 1][lane]);
                            const float4 *mp = &cs.metp[2][pair_row<N1>(2, nd)][0];
                            const float4 p0 = mp[0], p1 = mp[1];
                            const unsigned long long u =
                                ffma2(pack2(p1.x, p1.y), X2, ffma2(pack2(p0.z, p0.w), X1, fmul2(pack2(p0.x, p0.y), X0)));
                            F[j] = fmul2(u, fl[j]);
                        }
                        unsigned long long oL = 0ull, oR = 0ull;
#pragma unroll
                        for (int j = 0; j < N1; j++) {
                            oL = ffma2(dup2(A.ops.lm[j]), fl[j], oL);
                            oR = ffma2(dup2(A.ops.lp[j]), fl[j], oR);
                        }
                        float oL2[2], oR2[2], FI[2][2];
                        unpack2(oL, oL2[0], oL2[1]);
                        unpack2(oR, oR2[0], oR2[1]);
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            FI[0][h] = uLs[ln + h] * (uLs[ln + h] > 0.f ? tLs[ln + h] : oL2[h]);
                            FI[1][h] = uRs[ln + h] * (uRs[ln + h] < 0.f ? tRs[ln + h] : oR2[h]);
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
                            const int nd = ln + N1 * w + NQ * i;
                            sm.zc[nd][lane] = sa;
                            sm.zc[nd + 1][lane] = sb;
                        }
                    }
                } else
#pragma unroll
                for (int ln = 0; ln < N1; ln++) {
                    float fl[N1], u[N1], sv[N1];
                    int nd[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        nd[j] = ln + N1 * w + NQ * j;
                        fl[j] = sm.tile[b][nd[j]][lane];
                        const float4 m = cs.met[nd[j]][2];
                        u[j] = fmaf(m.z, x2, fmaf(m.y, x1, m.x * x0));
                    }
                    curv_line<N1>(sv, fl, u, uLs[ln], uRs[ln], tLs[ln], tRs[ln], A.ops);
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        sm.zc[nd[j]][lane] = sv[j];
                }
                __syncthreads();  // B2: z-sums complete
            }
            // BGK source towards the conservative Maxwellian, Shu-Osher combination, store
            const float gm = gm_c;
            const float cg = A.kg * gm, cf = bdt * gm;
            const float xs = x0 * x0 + x1 * x1 + x2 * x2;
            // squared indices (exact); the lean form has one spacing on every axis and needs their sum
            const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
            const bool iso = !GEN || A.viso;
            const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
            const unsigned long long U0 = iso ? pack2(mms, mms) : pack2(mm0, mm0);
            const unsigned long long U1 = iso ? U0 : pack2(mm1, mm1);
            const unsigned long long U2 = iso ? 0ull : pack2(mm2, mm2);
            float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
            float lsum = 0.f, lmin = 3.4e38f;  // limiter: this layer's weighted sum and minimum
            // two nodes at a time: the exponent a + b.m + q |m|^2 (+ the low part of q) and the range
            // reduction of 2^x in packed pairs
#pragma unroll
            for (int h = 0; h < (NQ + 1) / 2; h++) {
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[w][h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];  // (c, c+1) of both nodes
                const unsigned long long lin =
                    ffma2(pack2(p23.z, p23.w), M2,
                          ffma2(pack2(p23.x, p23.y), M1, ffma2(pack2(p01.z, p01.w), M0, pack2(p01.x, p01.y))));
                const unsigned long long ex =
                    GEN ? ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U1, ffma2(pack2(p67.x, p67.y), U2, lin)))
                        : ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U0, lin));
                float g[2];
                exp2_fp32x2(ex, pack2(p67.z, p67.w), g[0], g[1]);
#pragma unroll
                for (int sl = 0; sl < 2; sl++) {
                    const int q = 2 * h + sl;
                    if (q >= NQ)
                        break;
                    const int i = q + NQ * w;
                    const float a = CURV ? fmaf(-bdt * cs.met[i][0].w, sm.zc[i][lane], acc[q])
                                         : fmaf(cz, sm.zc[i][lane], acc[q]);
                    float gc = cg;
                    if (GEN && A.vtau) {  // kg = b - kb exactly, kb as in the accumulator above
                        const float itau = sl == 0 ? p67.x : p67.y;
                        gc = __fsub_rn(A.b, __fsub_rn(A.b, __fmul_rn(bdt, itau))) * gm;
                    }
                    if (GEN && A.fpar) {  // body-force source g (q0 + q . xi + q4 |xi|^2)
                        const float4 fq = *reinterpret_cast<const float4 *>(&sm.fpar[i][0]);
                        const float qv = fmaf(sm.fpar[i][4], xs, fmaf(fq.w, x2, fmaf(fq.z, x1, fmaf(fq.y, x0, fq.x))));
                        gc = fmaf(cf, qv, gc);  // on top of the node's own Maxwellian weight
                    }
                    const float o = fmaf(gc, g[sl], a);
                    if (GEN && A.limiter) {  // stored after the limiter below
                        lsum = fmaf(CURV ? cs.met[i][1].w : A.ops.wq[q % N1] * A.ops.wq[q / N1], o, lsum);
                        lmin = fminf(lmin, o);
                    } else {
                        __stcs(dst + i * kWarp, o);
                    }
                    sm.tile[b][q + NQ * w][lane ^ (4 * (q & 7))] = o;  // for the moments below
                }
            }
            if (GEN && A.limiter) {
                // Zhang-Shu (Sec. 2.1, Eqs. 10-11): element mean and minimum of every velocity over
                // the four layers, then the contraction of the values of this warp's layer
                sm.lim[0][w][lane] = CURV ? lsum : A.ops.wq[w] * lsum;
                sm.lim[1][w][lane] = lmin;
                __syncthreads();  // B3 (the general form only)
                float mean = 0.f, mn = sm.lim[1][0][lane];
#pragma unroll
                for (int lw = 0; lw < N1; lw++) {
                    mean += sm.lim[0][lw][lane];
                    mn = fminf(mn, sm.lim[1][lw][lane]);
                }
                if (CURV)  // the physical element's mean: weights W J over their sum
                    mean *= cs.iwj;
                const float beta = mn < 0.f ? fminf(fabsf(mean / (mean - mn)), 1.f) : 1.f;
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    float &slot_o = sm.tile[b][q + NQ * w][lane ^ (4 * (q & 7))];
                    float o = slot_o;
                    if (mn < 0.f) {
                        o = fmaf(beta, o - mean, mean);
                        slot_o = o;
                    }
                    __stcs(dst + (q + NQ * w) * kWarp, o);
                }
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
                sm.tile[b][q + NQ * w][lane ^ (4 * (q & 7))] = f[q];
        }
        // moments of this layer's nodes (Eq. 2 with Eq. 12) of the stored values (rows np + 8 h)
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
#pragma unroll
            for (int c = 0; c < 5; c++) {
                const float4 w4 = *reinterpret_cast<const float4 *>(&sm.wpsi[c][kk]);
                wv[c][0] = pack2(w4.x, w4.y);
                wv[c][1] = pack2(w4.z, w4.w);
            }
#pragma unroll
            for (int h = 0; h < NHR; h++) {
                const int row = min(np + 8 * h, NQ - 1);  // rows past the layer: discarded below
                const float4 v = *reinterpret_cast<const float4 *>(&sm.tile[b][row + NQ * w][kk ^ (4 * (row & 7))]);
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
                sm.msum[w][5 * h + c][lane] += sum2(pm[h][c]);
        __syncwarp();
    }
    // partial moments of this task: combine the 4 velocity eighths of every node pair
    const int grp = A.group0 + gl;
#pragma unroll
    for (int h = 0; h < NHR; h++) {
        const int q = np + 8 * h;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            float x = sm.msum[w][5 * h + c][lane];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (kg == 0 && q < NQ)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)e * NP + q + NQ * w] = x;
        }
    }
}


template <int N1, int MODE, int OCT, int GEN, int CURV = 0>
cudaError_t launch3(const StageArgs &A, cudaStream_t s)
{
    const int ngroups = (A.nvt + A.G - 1) / A.G;
    k_stage3<N1, MODE, OCT, GEN, CURV>
        <<<A.mesh.nelem * ngroups, kWarp * N1, stage3_smem_bytes<N1, GEN, CURV>(), s>>>(A);
    return cudaGetLastError();
}

template <int N1>
cudaError_t prepare3()
{
    const int s0 = (int)sizeof(Stage3Smem<N1, 0>);
    cudaError_t e = cudaFuncSetAttribute(k_stage3<N1, 1, 8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0);
    if constexpr (N1 <= 3) {
        if (e == cudaSuccess)
            e = prepare3w<N1>();
    } else {
        if (e == cudaSuccess)
            e = prepare3s<N1>();
    }
    if (e == cudaSuccess)
        e = prepare3c<N1>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stage3<N1, 0, 8, 1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 stage3_smem_bytes<N1, 1, 2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stage3<N1, 0, 8, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 stage3_smem_bytes<N1, 0, 2>());

    return e;
}

// mode 0: stage of octant oct (8 = mixed octants), lean (all periodic, no force) or general form;
// mode 1: moments only
template <int N1>
cudaError_t launch3_any(const StageArgs &A, int mode, int oct, cudaStream_t s)
{
    if (mode == 1)
        return launch3<N1, 1, 8, 0>(A, s);
    // the lean form: periodic faces, no force, no limiter, constant tau, one velocity spacing on all axes
    bool general = A.fpar != nullptr || !A.viso || A.limiter || A.vtau;
    for (int f = 0; f < 6; f++)  // Dirichlet or wall faces (exchange faces need only the neighbour's source)
        general = general || A.mesh.bc[f] == 1 || A.mesh.bc[f] == 2;
    if (A.met)  // curvilinear hexahedra: the metric, the upwind side per lane
        return A.ftab ? (general ? launch3<N1, 0, 8, 1, 2>(A, s) : launch3<N1, 0, 8, 0, 2>(A, s))
                      : (general ? launch3c<N1, 1>(A, s) : launch3c<N1, 0>(A, s));
    if constexpr (N1 <= 3) {  // p <= 2: one warp per element
        // Dirichlet faces and the limiter only (no wall, force or variable tau, one spacing): GEN = 2
        bool full = A.fpar != nullptr || !A.viso || A.vtau;
        for (int f = 0; f < 6; f++)
            full = full || A.mesh.bc[f] == 2;
        return !general ? launch3w_oct<N1, 0>(A, oct, s)
                        : (full ? launch3w_oct<N1, 1>(A, oct, s) : launch3w_oct<N1, 2>(A, oct, s));
    }
    else
        return general ? launch3s_oct<N1, 1>(A, oct, s) : launch3s_oct<N1, 0>(A, oct, s);
}

}  // namespace bgk
