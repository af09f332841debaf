// k_stage3w.cuh -- the fused SSP-RK3 stage kernel for affine hexahedra of degree p <= 2 (FP32-split
// form): one warp per element, every operand staged in shared memory by bulk asynchronous copies.
// Instantiated in k_stage3_p1.cu and k_stage3_p2.cu.
#pragma once
#include <type_traits>

#include "stage_common.cuh"

#ifndef BGK_STAGE3W_WARPS
#define BGK_STAGE3W_WARPS 1  // elements (warps) per CTA
#endif
#ifndef BGK_STAGE3W_MINCTAS_P2
#define BGK_STAGE3W_MINCTAS_P2 13  // resident CTAs per SM the register allocation is sized for (p = 2)
#endif

namespace bgk {

// ------------------------------------------------------------------------------------------------
// At p <= 2 an element has at most 27 nodes, so one warp holds all of them: lane = velocity of the
// tile, f_s and the accumulator of every node in registers. The x-, y- and z-lines are then all
// register-local, the positivity limiter's element mean and minimum are sums over the lane's own
// registers, and no warp waits for another: the CTA's warps (consecutive elements, the same run of
// velocity tiles) share no data and no barrier in the tile loop. Compared with one warp per z-layer,
// the per-tile work that does not grow with the nodes (barrier waits, copy issue, the velocity table,
// the moment pass's row layout) is spread over 27 nodes instead of 9.
// Shared memory per warp (bulk copies, the warp's own mbarriers):
//   fs     f_s of the element: read into registers at the start of the tile, after which the next
//          tile's f_s lands there;
//   sl[3]  three rotating slots of one element each, as k_stage3s: at tile t slot t mod 3 holds f^n,
//          slot t+1 the x-upwind neighbour and slot t+2 the y-upwind neighbour; slot t mod 3 then takes
//          the z-upwind neighbour (read by the z-lines), then the tile's output, transposed, for the
//          moment sums; each slot takes the next tile's copies as soon as it is consumed;
//   tab[2] the tile's velocity table (grid indices, W, energy weight), with f_s on its barrier.
// Forms: GEN = 0 every face periodic or an exchange face, no force, no limiter, constant tau, one
// velocity spacing; GEN = 2 adds Dirichlet ghosts and the limiter; GEN = 1 everything (diffuse walls,
// the force source, variable tau, per-axis spacings). Feature tests that are uniform over a launch sit
// outside the unrolled node loops, so every such loop stays one basic block.
// ------------------------------------------------------------------------------------------------
template <int N1, int GEN>
struct __align__(16) Stage3wWarp {  // a multiple of 16 bytes, so every warp's copy targets stay aligned
    static constexpr int NP = N1 * N1 * N1;
    float fs[NP][kWarp];
    float sl[3][NP][kWarp];
    float tab[2][5][kWarp];
    float par[(NP + 1) / 2][kParamStride][2];  // BGK exponents by node pair (the last pair repeats node NP-1)
    float fpar[GEN == 1 ? NP : 1][GEN == 1 ? kParamStride : 1];
    unsigned long long bar[5];  // fs and the table of tile parity 0 and 1, sl[0..2]
};

template <int N1, int OCT, int GEN>
__global__ void __launch_bounds__(kWarp *BGK_STAGE3W_WARPS, (N1 == 3 ? BGK_STAGE3W_MINCTAS_P2 : 16))
    k_stage3w(const StageArgs A)
{
    constexpr int NQ = N1 * N1;
    constexpr int NP = NQ * N1;
    constexpr int NH = (NP + 1) / 2;
    constexpr uint32_t kRow = kWarp * sizeof(float);
    using Sm = Stage3wWarp<N1, GEN>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    Sm &sm = reinterpret_cast<Sm *>(smraw)[wq];

    const int E = A.mesh.nelem;
    const int nblk = (E + BGK_STAGE3W_WARPS - 1) / BGK_STAGE3W_WARPS;
    const int gl = blockIdx.x / nblk;
    const int e = (blockIdx.x % nblk) * BGK_STAGE3W_WARPS + wq;
    if (e >= E)  // no barrier below involves other warps
        return;
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    int ec[3];
    ec[0] = e % A.mesh.ne[0];
    ec[1] = (e / A.mesh.ne[0]) % A.mesh.ne[1];
    ec[2] = e / (A.mesh.ne[0] * A.mesh.ne[1]);

    // per-point BGK exponents (and force polynomials) of the element, by node pair
    {
        const float *src = A.param + (int64_t)e * NP * kParamStride;
        for (int q = lane; q < NH * 2 * kParamStride; q += kWarp) {
            const int c = q % kParamStride, s2 = (q / kParamStride) & 1, h = q / (2 * kParamStride);
            sm.par[h][c][s2] = __ldg(src + min(2 * h + s2, NP - 1) * kParamStride + c);
        }
        if (GEN == 1 && A.fpar) {
            const float4 *f4 = reinterpret_cast<const float4 *>(A.fpar + (int64_t)e * NP * kParamStride);
            float4 *d4 = reinterpret_cast<float4 *>(&sm.fpar[0][0]);
            for (int q = lane; q < NP * kParamStride / 4; q += kWarp)
                d4[q] = __ldg(f4 + q);
        }
    }
    const uint32_t bar0 = smem_u32(&sm.bar[0]);
    auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 5; i++)
            mbar_init(bar(i), 1);
        fence_mbar_init();
    }
    __syncwarp();

    const bool has_fn = A.fn != nullptr;
    auto nbrs = [&](int vl, int (&en)[3]) {
        const int oct = OCT < 8 ? OCT : (int)__ldg(A.toct + A.vt0 + vl);
#pragma unroll
        for (int d = 0; d < 3; d++)
            en[d] = upwind_neighbour(A.mesh, ec, d, ((oct >> d) & 1) != 0);
    };
    // Copies, one role lane each: lane 0 f_s (and the velocity table), RFN f^n, RX / RY / RZ the x-, y-
    // and z-upwind neighbours (an element each; a halo element across an exchange x face; nothing on a
    // Dirichlet or wall face). A role lane keeps its source at tile 0 and adds its tile stride.
    constexpr int RFN = 1, RX = 2, RY = 3, RZ = 4;
    const int64_t tstride = (int64_t)E * NP * kWarp;
    const int64_t hstride = (int64_t)A.eface * NP * kWarp;
    int64_t cstride = tstride;
    auto role_src = [&](const int (&en)[3], int oct) -> const float * {
        cstride = tstride;
        if (lane == RX && en[0] == kHaloNeighbour) {
            cstride = hstride;
            const int64_t r = ec[1] + (int64_t)A.mesh.ne[1] * ec[2];
            return A.halo[(oct & 1) ? 0 : 1] + ((int64_t)A.vt0 * A.eface + r) * NP * kWarp;
        }
        if (lane == 0)
            return A.src + fidx(0, e, 0, 0, E, NP);
        if (lane == RFN)
            return A.fn ? A.fn + fidx(0, e, 0, 0, E, NP) : nullptr;
        if (lane == RX || lane == RY || lane == RZ) {
            const int n = lane == RX ? en[0] : (lane == RY ? en[1] : en[2]);
            return n >= 0 ? A.src + fidx(0, n, 0, 0, E, NP) : nullptr;
        }
        return nullptr;
    };
    const uint32_t fs0 = smem_u32(&sm.fs[0][0]), sl0 = smem_u32(&sm.sl[0][0][0]);
    constexpr uint32_t kElem = NP * kRow;
    auto issue_fs = [&](const float *csrc, int vl, int b) {  // lane 0
        mbar_arrive_expect_tx(bar(b), kElem + 5 * kRow);
        bulk_g2s(fs0, csrc + vl * tstride, kElem, bar(b));
        bulk_g2s(smem_u32(&sm.tab[b][0][0]), A.vtab + (int64_t)(A.vt0 + vl) * 5 * kWarp, 5 * kRow, bar(b));
    };
    auto issue_elem = [&](const float *csrc, int vl, int k) {  // role lanes
        const uint32_t bb = bar(2 + k);
        mbar_arrive_expect_tx(bb, csrc ? kElem : 0);
        if (csrc)
            bulk_g2s(sl0 + k * kElem, csrc + vl * cstride, kElem, bb);
    };

    int en[3];
    nbrs(vl0, en);
    const float *csrc = role_src(en, OCT < 8 ? OCT : (int)__ldg(A.toct + A.vt0 + vl0));
    if (lane == 0)
        issue_fs(csrc, vl0, 0);
    if (lane == RFN && has_fn)
        issue_elem(csrc, vl0, 0);
    if (lane == RX)
        issue_elem(csrc, vl0, 1);
    if (lane == RY)
        issue_elem(csrc, vl0, 2);
    uint32_t ph = 0;
    auto wait = [&](int i) {
        mbar_wait(bar(i), (ph >> i) & 1, A.err);
        ph ^= 1u << i;
    };

    // moment sums: lane = (row np = lane / 4 of every group of 8 nodes) x (velocity eighth kg = lane % 4),
    // rows np + 8 h; every row is summed in the same order (a y/z-homogeneous state gives bit-equal rows)
    const int np = lane >> 2, kg = lane & 3;
    constexpr int NHR = (NP + 7) / 8;
    float msum[NHR][5];
#pragma unroll
    for (int h = 0; h < NHR; h++)
#pragma unroll
        for (int c = 0; c < 5; c++)
            msum[h][c] = 0.f;
    const float kb = A.kb;
    const float bdt = A.b * A.dt;

    int ka = 0;  // slot of f^n (then of the z-neighbour) in this tile; x- and y-neighbours in ka + 1, ka + 2
    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const int b = (vl - vl0) & 1;
        const int kx = ka == 2 ? 0 : ka + 1, ky = ka == 0 ? 2 : ka - 1;
        int enn[3] = {en[0], en[1], en[2]};
        if (OCT == 8 && vl + 1 < vl1)
            nbrs(vl + 1, enn);
        const bool more = vl + 1 < vl1;
        const int oct = OCT < 8 ? OCT : (int)__ldg(A.toct + vt);
        const bool l0 = (oct & 1) != 0, l1 = (oct & 2) != 0, l2 = (oct & 4) != 0;
        const int enx = en[0], eny = en[1], enz = en[2];

        wait(b);
        const float m0 = sm.tab[b][0][lane], m1 = sm.tab[b][1][lane], m2 = sm.tab[b][2][lane];
        const float x0 = fmaf(A.vs[0], m0, A.vc[0]), x1 = fmaf(A.vs[1], m1, A.vc[1]), x2 = fmaf(A.vs[2], m2, A.vc[2]);
        float f[NP];
#pragma unroll
        for (int q = 0; q < NP; q++)
            f[q] = sm.fs[q][lane];
        // f_s is in registers: the next tile's lands in fs
        __syncwarp();
        if (lane == 0 && more) {
            fence_proxy_async();
            issue_fs(csrc, vl + 1, b ^ 1);
        }
        float acc[NP];
        if (has_fn) {
            wait(2 + ka);
#pragma unroll
            for (int q = 0; q < NP; q++)
                acc[q] = sm.sl[ka][q][lane];
        } else {
#pragma unroll
            for (int q = 0; q < NP; q++)
                acc[q] = 0.f;
        }
        // slot ka is consumed: the z-neighbour lands there
        __syncwarp();
        if (lane == RZ) {
            fence_proxy_async();
            issue_elem(OCT < 8 ? csrc : role_src(en, oct), vl, ka);
        }
        // acc = an f^n + b (1 - dt/tau) f_s
        // (the launch-uniform feature tests sit outside the unrolled node loops, which then stay one
        // basic block each)
        if (GEN == 1 && A.vtau) {
#pragma unroll
            for (int q = 0; q < NP; q++)
                acc[q] = fmaf(A.an, acc[q], __fsub_rn(A.b, __fmul_rn(bdt, sm.par[q / 2][6][q % 2])) * f[q]);
        } else {
#pragma unroll
            for (int q = 0; q < NP; q++)
                acc[q] = fmaf(A.an, acc[q], kb * f[q]);
        }
        const float cx = -A.mesh.inv_h2[0] * x0 * bdt, cy = -A.mesh.inv_h2[1] * x1 * bdt;
        const float cz = -A.mesh.inv_h2[2] * x2 * bdt;
        // upwind values on Dirichlet and wall faces; face point of a line: its two other indices
        const int fx = 0 + (l0 ? 0 : 1), fy = 2 + (l1 ? 0 : 1), fz = 4 + (l2 ? 0 : 1);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        const float *rwx = nullptr, *rwy = nullptr, *rwz = nullptr;
        if (GEN) {
            gx = enx != -1 ? 0.f : __ldg(A.ghost + fx * A.nslots + slot);
            gy = eny >= 0 ? 0.f : __ldg(A.ghost + fy * A.nslots + slot);
            gz = enz >= 0 ? 0.f : __ldg(A.ghost + fz * A.nslots + slot);
            if (GEN == 1 && enx < 0 && A.mesh.bc[fx] == 2)
                rwx = A.rhow + ((int64_t)fx * A.nfmax + face_elem(A.mesh, ec, 0)) * NQ;
            if (GEN == 1 && eny < 0 && A.mesh.bc[fy] == 2)
                rwy = A.rhow + ((int64_t)fy * A.nfmax + face_elem(A.mesh, ec, 1)) * NQ;
            if (GEN == 1 && enz < 0 && A.mesh.bc[fz] == 2)
                rwz = A.rhow + ((int64_t)fz * A.nfmax + face_elem(A.mesh, ec, 2)) * NQ;
        }
        // the wall densities of one direction's face points (1 where the face is not a wall)
        float rw[NQ];
        auto wall_rows = [&](const float *p) {
            if (GEN == 1 && p) {
#pragma unroll
                for (int k = 0; k < NQ; k++)
                    rw[k] = __ldg(p + k);
            } else {
#pragma unroll
                for (int k = 0; k < NQ; k++)
                    rw[k] = 1.f;
            }
        };
        // whether a direction's inflow face has an element behind it (else its ghost value); the trace
        // and the ghost jump are both formed and one is selected, so the line loops have no branch
        const bool inx = GEN == 0 || enx != -1, iny = GEN == 0 || eny >= 0, inz = GEN == 0 || enz >= 0;
        // x-lines (iy, iz): nodes j + N1 iy + NQ iz
        wait(2 + kx);
        wall_rows(rwx);
#pragma unroll
        for (int ln = 0; ln < NQ; ln++) {  // ln = iy + N1 iz, the line's face point
            float fl[N1], sv[N1], v[N1];
#pragma unroll
            for (int j = 0; j < N1; j++) {
                fl[j] = f[j + N1 * ln];
                v[j] = sm.sl[kx][j + N1 * ln][lane];
            }
            const float bx = gx * rw[ln];
            if (l0) {
                const float tj = trace_jump<N1, true>(v, fl[0], A.ops), gj = bx - fl[0];
                line_sums_jump<N1, true>(sv, fl, inx ? tj : gj, A.ops);
            } else {
                const float tj = trace_jump<N1, false>(v, fl[N1 - 1], A.ops), gj = bx - fl[N1 - 1];
                line_sums_jump<N1, false>(sv, fl, inx ? tj : gj, A.ops);
            }
#pragma unroll
            for (int j = 0; j < N1; j++)
                acc[j + N1 * ln] = fmaf(cx, sv[j], acc[j + N1 * ln]);
        }
        // y-lines (ix, iz): nodes ix + N1 j + NQ iz
        wait(2 + ky);
        wall_rows(rwy);
#pragma unroll
        for (int iz = 0; iz < N1; iz++)
#pragma unroll
            for (int ix = 0; ix < N1; ix++) {
                float fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = f[ix + N1 * j + NQ * iz];
                    v[j] = sm.sl[ky][ix + N1 * j + NQ * iz][lane];
                }
                const float by = gy * rw[ix + N1 * iz];
                if (l1) {
                    const float tj = trace_jump<N1, true>(v, fl[0], A.ops), gj = by - fl[0];
                    line_sums_jump<N1, true>(sv, fl, iny ? tj : gj, A.ops);
                } else {
                    const float tj = trace_jump<N1, false>(v, fl[N1 - 1], A.ops), gj = by - fl[N1 - 1];
                    line_sums_jump<N1, false>(sv, fl, iny ? tj : gj, A.ops);
                }
#pragma unroll
                for (int j = 0; j < N1; j++)
                    acc[ix + N1 * j + NQ * iz] = fmaf(cy, sv[j], acc[ix + N1 * j + NQ * iz]);
            }
        // slots kx and ky are consumed: the next tile's f^n and x-neighbour land there
        __syncwarp();
        if (more && ((lane == RFN && has_fn) || lane == RX)) {
            fence_proxy_async();
            issue_elem(lane == RX && OCT == 8 ? role_src(enn, (int)__ldg(A.toct + vt + 1)) : csrc, vl + 1,
                       lane == RX ? ky : kx);
        }
        // z-lines (ix, iy): nodes ix + N1 iy + NQ j
        wait(2 + ka);
        wall_rows(rwz);
#pragma unroll
        for (int q = 0; q < NQ; q++) {  // q = ix + N1 iy, the line's face point
            float fl[N1], sv[N1], v[N1];
#pragma unroll
            for (int j = 0; j < N1; j++) {
                fl[j] = f[q + NQ * j];
                v[j] = sm.sl[ka][q + NQ * j][lane];
            }
            const float bz = gz * rw[q];
            if (l2) {
                const float tj = trace_jump<N1, true>(v, fl[0], A.ops), gj = bz - fl[0];
                line_sums_jump<N1, true>(sv, fl, inz ? tj : gj, A.ops);
            } else {
                const float tj = trace_jump<N1, false>(v, fl[N1 - 1], A.ops), gj = bz - fl[N1 - 1];
                line_sums_jump<N1, false>(sv, fl, inz ? tj : gj, A.ops);
            }
#pragma unroll
            for (int j = 0; j < N1; j++)
                acc[q + NQ * j] = fmaf(cz, sv[j], acc[q + NQ * j]);
        }
        // BGK source towards the conservative Maxwellian, Shu-Osher combination (as k_stage3s)
        const float gm = sm.tab[b][3][lane] != 0.f ? 1.f : 0.f;
        const float cg = A.kg * gm, cf = bdt * gm;
        const float xs = x0 * x0 + x1 * x1 + x2 * x2;
        const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
        const bool iso = GEN != 1 || A.viso;
        const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
        const unsigned long long U0 = iso ? pack2(mms, mms) : pack2(mm0, mm0);
        const unsigned long long U1 = iso ? U0 : pack2(mm1, mm1);
        const unsigned long long U2 = iso ? 0ull : pack2(mm2, mm2);
        float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
        auto bgk_src = [&](auto vtau_c, auto force_c) {
            constexpr bool VT = decltype(vtau_c)::value, FP = decltype(force_c)::value;
#pragma unroll
            for (int h = 0; h < NH; h++) {
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];
                const unsigned long long lin =
                    ffma2(pack2(p23.z, p23.w), M2,
                          ffma2(pack2(p23.x, p23.y), M1, ffma2(pack2(p01.z, p01.w), M0, pack2(p01.x, p01.y))));
                const unsigned long long ex =
                    GEN == 1
                        ? ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U1, ffma2(pack2(p67.x, p67.y), U2, lin)))
                        : ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U0, lin));
                float g[2];
                exp2_fp32x2(ex, pack2(p67.z, p67.w), g[0], g[1]);
#pragma unroll
                for (int s2 = 0; s2 < 2; s2++) {
                    const int q = 2 * h + s2;
                    if (q >= NP)
                        break;
                    float gc = cg;
                    if constexpr (VT) {
                        const float itau = s2 == 0 ? p67.x : p67.y;
                        gc = __fsub_rn(A.b, __fsub_rn(A.b, __fmul_rn(bdt, itau))) * gm;
                    }
                    if constexpr (FP) {
                        const float4 fq = *reinterpret_cast<const float4 *>(&sm.fpar[q][0]);
                        const float qv = fmaf(sm.fpar[q][4], xs, fmaf(fq.w, x2, fmaf(fq.z, x1, fmaf(fq.y, x0, fq.x))));
                        gc = fmaf(cf, qv, gc);  // on top of the node's own Maxwellian weight
                    }
                    acc[q] = fmaf(gc, g[s2], acc[q]);  // the stage output
                }
            }
        };
        using T_ = std::true_type;
        using F_ = std::false_type;
        if constexpr (GEN == 1) {
            if (A.fpar)
                A.vtau ? bgk_src(T_{}, T_{}) : bgk_src(F_{}, T_{});
            else
                A.vtau ? bgk_src(T_{}, F_{}) : bgk_src(F_{}, F_{});
        } else {
            bgk_src(F_{}, F_{});
        }
        if (GEN && A.limiter) {
            // Zhang-Shu (Sec. 2.1, Eqs. 10-11): the element mean (tensor Gauss-Legendre weights) and
            // minimum of this velocity, all in this lane's registers, then the contraction
            float mean = 0.f, mn = acc[0];
#pragma unroll
            for (int iz = 0; iz < N1; iz++) {
                float lsum = 0.f;
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    lsum = fmaf(A.ops.wq[q % N1] * A.ops.wq[q / N1], acc[q + NQ * iz], lsum);
                    mn = fminf(mn, acc[q + NQ * iz]);
                }
                mean = fmaf(A.ops.wq[iz], lsum, mean);
            }
            if (mn < 0.f) {
                const float beta = fminf(fabsf(mean / (mean - mn)), 1.f);
#pragma unroll
                for (int q = 0; q < NP; q++)
                    acc[q] = fmaf(beta, acc[q] - mean, mean);
            }
        }
        __syncwarp();  // every lane's z-lines have read slot ka before it takes the output
#pragma unroll
        for (int q = 0; q < NP; q++) {
            __stcs(dst + q * kWarp, acc[q]);
            sm.sl[ka][q][lane ^ (4 * (q & 7))] = acc[q];  // for the moments below (slot ka is consumed)
        }
        // moments of the element's nodes (Eq. 2 with Eq. 12) of the stored values (rows np + 8 h)
        __syncwarp();
        unsigned long long pm[NHR][5];
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
                for (int d = 0; d < 3; d++) {  // W m_d: a power of two times an integer, exact
                    const float4 M4 = *reinterpret_cast<const float4 *>(&sm.tab[b][d][kk]);
                    wv[1 + d][0] = pack2(W4.x * M4.x, W4.y * M4.y);
                    wv[1 + d][1] = pack2(W4.z * M4.z, W4.w * M4.w);
                }
            }
#pragma unroll
            for (int h = 0; h < NHR; h++) {
                const int row = min(np + 8 * h, NP - 1);  // rows past the element: discarded below
                const float4 v = *reinterpret_cast<const float4 *>(&sm.sl[ka][row][kk ^ (4 * (row & 7))]);
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
        // slot ka is read: the next tile's y-neighbour lands there
        __syncwarp();
        if (lane == RY && more) {
            fence_proxy_async();
            issue_elem(OCT < 8 ? csrc : role_src(enn, (int)__ldg(A.toct + vt + 1)), vl + 1, ka);
        }
#pragma unroll
        for (int d = 0; d < 3; d++)
            en[d] = enn[d];
        ka = ka == 2 ? 0 : ka + 1;
    }
    // partial moments of this task: combine the 4 velocity eighths of every row
    const int grp = A.group0 + gl;
#pragma unroll
    for (int h = 0; h < NHR; h++) {
        const int q = np + 8 * h;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            float x = msum[h][c];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (kg == 0 && q < NP)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)e * NP + q] = x;
        }
    }
}

template <int N1, int OCT, int GEN>
cudaError_t launch3w(const StageArgs &A, cudaStream_t s)
{
    const int ngroups = (A.nvt + A.G - 1) / A.G;
    const int nblk = (A.mesh.nelem + BGK_STAGE3W_WARPS - 1) / BGK_STAGE3W_WARPS;
    k_stage3w<N1, OCT, GEN><<<nblk * ngroups, kWarp * BGK_STAGE3W_WARPS,
                              BGK_STAGE3W_WARPS * sizeof(Stage3wWarp<N1, GEN>), s>>>(A);
    return cudaGetLastError();
}

template <int N1>
cudaError_t prepare3w()
{
    const int s0 = BGK_STAGE3W_WARPS * (int)sizeof(Stage3wWarp<N1, 0>);
    const int s1 = BGK_STAGE3W_WARPS * (int)sizeof(Stage3wWarp<N1, 1>);
    const int s2 = BGK_STAGE3W_WARPS * (int)sizeof(Stage3wWarp<N1, 2>);
    cudaError_t e = cudaSuccess;
#define BGK_P3W(O)                                                                                       \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_stage3w<N1, O, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0); \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_stage3w<N1, O, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1); \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_stage3w<N1, O, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
    BGK_P3W(0) BGK_P3W(1) BGK_P3W(2) BGK_P3W(3) BGK_P3W(4) BGK_P3W(5) BGK_P3W(6) BGK_P3W(7) BGK_P3W(8)
#undef BGK_P3W
    return e;
}

template <int N1, int GEN>
cudaError_t launch3w_oct(const StageArgs &A, int oct, cudaStream_t s)
{
    switch (oct) {
    case 0: return launch3w<N1, 0, GEN>(A, s);
    case 1: return launch3w<N1, 1, GEN>(A, s);
    case 2: return launch3w<N1, 2, GEN>(A, s);
    case 3: return launch3w<N1, 3, GEN>(A, s);
    case 4: return launch3w<N1, 4, GEN>(A, s);
    case 5: return launch3w<N1, 5, GEN>(A, s);
    case 6: return launch3w<N1, 6, GEN>(A, s);
    case 7: return launch3w<N1, 7, GEN>(A, s);
    default: return launch3w<N1, 8, GEN>(A, s);
    }
}

}  // namespace bgk
