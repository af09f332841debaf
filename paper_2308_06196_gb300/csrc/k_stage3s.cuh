// k_stage3s.cuh -- the fused SSP-RK3 stage kernel for affine hexahedra (FP32-split form) with every
// operand staged in shared memory by bulk asynchronous copies; instantiated per degree in
// k_stage3_p*.cu.
#pragma once
#include <type_traits>

#include "stage_common.cuh"

#ifndef BGK_STAGE3S_MINCTAS_P3
#define BGK_STAGE3S_MINCTAS_P3 5
#endif
#ifndef BGK_STAGE3S_MINCTAS_P3_GEN
#define BGK_STAGE3S_MINCTAS_P3_GEN 4
#endif
#ifndef BGK_STAGE3S_MINCTAS_P2
#define BGK_STAGE3S_MINCTAS_P2 8
#endif

namespace bgk {

// ------------------------------------------------------------------------------------------------
// One CTA per (element, run of G velocity tiles), one warp per z-layer of the element's nodes, lane =
// velocity of the tile (as k_stage3). Every warp streams its own rows through shared memory with
// bulk asynchronous copies issued by its lane 0 and completed on the warp's own mbarriers:
//   fs[b]  its layer of f_s, double-buffered (the next tile's layer is in flight while this one is
//          used); the z-lines read the other layers' rows after the first block barrier and write
//          their derivative sums back over the rows they read (the tile is consumed by then); the
//          stage output of the layer is then transposed through its own rows for the moment sums;
//   sl[3]  three rotating slots of one layer each for the operands read once per tile: at tile t
//          slot t mod 3 holds f^n (read first), slot t+1 the x-upwind neighbour's layer and slot t+2
//          the y-upwind neighbour's; each slot is refilled as soon as it is consumed -- with the z-upwind
//          neighbour's rows of the warp's z-line slice (read by the z-lines), the next tile's f^n, x- and
//          y-neighbour layer -- so every copy is issued between a third and all of a tile ahead.
// Warp 0 also brings the tile's velocity tables (grid indices, padding mask, moment weights) into a
// double-buffered block with a barrier of its own, which every warp waits on; it issues them after the
// previous tile's first block barrier, once every warp is done with the buffer's old contents. The neighbour lines thus come
// from shared memory instead of per-lane loads from L2 into registers, no global load is left in the
// tile loop of the periodic form, and the running moment sums stay in registers.
// ------------------------------------------------------------------------------------------------
// velocity table rows per tile: the grid indices m_x, m_y, m_z, the index-basis weight W (0 on padded
// slots) and the energy weight W sum_d r_d m_d^2; the moment weights W m_d are formed from them (exact)
constexpr int kTabRows = 5;

template <int N1, int GEN>
struct Stage3sSmem {
    static constexpr int NP = N1 * N1 * N1, NQ = N1 * N1;
    float fs[2][NP][kWarp];
    float sl[N1][3][NQ][kWarp];
    float tab[2][kTabRows][kWarp];
    float par[N1][(NQ + 1) / 2][kParamStride][2];  // BGK exponents by layer and node pair (see k_stage3)
    float fpar[GEN ? NP : 1][GEN ? kParamStride : 1];
    float lim[GEN ? 2 : 1][GEN ? N1 : 1][GEN ? kWarp : 1];
    unsigned long long bar[N1][5];  // per warp: fs[0], fs[1], sl[0..2]
    unsigned long long tbar[2];     // the velocity tables' buffers
};

template <int N1, int OCT, int GEN>
__global__ void __launch_bounds__(kWarp *N1, (N1 >= 4 ? (GEN ? BGK_STAGE3S_MINCTAS_P3_GEN : BGK_STAGE3S_MINCTAS_P3)
                                               : (N1 == 3 ? BGK_STAGE3S_MINCTAS_P2 : 8))) k_stage3s(const StageArgs A)
{
    constexpr int NQ = N1 * N1;
    constexpr int NP = NQ * N1;
    constexpr int NT = kWarp * N1;
    constexpr uint32_t kRow = kWarp * sizeof(float);  // one node's row of a tile: 128 bytes
    using Sm = Stage3sSmem<N1, GEN>;
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

    // per-point BGK exponents (and force polynomials) of the element, as k_stage3
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
    }
    // barrier addresses: bar(i) = fs[0], fs[1], sl[0], sl[1], sl[2] of this warp; tbar(b) the tables'
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
    __syncthreads();  // exponents and barriers visible to every warp

    const bool has_fn = A.fn != nullptr;
    // upwind neighbours of tile vl (one-octant launches: the same for the whole task), -1 on a
    // Dirichlet or wall face
    auto nbrs = [&](int vl, int (&en)[3]) {
        const int oct = OCT < 8 ? OCT : (int)__ldg(A.toct + A.vt0 + vl);
#pragma unroll
        for (int d = 0; d < 3; d++)
            en[d] = upwind_neighbour(A.mesh, ec, d, ((oct >> d) & 1) != 0);
    };
    // Bulk copies. Each copy of a tile has a role lane, so that the copies of one issue point cost the
    // warp one short code path: lane 0 the warp's f_s layer, lanes RZ .. RZ + N1 - 1 the z-upwind
    // neighbour's row groups j = lane - RZ of the warp's z-line slice (rows ix + N1 w + NQ j, landing as
    // ix + N1 j), lane RFN the warp's layer of f^n, lanes RX and RY the x- and y-upwind neighbours' layer
    // w; lane RT of warp 0 the tile's velocity table. A role lane keeps the source of its copy at
    // tile 0 and adds the tile stride; a boundary face (no neighbour) gives only the barrier's arrival.
    // Across an exchange face the x-upwind neighbour is the element of the face's halo (the neighbouring
    // subdomain's layer, [tile][face element][node][lane]), whose tiles are eface elements apart.
    constexpr int RZ = 1, RFN = N1 + 1, RX = N1 + 2, RY = N1 + 3, RT = N1 + 4;
    const int64_t tstride = (int64_t)E * NP * kWarp;  // floats between consecutive tiles of one element
    const int64_t hstride = (int64_t)A.eface * NP * kWarp;
    int64_t cstride = tstride;  // this lane's stride (hstride for a halo source)
    auto role_src = [&](const int (&en)[3], int oct) -> const float * {
        cstride = tstride;
        if (lane == RX && en[0] == kHaloNeighbour) {
            cstride = hstride;
            const int64_t r = ec[1] + (int64_t)A.mesh.ne[1] * ec[2];
            return A.halo[(oct & 1) ? 0 : 1] + (((int64_t)A.vt0 * A.eface + r) * NP + NQ * w) * kWarp;
        }
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
    // one layer (or nothing, at a boundary) into slot k of this warp, from csrc at tile vl (role lane only)
    auto issue_layer = [&](const float *csrc, int vl, int k) {
        const uint32_t bb = bar(2 + k);
        mbar_arrive_expect_tx(bb, csrc ? kSlot : 0);
        if (csrc)
            bulk_g2s(sl0 + k * kSlot, csrc + vl * cstride, kSlot, bb);
    };

    int en[3];
    nbrs(vl0, en);
    const float *csrc = role_src(en, OCT < 8 ? OCT : (int)__ldg(A.toct + A.vt0 + vl0));  // at tile 0
    if (lane == 0) {
        mbar_arrive_expect_tx(bar(0), kSlot);
        bulk_g2s(fs0, csrc + vl0 * tstride, kSlot, bar(0));
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
    uint32_t ph = 0;  // phase parity of every barrier, bit i for bar[i], bit 5 + b for tbar(b)
    auto wait = [&](int i) {
        mbar_wait(bar(i), (ph >> i) & 1, A.err);
        ph ^= 1u << i;
    };

    // moment sums: lane = (node pair np = lane / 4: layer nodes np and np + 8) x (velocity eighth
    // kg = lane % 4), as k_stage3, running in registers
    const int np = lane >> 2, kg = lane & 3;
    constexpr int NHR = NQ > 8 ? 2 : 1;
    float msum[NHR][5];
#pragma unroll
    for (int h = 0; h < NHR; h++)
#pragma unroll
        for (int c = 0; c < 5; c++)
            msum[h][c] = 0.f;
    const float kb = A.kb;
    const float bdt = A.b * A.dt;

    int ka = 0;  // slot of f^n in this tile; the x- and y-neighbour layers are in slots ka + 1, ka + 2
    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const int b = (vl - vl0) & 1;
        const int kx = ka == 2 ? 0 : ka + 1, ky = ka == 0 ? 2 : ka - 1;
        int enn[3] = {en[0], en[1], en[2]};  // the next tile's neighbours
        if (OCT == 8 && vl + 1 < vl1)
            nbrs(vl + 1, enn);
        const bool more = vl + 1 < vl1;
        const int oct = OCT < 8 ? OCT : (int)__ldg(A.toct + vt);
        const bool l0 = (oct & 1) != 0, l1 = (oct & 2) != 0, l2 = (oct & 4) != 0;
        const int enx = en[0], eny = en[1], enz = en[2];

        wait(b);
        mbar_wait(tbar(b), (ph >> (5 + b)) & 1, A.err);
        ph ^= 1u << (5 + b);
        const float m0 = sm.tab[b][0][lane], m1 = sm.tab[b][1][lane], m2 = sm.tab[b][2][lane];
        const float x0 = fmaf(A.vs[0], m0, A.vc[0]), x1 = fmaf(A.vs[1], m1, A.vc[1]), x2 = fmaf(A.vs[2], m2, A.vc[2]);
        float f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++)
            f[q] = sm.fs[b][q + NQ * w][lane];
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
            const float *zs = OCT < 8 ? csrc : role_src(en, oct);
            const uint32_t bb = bar(2 + ka);
            fence_proxy_async();
            if (lane == RZ)
                mbar_arrive_expect_tx(bb, zs ? kSlot : 0);
            if (zs)
                bulk_g2s(sl0 + ka * kSlot + (lane - RZ) * N1 * kRow, zs + vl * tstride, N1 * kRow, bb);
        }
        // acc = an f^n + b (1 - dt/tau) f_s, then x and y lines
        // (launch-uniform feature tests sit outside the unrolled node loops, which stay one basic block)
        if (GEN && A.vtau) {  // variable collision time: b (1 - dt/tau) of every node
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = fmaf(A.an, acc[q], __fsub_rn(A.b, __fmul_rn(bdt, sm.par[w][q / 2][6][q % 2])) * f[q]);
        } else {
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = fmaf(A.an, acc[q], kb * f[q]);
        }
        const float cx = -A.mesh.inv_h2[0] * x0 * bdt, cy = -A.mesh.inv_h2[1] * x1 * bdt;
        const float cz = -A.mesh.inv_h2[2] * x2 * bdt;
        // upwind value on a non-periodic face: the Dirichlet ghost Maxwellian, or the diffuse-wall
        // Maxwellian scaled by the wall density of the face point (face point of every line of this
        // warp: its index + N1 * w)
        const int fx = 0 + (l0 ? 0 : 1), fy = 2 + (l1 ? 0 : 1), fz = 4 + (l2 ? 0 : 1);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        const float *rwx = nullptr, *rwy = nullptr, *rwz = nullptr;
        if (GEN) {
            gx = enx != -1 ? 0.f : __ldg(A.ghost + fx * A.nslots + slot);
            gy = eny >= 0 ? 0.f : __ldg(A.ghost + fy * A.nslots + slot);
            gz = enz >= 0 ? 0.f : __ldg(A.ghost + fz * A.nslots + slot);
            if (enx < 0 && A.mesh.bc[fx] == 2)
                rwx = A.rhow + ((int64_t)fx * A.nfmax + face_elem(A.mesh, ec, 0)) * NQ + N1 * w;
            if (eny < 0 && A.mesh.bc[fy] == 2)
                rwy = A.rhow + ((int64_t)fy * A.nfmax + face_elem(A.mesh, ec, 1)) * NQ + N1 * w;
            if (enz < 0 && A.mesh.bc[fz] == 2)
                rwz = A.rhow + ((int64_t)fz * A.nfmax + face_elem(A.mesh, ec, 2)) * NQ + N1 * w;
        }
        // the wall densities of a direction's face points of this warp's lines (1 off a wall face)
        float rw[N1];
        auto wall_rows = [&](const float *p) {
            if (GEN && p) {
#pragma unroll
                for (int k = 0; k < N1; k++)
                    rw[k] = __ldg(p + k);
            } else {
#pragma unroll
                for (int k = 0; k < N1; k++)
                    rw[k] = 1.f;
            }
        };
        // The three line directions. Where the upwind neighbour of the line ends is an element (not a
        // Dirichlet or wall ghost) and N1 is even, two adjacent lines run at a time on packed pairs.
        constexpr bool kPair = N1 % 2 == 0;
        wait(2 + kx);
        if (kPair && (GEN == 0 || enx != -1)) {
#pragma unroll
            for (int iy = 0; iy < N1; iy += 2) {
                unsigned long long fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = pack2(f[j + N1 * iy], f[j + N1 * iy + N1]);
                    v[j] = pack2(sm.sl[w][kx][j + N1 * iy][lane], sm.sl[w][kx][j + N1 * iy + N1][lane]);
                }
                if (l0)
                    line_sums_jump2<N1, true>(sv, fl, trace_jump2<N1, true>(v, fl[0], A.ops), A.ops);
                else
                    line_sums_jump2<N1, false>(sv, fl, trace_jump2<N1, false>(v, fl[N1 - 1], A.ops), A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    float lo, hi;
                    unpack2(sv[j], lo, hi);
                    acc[j + N1 * iy] = fmaf(cx, lo, acc[j + N1 * iy]);
                    acc[j + N1 * iy + N1] = fmaf(cx, hi, acc[j + N1 * iy + N1]);
                }
            }
        } else {
            wall_rows(rwx);
#pragma unroll
            for (int iy = 0; iy < N1; iy++) {
                float fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = f[j + N1 * iy];
                    v[j] = sm.sl[w][kx][j + N1 * iy][lane];
                }
                const float bx = gx * rw[iy];
                if (l0)
                    line_sums_jump<N1, true>(sv, fl, enx != -1 ? trace_jump<N1, true>(v, fl[0], A.ops) : bx - fl[0],
                                             A.ops);
                else
                    line_sums_jump<N1, false>(sv, fl,
                                              enx != -1 ? trace_jump<N1, false>(v, fl[N1 - 1], A.ops) : bx - fl[N1 - 1],
                                              A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    acc[j + N1 * iy] = fmaf(cx, sv[j], acc[j + N1 * iy]);
            }
        }
        wait(2 + ky);
        if (kPair && (GEN == 0 || eny >= 0)) {
#pragma unroll
            for (int ix = 0; ix < N1; ix += 2) {
                unsigned long long fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = pack2(f[ix + N1 * j], f[ix + 1 + N1 * j]);
                    v[j] = pack2(sm.sl[w][ky][ix + N1 * j][lane], sm.sl[w][ky][ix + 1 + N1 * j][lane]);
                }
                if (l1)
                    line_sums_jump2<N1, true>(sv, fl, trace_jump2<N1, true>(v, fl[0], A.ops), A.ops);
                else
                    line_sums_jump2<N1, false>(sv, fl, trace_jump2<N1, false>(v, fl[N1 - 1], A.ops), A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    float lo, hi;
                    unpack2(sv[j], lo, hi);
                    acc[ix + N1 * j] = fmaf(cy, lo, acc[ix + N1 * j]);
                    acc[ix + 1 + N1 * j] = fmaf(cy, hi, acc[ix + 1 + N1 * j]);
                }
            }
        } else {
            wall_rows(rwy);
#pragma unroll
            for (int ix = 0; ix < N1; ix++) {
                float fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = f[ix + N1 * j];
                    v[j] = sm.sl[w][ky][ix + N1 * j][lane];
                }
                const float by = gy * rw[ix];
                if (l1)
                    line_sums_jump<N1, true>(sv, fl, eny >= 0 ? trace_jump<N1, true>(v, fl[0], A.ops) : by - fl[0],
                                             A.ops);
                else
                    line_sums_jump<N1, false>(sv, fl,
                                              eny >= 0 ? trace_jump<N1, false>(v, fl[N1 - 1], A.ops) : by - fl[N1 - 1],
                                              A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    acc[ix + N1 * j] = fmaf(cy, sv[j], acc[ix + N1 * j]);
            }
        }
        // slots kx and ky are consumed: the next tile's f^n and x-neighbour layer land there
        // and the next tile's f_s layer into the other buffer, whose rows were last read and written
        // before the previous tile's B2 (the z-lines) and by this warp's own moment pass: one code path
        // for the three role lanes
        __syncwarp();
        if (more && (lane == 0 || (lane == RFN && has_fn) || lane == RX)) {
            const float *ns = lane == RX && OCT == 8 ? role_src(enn, (int)__ldg(A.toct + vt + 1)) : csrc;
            const int k = lane == RX ? ky : kx;
            const uint32_t bb = lane == 0 ? bar(b ^ 1) : bar(2 + k);
            const uint32_t dst = lane == 0 ? fs0 + (b ^ 1) * kFsBuf : sl0 + k * kSlot;
            fence_proxy_async();
            mbar_arrive_expect_tx(bb, ns ? kSlot : 0);
            if (ns)
                bulk_g2s(dst, ns + (vl + 1) * cstride, kSlot, bb);
        }
        __syncthreads();  // B1: every layer of the element tile has landed (each warp waited for its own)
        // z-lines of slice iy = w (all layers) from the shared tile, the upwind trace from the staged
        // neighbour rows; each line's derivative sums overwrite the rows it read
        wait(2 + ka);
        if (kPair && (GEN == 0 || enz >= 0)) {
#pragma unroll
            for (int ix = 0; ix < N1; ix += 2) {
                const int q = ix + N1 * w;
                unsigned long long fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = pack2(sm.fs[b][q + NQ * j][lane], sm.fs[b][q + 1 + NQ * j][lane]);
                    v[j] = pack2(sm.sl[w][ka][ix + N1 * j][lane], sm.sl[w][ka][ix + 1 + N1 * j][lane]);
                }
                if (l2)
                    line_sums_jump2<N1, true>(sv, fl, trace_jump2<N1, true>(v, fl[0], A.ops), A.ops);
                else
                    line_sums_jump2<N1, false>(sv, fl, trace_jump2<N1, false>(v, fl[N1 - 1], A.ops), A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    float lo, hi;
                    unpack2(sv[j], lo, hi);
                    sm.fs[b][q + NQ * j][lane] = lo;
                    sm.fs[b][q + 1 + NQ * j][lane] = hi;
                }
            }
        } else {
            wall_rows(rwz);
#pragma unroll
            for (int ix = 0; ix < N1; ix++) {
                const int q = ix + N1 * w;
                float fl[N1], sv[N1], v[N1];
#pragma unroll
                for (int j = 0; j < N1; j++) {
                    fl[j] = sm.fs[b][q + NQ * j][lane];
                    v[j] = sm.sl[w][ka][ix + N1 * j][lane];
                }
                const float bz = gz * rw[ix];
                if (l2)
                    line_sums_jump<N1, true>(sv, fl, enz >= 0 ? trace_jump<N1, true>(v, fl[0], A.ops) : bz - fl[0],
                                             A.ops);
                else
                    line_sums_jump<N1, false>(sv, fl,
                                              enz >= 0 ? trace_jump<N1, false>(v, fl[N1 - 1], A.ops) : bz - fl[N1 - 1],
                                              A.ops);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    sm.fs[b][q + NQ * j][lane] = sv[j];
            }
        }
        // slot ka is consumed: the next tile's y-neighbour layer lands there; warp 0 also brings the next
        // tile's velocity table into the other table buffer, which every warp is done with (B1)
        __syncwarp();
        if (more && (lane == RY || (w == 0 && lane == RT))) {  // one code path for both role lanes
            const bool t = lane == RT;
            const float *ys = t ? nullptr : (OCT < 8 ? csrc : role_src(enn, (int)__ldg(A.toct + vt + 1)));
            const float *ns = t ? A.vtab + (int64_t)(vt + 1) * kTabRows * kWarp : (ys ? ys + (vl + 1) * cstride : nullptr);
            const uint32_t bb = t ? tbar(b ^ 1) : bar(2 + ka);
            const uint32_t dst = t ? smem_u32(&sm.tab[b ^ 1][0][0]) : sl0 + ka * kSlot;
            const uint32_t bytes = t ? kTabRows * kRow : kSlot;
            fence_proxy_async();
            mbar_arrive_expect_tx(bb, ns ? bytes : 0);
            if (ns)
                bulk_g2s(dst, ns, bytes, bb);
        }
        __syncthreads();  // B2: z-sums complete
#pragma unroll
        for (int q = 0; q < NQ; q++)
            acc[q] = fmaf(cz, sm.fs[b][q + NQ * w][lane], acc[q]);
        __syncwarp();  // the z-sums of this layer are read before its rows take the stage output
        // BGK source towards the conservative Maxwellian, Shu-Osher combination, store (as k_stage3)
        const float gm = sm.tab[b][3][lane] != 0.f ? 1.f : 0.f;  // the padding mask
        const float cg = A.kg * gm, cf = bdt * gm;
        const float xs = x0 * x0 + x1 * x1 + x2 * x2;
        const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
        const bool iso = !GEN || A.viso;
        const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
        const unsigned long long U0 = iso ? pack2(mms, mms) : pack2(mm0, mm0);
        const unsigned long long U1 = iso ? U0 : pack2(mm1, mm1);
        const unsigned long long U2 = iso ? 0ull : pack2(mm2, mm2);
        float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
        float lsum = 0.f, lmin = 3.4e38f;  // limiter: this layer's weighted sum and minimum
        auto bgk_src = [&](auto vtau_c, auto force_c, auto lim_c) {
            constexpr bool VT = decltype(vtau_c)::value, FP = decltype(force_c)::value;
            constexpr bool LIM = decltype(lim_c)::value;
#pragma unroll
            for (int h = 0; h < (NQ + 1) / 2; h++) {
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[w][h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];  // (c, c+1) of both nodes
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
                    if constexpr (VT) {  // kg = b - kb exactly, kb as in the accumulator above
                        const float itau = sl == 0 ? p67.x : p67.y;
                        gc = __fsub_rn(A.b, __fsub_rn(A.b, __fmul_rn(bdt, itau))) * gm;
                    }
                    if constexpr (FP) {  // body-force source g (q0 + q . xi + q4 |xi|^2)
                        const float4 fq = *reinterpret_cast<const float4 *>(&sm.fpar[i][0]);
                        const float qv =
                            fmaf(sm.fpar[i][4], xs, fmaf(fq.w, x2, fmaf(fq.z, x1, fmaf(fq.y, x0, fq.x))));
                        gc = fmaf(cf, qv, gc);  // on top of the node's own Maxwellian weight
                    }
                    const float o = fmaf(gc, g[sl], a);
                    if constexpr (LIM) {  // stored after the limiter below
                        lsum = fmaf(A.ops.wq[q % N1] * A.ops.wq[q / N1], o, lsum);
                        lmin = fminf(lmin, o);
                    } else {
                        __stcs(dst + i * kWarp, o);
                    }
                    sm.fs[b][q + NQ * w][lane ^ (4 * (q & 7))] = o;  // for the moments below
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
            // Zhang-Shu (Sec. 2.1, Eqs. 10-11): element mean and minimum of every velocity over the
            // layers, then the contraction of the values of this warp's layer
            sm.lim[0][w][lane] = A.ops.wq[w] * lsum;
            sm.lim[1][w][lane] = lmin;
            __syncthreads();  // B3 (the general form only)
            float mean = 0.f, mn = sm.lim[1][0][lane];
#pragma unroll
            for (int lw = 0; lw < N1; lw++) {
                mean += sm.lim[0][lw][lane];
                mn = fminf(mn, sm.lim[1][lw][lane]);
            }
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
                    wv[1 + d][0] = fmul2(pack2(W4.x, W4.y), pack2(M4.x, M4.y));
                    wv[1 + d][1] = fmul2(pack2(W4.z, W4.w), pack2(M4.z, M4.w));
                }
            }
#pragma unroll
            for (int h = 0; h < NHR; h++) {
                const int row = min(np + 8 * h, NQ - 1);  // rows past the layer: discarded below
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
        ka = ka == 2 ? 0 : ka + 1;
    }
    // partial moments of this task: combine the 4 velocity eighths of every node pair
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

template <int N1, int OCT, int GEN>
cudaError_t launch3s(const StageArgs &A, cudaStream_t s)
{
    const int ngroups = (A.nvt + A.G - 1) / A.G;
    k_stage3s<N1, OCT, GEN><<<A.mesh.nelem * ngroups, kWarp * N1, sizeof(Stage3sSmem<N1, GEN>), s>>>(A);
    return cudaGetLastError();
}

template <int N1>
cudaError_t prepare3s()
{
    const int s0 = (int)sizeof(Stage3sSmem<N1, 0>), s1 = (int)sizeof(Stage3sSmem<N1, 1>);
    cudaError_t e = cudaSuccess;
#define BGK_P3S(O)                                                                                       \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_stage3s<N1, O, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0); \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_stage3s<N1, O, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
    BGK_P3S(0) BGK_P3S(1) BGK_P3S(2) BGK_P3S(3) BGK_P3S(4) BGK_P3S(5) BGK_P3S(6) BGK_P3S(7) BGK_P3S(8)
#undef BGK_P3S
    return e;
}

template <int N1, int GEN>
cudaError_t launch3s_oct(const StageArgs &A, int oct, cudaStream_t s)
{
    switch (oct) {
    case 0: return launch3s<N1, 0, GEN>(A, s);
    case 1: return launch3s<N1, 1, GEN>(A, s);
    case 2: return launch3s<N1, 2, GEN>(A, s);
    case 3: return launch3s<N1, 3, GEN>(A, s);
    case 4: return launch3s<N1, 4, GEN>(A, s);
    case 5: return launch3s<N1, 5, GEN>(A, s);
    case 6: return launch3s<N1, 6, GEN>(A, s);
    case 7: return launch3s<N1, 7, GEN>(A, s);
    default: return launch3s<N1, 8, GEN>(A, s);
    }
}

}  // namespace bgk
