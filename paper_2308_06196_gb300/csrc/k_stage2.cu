// k_stage2.cu -- the fused SSP-RK3 stage kernel for quadrilaterals (dim = 2, FP32-split form): the
// planar problems of the method (Sec. 2 with d = 2, velocity dimension m = 2 or 3).
//
// One CTA per (block of 4 elements, run of G tiles); warp w owns element 4 b + w and works alone (no
// block barrier): lane l owns velocity l of the tile and keeps the element's N1^2 values in registers,
// so both the x and the y derivatives are register-local. The element's f_s rows are double-buffered
// in shared memory with cp.async one tile ahead, f^n is refilled after use; the upwind neighbours'
// lines come from L2. The Maxwellian, the Shu-Osher combination, the positivity limiter (in registers:
// the element is the warp's) and the moment sums of the stored output follow as in the hexahedral kernel.
#include "stage_common.cuh"

namespace bgk {

template <int N1>
struct alignas(16) QuadSmem {
    static constexpr int NQ = N1 * N1;
    float tile[2][NQ][kWarp];                  // f_s of the element, [node][lane] (cp.async)
    float fnb[NQ][kWarp];                      // f^n of the element
    float msum[10][kWarp];                     // running moment sums: 2 nodes x 5 moments per lane
    float par[(NQ + 1) / 2][kParamStride][2];  // BGK exponents by node pair (as the hexahedral kernel)
    float wpsi[5][kWarp];                      // w psi of the tile's velocities
};

// Resident CTAs per SM the register allocation is sized for: 5 (96 registers); 6 (80 registers, a few
// bytes of spills) runs 3 % slower on the planar Taylor-Green quadrilaterals.
#ifndef BGK_STAGE2_MINCTAS
#define BGK_STAGE2_MINCTAS 5
#endif

template <int N1, int MODE, int OCT>
__global__ void __launch_bounds__(kWarp *kWarpsPerCta, BGK_STAGE2_MINCTAS) k_stage2(const StageArgs A)
{
    constexpr int NQ = N1 * N1;
    constexpr int NCH = NQ * kWarp / 4;  // 16-byte chunks of one element tile
    __shared__ QuadSmem<N1> smw[kWarpsPerCta];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int E = A.mesh.nelem;
    const int EB = (E + kWarpsPerCta - 1) / kWarpsPerCta;
    const int gl = blockIdx.x / EB;
    const int e = (blockIdx.x % EB) * kWarpsPerCta + w;
    if (e >= E)
        return;  // the warps of a CTA never wait for one another
    QuadSmem<N1> &sm = smw[w];
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    const int ec[3] = {e % A.mesh.ne[0], e / A.mesh.ne[0], 0};

    if (MODE == 0) {
        constexpr int NH = (NQ + 1) / 2;
        const float *src = A.param + (int64_t)e * NQ * kParamStride;
        for (int q = lane; q < NH * 2 * kParamStride; q += kWarp) {
            const int c = q % kParamStride, sl = (q / kParamStride) & 1, h = q / (2 * kParamStride);
            sm.par[h][c][sl] = __ldg(src + min(2 * h + sl, NQ - 1) * kParamStride + c);
        }
    }
    const int np = lane >> 2, kg = lane & 3;  // moment sums: node pair (np, np + 8) x velocity eighth
#pragma unroll
    for (int m = 0; m < 10; m++)
        sm.msum[m][lane] = 0.f;
    const float kb = A.kb;
    const float bdt = A.b * A.dt;
    const bool has_fn = MODE == 0 && A.fn != nullptr;

    auto prefetch = [&](int vl, int b) {
        const float4 *gs = reinterpret_cast<const float4 *>(A.src + fidx(vl, e, 0, 0, E, NQ));
        float4 *ss = reinterpret_cast<float4 *>(&sm.tile[b][0][0]);
        for (int m = lane; m < NCH; m += kWarp)
            cp_async16(ss + m, gs + m);
        cp_commit();
    };
    auto prefetch_fn = [&](int vl) {
        if (has_fn) {
            const float4 *gf = reinterpret_cast<const float4 *>(A.fn + fidx(vl, e, 0, 0, E, NQ));
            float4 *sf = reinterpret_cast<float4 *>(&sm.fnb[0][0]);
            for (int m = lane; m < NCH; m += kWarp)
                cp_async16(sf + m, gf + m);
        }
        cp_commit();
    };
    prefetch(vl0, 0);
    prefetch_fn(vl0);
    __syncwarp();  // the parameter rows of every lane

    // the tile's velocity rows (w psi, grid indices, mask) are loaded one tile ahead into registers
    float wp_n[5], mi_n[3], gm_n = 0.f;
    auto load_rows = [&](int vt) {
        const int sl = vt * kWarp + lane;
#pragma unroll
        for (int c = 0; c < 5; c++)
            wp_n[c] = __ldg(A.wpsi + ((int64_t)vt * 5 + c) * kWarp + lane);
        if (MODE == 0) {
#pragma unroll
            for (int d = 0; d < 3; d++)
                mi_n[d] = __ldg(A.mi + d * A.nslots + sl);
            gm_n = __ldg(A.gmask + sl);
        }
    };
    if (vl0 < vl1)
        load_rows(A.vt0 + vl0);
    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        const int b = (vl - vl0) & 1;
        float wp_c[5], mi_c[3];
#pragma unroll
        for (int c = 0; c < 5; c++)
            wp_c[c] = wp_n[c];
#pragma unroll
        for (int d = 0; d < 3; d++)
            mi_c[d] = mi_n[d];
        const float gm_c = gm_n;
        if (vl + 1 < vl1)
            load_rows(vt + 1);
        if (vl + 1 < vl1) {  // pending: tile vl, f^n vl, then tile vl + 1
            prefetch(vl + 1, b ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 5; c++)
            sm.wpsi[c][lane] = wp_c[c];
        float f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++)
            f[q] = sm.tile[b][q][lane];
        if (MODE == 0) {
            const float m0 = mi_c[0], m1 = mi_c[1], m2 = mi_c[2];
            const float x0 = fmaf(A.vs[0], m0, A.vc[0]), x1 = fmaf(A.vs[1], m1, A.vc[1]);
            const bool l0 = OCT < 8 ? (OCT & 1) != 0 : x0 >= 0.f;
            const bool l1 = OCT < 8 ? (OCT & 2) != 0 : x1 >= 0.f;
            float acc[NQ];
#pragma unroll
            for (int q = 0; q < NQ; q++)
                acc[q] = has_fn ? sm.fnb[q][lane] : 0.f;
            __syncwarp();
            if (vl + 1 < vl1)
                prefetch_fn(vl + 1);
            else
                cp_commit();
            // upwind neighbours (or the face's ghost) in x and y
            const int enx = upwind_neighbour(A.mesh, ec, 0, l0), eny = upwind_neighbour(A.mesh, ec, 1, l1);
            float vx[N1][N1], vy[N1][N1];
            {  // (a boundary face: zeros, whose trace is discarded below)
                const float *nb = A.src + fidx(vl, max(enx, 0), 0, lane, E, NQ);
#pragma unroll
                for (int iy = 0; iy < N1; iy++)
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        vx[iy][j] = enx >= 0 ? __ldg(nb + (j + N1 * iy) * kWarp) : 0.f;
            }
            {
                const float *nb = A.src + fidx(vl, max(eny, 0), 0, lane, E, NQ);
#pragma unroll
                for (int ix = 0; ix < N1; ix++)
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        vy[ix][j] = eny >= 0 ? __ldg(nb + (ix + N1 * j) * kWarp) : 0.f;
            }
            const float gx = enx >= 0 ? 0.f : __ldg(A.ghost + (l0 ? 0 : 1) * A.nslots + slot);
            const float gy = eny >= 0 ? 0.f : __ldg(A.ghost + (l1 ? 2 : 3) * A.nslots + slot);
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                float kbq = kb;
                if (A.vtau)  // variable collision time: b (1 - dt/tau) of this node
                    kbq = __fsub_rn(A.b, __fmul_rn(bdt, sm.par[q / 2][6][q % 2]));
                acc[q] = fmaf(A.an, acc[q], kbq * f[q]);
            }
            const float cx = -A.mesh.inv_h2[0] * x0 * bdt, cy = -A.mesh.inv_h2[1] * x1 * bdt;
            if constexpr (N1 % 2 == 0) {
                // two adjacent lines of a direction at a time on packed FP32 pairs, the upwind value in
                // jump form inside the trace (as the hexahedral kernels), selected against the ghost jump
                constexpr int RL = 0, RR = N1 - 1;
#pragma unroll
                for (int iy = 0; iy < N1; iy += 2) {
                    unsigned long long fl[N1], v[N1], sv[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        fl[j] = pack2(f[j + N1 * iy], f[j + N1 * iy + N1]);
                        v[j] = pack2(vx[iy][j], vx[iy + 1][j]);
                    }
                    if (l0) {
                        const unsigned long long tj = trace_jump2<N1, true>(v, fl[RL], A.ops);
                        const unsigned long long gj = fsub2(dup2(gx), fl[RL]);
                        line_sums_jump2<N1, true>(sv, fl, enx >= 0 ? tj : gj, A.ops);
                    } else {
                        const unsigned long long tj = trace_jump2<N1, false>(v, fl[RR], A.ops);
                        const unsigned long long gj = fsub2(dup2(gx), fl[RR]);
                        line_sums_jump2<N1, false>(sv, fl, enx >= 0 ? tj : gj, A.ops);
                    }
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        float lo, hi;
                        unpack2(sv[j], lo, hi);
                        acc[j + N1 * iy] = fmaf(cx, lo, acc[j + N1 * iy]);
                        acc[j + N1 * iy + N1] = fmaf(cx, hi, acc[j + N1 * iy + N1]);
                    }
                }
#pragma unroll
                for (int ix = 0; ix < N1; ix += 2) {
                    unsigned long long fl[N1], v[N1], sv[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        fl[j] = pack2(f[ix + N1 * j], f[ix + 1 + N1 * j]);
                        v[j] = pack2(vy[ix][j], vy[ix + 1][j]);
                    }
                    if (l1) {
                        const unsigned long long tj = trace_jump2<N1, true>(v, fl[RL], A.ops);
                        const unsigned long long gj = fsub2(dup2(gy), fl[RL]);
                        line_sums_jump2<N1, true>(sv, fl, eny >= 0 ? tj : gj, A.ops);
                    } else {
                        const unsigned long long tj = trace_jump2<N1, false>(v, fl[RR], A.ops);
                        const unsigned long long gj = fsub2(dup2(gy), fl[RR]);
                        line_sums_jump2<N1, false>(sv, fl, eny >= 0 ? tj : gj, A.ops);
                    }
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        float lo, hi;
                        unpack2(sv[j], lo, hi);
                        acc[ix + N1 * j] = fmaf(cy, lo, acc[ix + N1 * j]);
                        acc[ix + 1 + N1 * j] = fmaf(cy, hi, acc[ix + 1 + N1 * j]);
                    }
                }
            } else {
#pragma unroll
                for (int iy = 0; iy < N1; iy++) {
                    float fl[N1], sv[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        fl[j] = f[j + N1 * iy];
                    if (l0) {
                        const float t = trace_line<N1, true>(vx[iy], A.ops);
                        line_sums<N1, true>(sv, fl, enx >= 0 ? t : gx, A.ops);
                    } else {
                        const float t = trace_line<N1, false>(vx[iy], A.ops);
                        line_sums<N1, false>(sv, fl, enx >= 0 ? t : gx, A.ops);
                    }
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
                    if (l1) {
                        const float t = trace_line<N1, true>(vy[ix], A.ops);
                        line_sums<N1, true>(sv, fl, eny >= 0 ? t : gy, A.ops);
                    } else {
                        const float t = trace_line<N1, false>(vy[ix], A.ops);
                        line_sums<N1, false>(sv, fl, eny >= 0 ? t : gy, A.ops);
                    }
#pragma unroll
                    for (int j = 0; j < N1; j++)
                        acc[ix + N1 * j] = fmaf(cy, sv[j], acc[ix + N1 * j]);
                }
            }
            // BGK source towards the conservative Maxwellian and the Shu-Osher combination, two nodes at
            // a time (exponent a + b.m + q |m|^2, or per-axis q on grids of several spacings)
            const float gm = gm_c;
            const float cg = A.kg * gm;
            const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
            const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
            const unsigned long long U0 = A.viso ? pack2(mms, mms) : pack2(mm0, mm0);
            const unsigned long long U1 = A.viso ? U0 : pack2(mm1, mm1);
            const unsigned long long U2 = A.viso ? 0ull : pack2(mm2, mm2);
#pragma unroll
            for (int h = 0; h < (NQ + 1) / 2; h++) {
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];
                const unsigned long long lin =
                    ffma2(pack2(p23.z, p23.w), M2,
                          ffma2(pack2(p23.x, p23.y), M1, ffma2(pack2(p01.z, p01.w), M0, pack2(p01.x, p01.y))));
                const unsigned long long ex =
                    ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U1, ffma2(pack2(p67.x, p67.y), U2, lin)));
                float g[2];
                exp2_fp32x2(ex, pack2(p67.z, p67.w), g[0], g[1]);
#pragma unroll
                for (int sl = 0; sl < 2; sl++) {
                    const int q = 2 * h + sl;
                    if (q >= NQ)
                        break;
                    float gc = cg;
                    if (A.vtau) {  // kg = b - kb exactly, kb as in the accumulator above
                        const float itau = sl == 0 ? p67.x : p67.y;
                        gc = __fsub_rn(A.b, __fsub_rn(A.b, __fmul_rn(bdt, itau))) * gm;
                    }
                    acc[q] = fmaf(gc, g[sl], acc[q]);
                }
            }
            if (A.limiter) {
                // Zhang-Shu (Sec. 2.1, Eqs. 10-11): the element mean (tensor Gauss-Legendre weights / 4,
                // summing to 1) and minimum of this velocity, all in this lane's registers
                float mean = 0.f, mn = acc[0];
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    mean = fmaf(A.ops.wq[q % N1] * A.ops.wq[q / N1], acc[q], mean);
                    mn = fminf(mn, acc[q]);
                }
                if (mn < 0.f) {
                    const float beta = fminf(fabsf(mean / (mean - mn)), 1.f);
#pragma unroll
                    for (int q = 0; q < NQ; q++)
                        acc[q] = fmaf(beta, acc[q] - mean, mean);
                }
            }
            float *dst = A.dst + fidx(vl, e, 0, lane, E, NQ);
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                __stcs(dst + q * kWarp, acc[q]);
                sm.tile[b][q][lane ^ (4 * (q & 7))] = acc[q];  // for the moments below
            }
        } else {
#pragma unroll
            for (int q = 0; q < NQ; q++)
                sm.tile[b][q][lane ^ (4 * (q & 7))] = f[q];
        }
        // moments of the element's nodes (Eq. 2 with Eq. 12) of the stored values
        __syncwarp();
        unsigned long long pm[2][5];
#pragma unroll
        for (int h = 0; h < 2; h++)
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
            for (int h = 0; h < 2; h++) {
                const int row = min(np + 8 * h, NQ - 1);  // rows past the element: discarded below
                const float4 v = *reinterpret_cast<const float4 *>(&sm.tile[b][row][kk ^ (4 * (row & 7))]);
                const unsigned long long v01 = pack2(v.x, v.y), v23 = pack2(v.z, v.w);
#pragma unroll
                for (int c = 0; c < 5; c++) {
                    pm[h][c] = ffma2(wv[c][0], v01, pm[h][c]);
                    pm[h][c] = ffma2(wv[c][1], v23, pm[h][c]);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int c = 0; c < 5; c++)
                sm.msum[5 * h + c][lane] += sum2(pm[h][c]);
        __syncwarp();  // every lane is done with this tile's rows before they are refilled
    }
    const int grp = A.group0 + gl;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int q = np + 8 * h;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            float x = sm.msum[5 * h + c][lane];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (kg == 0 && q < NQ)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)e * NQ + q] = x;
        }
    }
}

template <int N1, int MODE, int OCT>
cudaError_t launch2(const StageArgs &A, cudaStream_t s)
{
    const int ngroups = (A.nvt + A.G - 1) / A.G;
    const int EB = (A.mesh.nelem + kWarpsPerCta - 1) / kWarpsPerCta;
    k_stage2<N1, MODE, OCT><<<EB * ngroups, kWarp * kWarpsPerCta, 0, s>>>(A);
    return cudaGetLastError();
}

template <int N1>
cudaError_t launch2_any(const StageArgs &A, int mode, int oct, cudaStream_t s)
{
    if (mode == 1)
        return launch2<N1, 1, 8>(A, s);
    switch (oct & 3) {  // the z sign takes no part in a planar advection
    case 0: return oct < 8 ? launch2<N1, 0, 0>(A, s) : launch2<N1, 0, 8>(A, s);
    case 1: return oct < 8 ? launch2<N1, 0, 1>(A, s) : launch2<N1, 0, 8>(A, s);
    case 2: return oct < 8 ? launch2<N1, 0, 2>(A, s) : launch2<N1, 0, 8>(A, s);
    default: return oct < 8 ? launch2<N1, 0, 3>(A, s) : launch2<N1, 0, 8>(A, s);
    }
}

cudaError_t launch_stage2(const StageArgs &A, int p, int mode, int oct, cudaStream_t s)
{
    switch (p) {
    case 1: return launch2_any<2>(A, mode, oct, s);
    case 2: return launch2_any<3>(A, mode, oct, s);
    case 3: return launch2_any<4>(A, mode, oct, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bgk
