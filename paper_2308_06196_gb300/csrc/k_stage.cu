// k_stage.cu -- the fused SSP-RK3 stage kernel of the line-element (1-D in space, 3-D in velocity)
// form, FP32-split, its batched persistent variant, and the dispatch of all stage kernels.
//
// One task = a block of kWarpsPerCta consecutive elements x a run of G velocity tiles (32 velocities
// of one sign octant each); warp w of the CTA takes element w of the block. Lane l owns velocity l of
// the tile. The CTA streams its tiles through a ring of shared slots with cp.async, several tiles
// ahead. Per tile the warp
//   1. reads f_s and f^n of its element from the slot (staged as coalesced 128-byte rows),
//   2. adds the FR advection residual (Sec. 2.1, Eqs. 7-9): it reads the upwind neighbour element's
//      line (same tile) and interpolates the neighbour's trace at the shared face, the interior trace
//      being folded into the merged operator; a Dirichlet end supplies the sampled ghost value,
//   3. evaluates the conservative Maxwellian g = 2^j exp2(a + sum_d (b_d m_d + q_d m_d^2)) of every node
//      (m = the exact centred grid index of the velocity) from the per-point exponent the Newton kernel
//      wrote (Sec. 2.1, text after Eq. 13), applies the BGK
//      relaxation (Eq. 3) and the Shu-Osher combination of the stage (Sec. 2.2), stores f_{s+1},
//   4. accumulates w_k psi_k f_{s+1} (Eq. 2 with Eq. 12) per lane, node and moment (two nodes per
//      packed FP32 pair).
// At the end of the task a transpose-reduction over the 32 lanes leaves one (moment, node) total per
// lane, written as the task's FP32 partial; the Newton kernel sums the partials of all tasks exactly
// (double-float) before solving for the next stage's Maxwellian.
//
// The stage never reads what another task of the same launch writes: it reads f_s (source), f^n,
// the BGK exponent table and the ghost table, and writes only its own part of the destination and
// of the partial-moment table. The destination may alias f^n (the last stage updates f^n in place).
#include "stage_common.cuh"

namespace bgk {

// FR operators of the line kernel for each p + 1 (they depend on p only), read by the batched launch.
__constant__ Ops c_ops1d[kMaxN1 + 1];

// Sum of V <= 32 per-lane values over the warp, one total per lane: after the call, lane l of the
// warp holds sum over lanes of v[l] (v padded with zeros to 32). Five halving exchange steps.
__device__ __forceinline__ void transpose_reduce(float (&v)[32], int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = lane & s;
#pragma unroll
        for (int j = 0; j < s; j++) {
            const float send = up ? v[j] : v[j + s];
            const float keep = up ? v[j + s] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
}

constexpr int kLineDepth = 4;  // tiles in flight per CTA in the line-element stage

// Shared staging of one tile of the line-element stage: f_s and f^n of the CTA's block of elements,
// the upwind neighbour element just outside the block, and the tile's velocity tables.
template <int N1>
struct alignas(16) LineSlot {
    float fs[kWarpsPerCta][N1][kWarp];
    float fn[kWarpsPerCta][N1][kWarp];
    float nb[N1][kWarp];
    float mi[3][kWarp];
    float wp[5][kWarp];
    float gm[kWarp];
};
template <int N1>
struct alignas(16) LineSmem {  // cp.async and the 16-byte parameter loads need 16-byte alignment
    LineSlot<N1> s[kLineDepth];
    // BGK exponents of the block's nodes by element and node pair, [element][pair][param][node of the
    // pair], so that one 16-byte load gives two parameters of both nodes (an odd last pair repeats)
    float par[kWarpsPerCta][(N1 + 1) / 2][kParamStride][2];
};

// One task of the line-element stage: a block of kWarpsPerCta consecutive elements (warp w takes
// element eb + w) x a run of G tiles. The CTA streams the tiles through a kLineDepth-deep ring of
// shared slots (cp.async, kLineDepth - 1 tiles ahead), so every warp reads its element, its upwind
// neighbour (a sibling's element, or the staged outside neighbour) and the velocity tables from
// shared memory. MODE 0: full stage. MODE 1: moments of src only (no advection, no store).
// op: the FR operators of degree N1 - 1. Every thread of the CTA must call it (barriers).
template <int N1, int MODE>
__device__ __forceinline__ void stage1d_task(const StageArgs &A, const int task, const Ops &op, LineSmem<N1> &sm)
{
    constexpr int NP = N1;
    constexpr int NQ = (NP + 1) / 2;  // packed node pairs
    static_assert(5 * NP <= 32, "one (moment, node) total per lane");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int E = A.mesh.nelem;
    const int nEB = (E + kWarpsPerCta - 1) / kWarpsPerCta;
    const int gl = task / nEB;
    const int eb = (task % nEB) * kWarpsPerCta;
    const int ne = min(kWarpsPerCta, E - eb);
    const int e = eb + wid;
    const bool active = e < E;
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    int ec[3] = {e, 0, 0};
    const int eL = upwind_neighbour(A.mesh, ec, 0, true), eR = upwind_neighbour(A.mesh, ec, 0, false);
    ec[0] = eb;
    const int eoL = upwind_neighbour(A.mesh, ec, 0, true);  // outside neighbours of the block
    ec[0] = eb + ne - 1;
    const int eoR = upwind_neighbour(A.mesh, ec, 0, false);
    const bool has_fn = MODE == 0 && A.fn != nullptr;

    // Copy plan of the task, fixed for all its tiles (16-byte chunks; a slot's rows nb, mi, wp, gm
    // are contiguous in shared memory): the element block's f_s and f^n rows (stride tileA per tile)
    // and at most one table chunk per thread: a row of the outside neighbour (its element depends on
    // the tile's inflow side), of the grid index, of w psi or of the mask.
    const int tid = threadIdx.x;
    constexpr int CH = kWarp / 4;  // chunks per 128-byte row
    const int nA = ne * NP * CH;
    const int64_t tileA = (int64_t)E * NP * kWarp;
    const float *gA = A.src + (int64_t)eb * NP * kWarp;
    const float *gB = has_fn ? A.fn + (int64_t)eb * NP * kWarp : nullptr;
    const float *gC = nullptr;
    int64_t sC = 0;
    int cnb = -1;  // >= 0: this thread copies chunk cnb of the outside neighbour's rows
    if (MODE == 0) {
        const int q = tid - N1 * CH;
        if (tid < N1 * CH)
            cnb = 4 * tid;
        else if (q < 3 * CH) {
            gC = A.mi + (int64_t)(q / CH) * A.nslots + (int64_t)A.vt0 * kWarp + 4 * (q % CH);
            sC = kWarp;
        } else if (q < 8 * CH) {
            gC = A.wpsi + (int64_t)A.vt0 * 5 * kWarp + 4 * (q - 3 * CH);
            sC = 5 * kWarp;
        } else if (q < 9 * CH) {
            gC = A.gmask + (int64_t)A.vt0 * kWarp + 4 * (q - 8 * CH);
            sC = kWarp;
        }
    } else if (tid < 5 * CH) {  // moments only: the w psi rows
        gC = A.wpsi + (int64_t)A.vt0 * 5 * kWarp + 4 * tid;
        sC = 5 * kWarp;
    }
    auto prefetch = [&](int vl, int slot) {
        LineSlot<N1> &S = sm.s[slot];
        for (int k = tid; k < nA; k += blockDim.x)
            cp_async16(&S.fs[0][0][0] + 4 * k, gA + vl * tileA + 4 * k);
        if (MODE == 0 && has_fn)
            for (int k = tid; k < nA; k += blockDim.x)
                cp_async16(&S.fn[0][0][0] + 4 * k, gB + vl * tileA + 4 * k);
        float *tables = MODE == 0 ? &S.nb[0][0] : &S.wp[0][0];
        if (cnb >= 0) {
            const int eo = (__ldg(A.toct + A.vt0 + vl) & 1) ? eoL : eoR;
            if (eo >= 0)
                cp_async16(tables + cnb, A.src + fidx(vl, eo, 0, 0, E, NP) + cnb);
        } else if (gC) {
            cp_async16(tables + 4 * tid, gC + vl * sC);
        }
    };

    // BGK exponents of the block's nodes into shared memory (pair-interleaved); the first barrier of
    // the tile loop orders these stores before their reads
    if (MODE == 0) {
        const float *src = A.param + (int64_t)eb * NP * kParamStride;
        for (int q = threadIdx.x; q < ne * NQ * 2 * kParamStride; q += blockDim.x) {
            const int c = q % kParamStride, sl = (q / kParamStride) & 1, h = (q / (2 * kParamStride)) % NQ;
            const int el = q / (2 * kParamStride * NQ);
            sm.par[el][h][c][sl] = __ldg(src + (el * NP + min(2 * h + sl, NP - 1)) * kParamStride + c);
        }
    }
    const bool viso = A.viso != 0;
    unsigned long long m[5][NQ];
#pragma unroll
    for (int c = 0; c < 5; c++)
#pragma unroll
        for (int q = 0; q < NQ; q++)
            m[c][q] = 0ull;

    const float kb = A.kb;
    const float bdt = A.b * A.dt;
    const float cdt = -A.mesh.inv_h2[0] * bdt;
    const float cgt = A.kg;

#pragma unroll
    for (int d = 0; d < kLineDepth - 1; d++) {
        if (vl0 + d < vl1)
            prefetch(vl0 + d, d);
        cp_commit();
    }
    for (int vl = vl0; vl < vl1; vl++) {
        const int it = vl - vl0;
        cp_wait<kLineDepth - 2>();  // tile vl has landed (this thread's copies) ...
        __syncthreads();            // ... for every thread; and every warp is done with tile vl - 1
        {
            const int vn = vl + kLineDepth - 1;
            if (vn < vl1)
                prefetch(vn, (it + kLineDepth - 1) % kLineDepth);  // the slot of tile vl - 1
            cp_commit();
        }
        if (!active)
            continue;
        const LineSlot<N1> &S = sm.s[it % kLineDepth];
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        float o[NP];
        if (MODE == 0) {
            float f[NP];
#pragma unroll
            for (int i = 0; i < NP; i++)
                f[i] = S.fs[wid][i][lane];
            const float m0 = S.mi[0][lane], m1 = S.mi[1][lane], m2 = S.mi[2][lane];
            const float x0 = fmaf(A.vs[0], m0, A.vc[0]);
            // squared indices (exact) as the exponent's quadratic terms take them
            const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
            const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
            const unsigned long long U0 = viso ? pack2(mms, mms) : pack2(mm0, mm0);
            const unsigned long long U1 = viso ? U0 : pack2(mm1, mm1);
            const unsigned long long U2 = viso ? 0ull : pack2(mm2, mm2);
            // inflow side of the tile (one sign octant per tile)
            const bool left = (__ldg(A.toct + vt) & 1) != 0;
            const int en = left ? eL : eR;
            // upwind trace at the shared face: a sibling's element, the staged outside neighbour, or
            // the Dirichlet ghost value
            float T;
            if (en >= 0) {
                float v[N1];
                const int r = en - eb;
                const float *vrow = (r >= 0 && r < ne) ? &S.fs[r][0][0] : &S.nb[0][0];
#pragma unroll
                for (int j = 0; j < N1; j++)
                    v[j] = vrow[j * kWarp + lane];
                T = left ? trace_line<N1, true>(v, op) : trace_line<N1, false>(v, op);
            } else {
                T = __ldg(A.ghost + (left ? 0 : 1) * A.nslots + slot);
            }
            float sd[N1];
            if (left)
                line_sums<N1, true>(sd, f, T, op);
            else
                line_sums<N1, false>(sd, f, T, op);
            const float cd = cdt * x0;
            const float cg = cgt * S.gm[lane];
            float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
#pragma unroll
            for (int h = 0; h < NQ; h++) {
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[wid][h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];  // (c, c+1) of both nodes
                const unsigned long long lin =
                    ffma2(pack2(p23.z, p23.w), M2,
                          ffma2(pack2(p23.x, p23.y), M1, ffma2(pack2(p01.z, p01.w), M0, pack2(p01.x, p01.y))));
                const unsigned long long ex =
                    ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U1, ffma2(pack2(p67.x, p67.y), U2, lin)));
                float g[2];
                exp2_fp32x2(ex, pack2(p67.z, p67.w), g[0], g[1]);
                const float itau[2] = {p67.x, p67.y};  // variable collision time: 1/tau of both nodes
#pragma unroll
                for (int sl = 0; sl < 2; sl++) {
                    const int i = 2 * h + sl;
                    if (i < NP) {
                        const float fnv = has_fn ? S.fn[wid][i][lane] : 0.f;
                        float kbi = kb, cgi = cg;
                        if (A.vtau) {  // per-node weights, rounded so that kb + kg = b exactly
                            kbi = __fsub_rn(A.b, __fmul_rn(bdt, itau[sl]));
                            cgi = __fsub_rn(A.b, kbi) * S.gm[lane];
                        }
                        const float a = fmaf(cd, sd[i], fmaf(A.an, fnv, kbi * f[i]));
                        o[i] = fmaf(cgi, g[sl], a);
                    }
                }
            }
            if (A.limiter) {
                // Zhang-Shu (Sec. 2.1, Eqs. 10-11): contract towards the element mean where a node
                // value of this velocity is negative
                float mean = 0.f, mn = o[0];
#pragma unroll
                for (int i = 0; i < NP; i++) {
                    mean = fmaf(op.wq[i], o[i], mean);
                    mn = fminf(mn, o[i]);
                }
                if (mn < 0.f) {
                    const float beta = fminf(fabsf(mean / (mean - mn)), 1.f);
#pragma unroll
                    for (int i = 0; i < NP; i++)
                        o[i] = fmaf(beta, o[i] - mean, mean);
                }
            }
#pragma unroll
            for (int i = 0; i < NP; i++)
                __stcs(dst + i * kWarp, o[i]);
        } else {
#pragma unroll
            for (int i = 0; i < NP; i++)
                o[i] = S.fs[wid][i][lane];
        }
        // moments of this tile, accumulated per lane: m[c][q] += W psi_c (o_2q, o_2q+1)
#pragma unroll
        for (int c = 0; c < 5; c++) {
            const float w = S.wp[c][lane];
            const unsigned long long ww = pack2(w, w);
#pragma unroll
            for (int q = 0; q < NQ; q++)
                m[c][q] = ffma2(ww, pack2(o[2 * q], 2 * q + 1 < NP ? o[2 * q + 1] : 0.f), m[c][q]);
        }
    }
    cp_wait<0>();
    __syncthreads();  // the ring is free for the CTA's next task
    if (!active)
        return;

    // totals over the 32 velocities of every tile: value (c, i) at index c * NP + i
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; j++)
        v[j] = 0.f;
#pragma unroll
    for (int c = 0; c < 5; c++)
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            float lo, hi;
            unpack2(m[c][q], lo, hi);
            v[c * NP + 2 * q] = lo;
            if (2 * q + 1 < NP)
                v[c * NP + 2 * q + 1] = hi;
        }
    transpose_reduce(v, lane);
    if (lane < 5 * NP) {
        const int c = lane / NP, i = lane - c * NP;
        A.partial[((int64_t)(A.group0 + gl) * 5 + c) * A.npts + (int64_t)e * NP + i] = v[0];
    }
}

// Resident CTAs per SM the register allocation of the line kernels is sized for: 6 (80 registers, no
// spills) runs the planar shear wave's stage 5 % faster than 5 (96 registers); the batch is the same.
#ifndef BGK_STAGE1D_MINCTAS
#define BGK_STAGE1D_MINCTAS 6
#endif

template <int N1, int MODE>
__global__ void __launch_bounds__(kWarp *kWarpsPerCta, BGK_STAGE1D_MINCTAS) k_stage1d(const StageArgs A)
{
    __shared__ __align__(16) LineSmem<N1> sm;
    stage1d_task<N1, MODE>(A, blockIdx.x, A.ops, sm);
}

// Batched line-element stages: one persistent launch over the tasks of many independent problems
// (each with its own arguments, degree, mesh, velocity grid and task count). CTAs take tasks from an
// atomic counter; a binary search over the task prefix sums finds the problem. The degree selects the
// body; the FR operators of each degree come from constant memory.
__global__ void __launch_bounds__(kWarp *kWarpsPerCta, BGK_STAGE1D_MINCTAS)
    k_stage1d_batch(const StageArgs *__restrict__ args, const int *__restrict__ task_start, int n, int *counter)
{
    __shared__ int s_item;
    __shared__ __align__(16) LineSmem<4> sm;  // the largest degree of the batch (p = 3); smaller ones use its front
    const int total = task_start[n];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total)
            break;
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(task_start + mid) <= item)
                lo = mid;
            else
                hi = mid;
        }
        const StageArgs &A = args[lo];
        const int task = item - __ldg(task_start + lo);
        switch (A.n1) {
        case 2: stage1d_task<2, 0>(A, task, c_ops1d[2], *reinterpret_cast<LineSmem<2> *>(&sm)); break;
        case 3: stage1d_task<3, 0>(A, task, c_ops1d[3], *reinterpret_cast<LineSmem<3> *>(&sm)); break;
        case 4: stage1d_task<4, 0>(A, task, c_ops1d[4], sm); break;
        default: break;
        }
    }
}

// Tasks of one line-element launch of A (the batch prefix sums use the same count).
int stage1d_tasks(const StageArgs &A)
{
    const int nEB = (A.mesh.nelem + kWarpsPerCta - 1) / kWarpsPerCta;
    return nEB * ((A.nvt + A.G - 1) / A.G);
}

// Copy the line operators of degree n1 - 1 into the constant table of the batched launch.
cudaError_t set_batch_ops(int n1, const Ops &op)
{
    return cudaMemcpyToSymbol(c_ops1d, &op, sizeof(Ops), (size_t)n1 * sizeof(Ops));
}

// The work counter is reset in the same stream before every launch (a captured memset node).
cudaError_t launch_stage1d_batch(const StageArgs *d_args, const int *d_task_start, int n, int *d_counter,
                                 int ctas, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    k_stage1d_batch<<<ctas, kWarp * kWarpsPerCta, 0, s>>>(d_args, d_task_start, n, d_counter);
    return cudaGetLastError();
}

// CTAs of the persistent launch: every SM filled to the kernel's occupancy.
int stage1d_batch_ctas()
{
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage1d_batch, kWarp * kWarpsPerCta, 0);
    return nsm * (per > 0 ? per : 1);
}

cudaError_t prepare_stage3_p1();
cudaError_t prepare_stage3_p2();
cudaError_t prepare_stage3_p3();
cudaError_t launch_stage3_p1(const StageArgs &A, int mode, int oct, cudaStream_t s);
cudaError_t launch_stage3_p2(const StageArgs &A, int mode, int oct, cudaStream_t s);
cudaError_t launch_stage3_p3(const StageArgs &A, int mode, int oct, cudaStream_t s);
cudaError_t launch_stage2(const StageArgs &A, int p, int mode, int oct, cudaStream_t s);

template <int N1>
static cudaError_t launch_1d(const StageArgs &A, int mode, cudaStream_t s)
{
    const int ntask = stage1d_tasks(A);
    if (mode == 0)
        k_stage1d<N1, 0><<<ntask, kWarp * kWarpsPerCta, 0, s>>>(A);
    else
        k_stage1d<N1, 1><<<ntask, kWarp * kWarpsPerCta, 0, s>>>(A);
    return cudaGetLastError();
}

// Set the shared-memory attributes of the stage kernels of one (dim, p); call before any capture.
cudaError_t prepare_stage(int dim, int p)
{
    if (dim == 3) {
        switch (p) {
        case 1: return prepare_stage3_p1();
        case 2: return prepare_stage3_p2();
        case 3: return prepare_stage3_p3();
        }
    } else if (dim == 1 && p >= 1 && p <= 5) {
        return cudaSuccess;  // the line kernels use static shared memory only
    } else if (dim == 2 && p >= 1 && p <= 3) {
        return cudaSuccess;  // so do the quadrilateral kernels
    }
    return cudaErrorInvalidValue;
}

// Launch one stage (mode 0) or a moments-only pass (mode 1) over one velocity chunk whose tiles all
// lie in sign octant oct (8: mixed octants).
cudaError_t launch_stage(const StageArgs &A, int p, int mode, int oct, cudaStream_t s)
{
    if (A.mesh.dim == 3) {
        switch (p) {
        case 1: return launch_stage3_p1(A, mode, oct, s);
        case 2: return launch_stage3_p2(A, mode, oct, s);
        case 3: return launch_stage3_p3(A, mode, oct, s);
        }
    } else if (A.mesh.dim == 2) {
        return launch_stage2(A, p, mode, oct, s);
    } else if (A.mesh.dim == 1) {
        switch (p) {
        case 1: return launch_1d<2>(A, mode, s);
        case 2: return launch_1d<3>(A, mode, s);
        case 3: return launch_1d<4>(A, mode, s);
        case 4: return launch_1d<5>(A, mode, s);
        case 5: return launch_1d<6>(A, mode, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace bgk
