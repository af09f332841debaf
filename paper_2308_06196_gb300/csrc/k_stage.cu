// k_stage.cu -- the fused SSP-RK3 stage kernel of the line-element (1-D in space, 3-D in velocity)
// form, FP32-split, its batched persistent variant, and the dispatch of all stage kernels.
//
// One task = a block of kWarpsPerCta consecutive elements x a run of G velocity tiles (32 velocities
// of one sign octant each); warp w of the CTA takes element w of the block. Lane l owns velocity l of
// the tile and keeps the p+1 nodes of its element in registers. Per tile the warp
//   1. loads f_s and f^n of its element (coalesced 128-byte lines, one per node; the next tile's
//      values are prefetched while the current one is computed),
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

// One task of the line-element stage. MODE 0: full stage. MODE 1: moments of src only (no advection,
// no store). op: the FR operators of degree N1 - 1.
template <int N1, int MODE>
__device__ __forceinline__ void stage1d_task(const StageArgs &A, const int task, const Ops &op)
{
    constexpr int NP = N1;
    constexpr int NQ = (NP + 1) / 2;  // packed node pairs
    static_assert(5 * NP <= 32, "one (moment, node) total per lane");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int E = A.mesh.nelem;
    const int nEB = (E + kWarpsPerCta - 1) / kWarpsPerCta;
    const int gl = task / nEB;
    const int e = (task % nEB) * kWarpsPerCta + wid;
    if (e >= E)
        return;  // whole warp; the task uses no CTA-wide synchronisation
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    const int ec[3] = {e, 0, 0};
    const int eL = upwind_neighbour(A.mesh, ec, 0, true), eR = upwind_neighbour(A.mesh, ec, 0, false);
    const float *__restrict__ src = A.src;
    const float *__restrict__ fnp = A.fn;

    // BGK exponents of the element's nodes (the same for every lane)
    float pb[NP][8];
    if (MODE == 0) {
#pragma unroll
        for (int i = 0; i < NP; i++) {
            const float *q = A.param + ((int64_t)e * NP + i) * kParamStride;
            const float4 v = __ldg(reinterpret_cast<const float4 *>(q));
            const float4 u = __ldg(reinterpret_cast<const float4 *>(q + 4));
            pb[i][0] = v.x;
            pb[i][1] = v.y;
            pb[i][2] = v.z;
            pb[i][3] = v.w;
            pb[i][4] = u.x;
            pb[i][5] = u.y;
            pb[i][6] = u.z;
            pb[i][7] = u.w;
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
    const float cdt = -A.mesh.inv_h2[0] * (A.b * A.dt);
    const float cgt = A.kg;
    // f: f_s of the current tile; acc: f^n of the current tile (or 0), prefetched one tile ahead
    float f[NP], acc[NP];
    {
        const int64_t b0 = fidx(vl0, e, 0, lane, E, NP);
#pragma unroll
        for (int i = 0; i < NP; i++) {
            f[i] = __ldg(src + b0 + i * kWarp);
            acc[i] = (MODE == 0 && fnp) ? __ldcs(fnp + b0 + i * kWarp) : 0.f;
        }
    }
    for (int vl = vl0; vl < vl1; vl++) {
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        float nf[NP], nacc[NP];
        if (vl + 1 < vl1) {
            const int64_t b1 = fidx(vl + 1, e, 0, lane, E, NP);
#pragma unroll
            for (int i = 0; i < NP; i++) {
                nf[i] = __ldg(src + b1 + i * kWarp);
                nacc[i] = (MODE == 0 && fnp) ? __ldcs(fnp + b1 + i * kWarp) : 0.f;
            }
        }
        float o[NP];
        if (MODE == 0) {
            const float m0 = __ldg(A.mi + slot), m1 = __ldg(A.mi + A.nslots + slot);
            const float m2 = __ldg(A.mi + 2 * A.nslots + slot);
            const float x0 = fmaf(A.vs[0], m0, A.vc[0]);
            // squared indices (exact) as the exponent's quadratic terms take them
            const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
            const float u0 = viso ? mms : mm0, u1 = viso ? mms : mm1, u2 = viso ? 0.f : mm2;
            const bool left = x0 >= 0.f;
            const int en = left ? eL : eR;
            // upwind trace at the shared face
            float T;
            if (en >= 0) {
                float v[N1];
                const int64_t bn = fidx(vl, en, 0, lane, E, NP);
#pragma unroll
                for (int j = 0; j < N1; j++)
                    v[j] = __ldg(src + bn + j * kWarp);
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
            const float cg = cgt * __ldg(A.gmask + slot);
            float *dst = A.dst + fidx(vl, e, 0, lane, E, NP);
#pragma unroll
            for (int i = 0; i < NP; i++) {
                const float lin = fmaf(pb[i][3], m2, fmaf(pb[i][2], m1, fmaf(pb[i][1], m0, pb[i][0])));
                const float ex = fmaf(pb[i][4], u0, fmaf(pb[i][5], u1, fmaf(pb[i][6], u2, lin)));
                const float a = fmaf(cd, sd[i], fmaf(A.an, acc[i], kb * f[i]));
                o[i] = fmaf(cg, exp2_fp32(ex, pb[i][7]), a);
                __stcs(dst + i * kWarp, o[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NP; i++)
                o[i] = f[i];
        }
        // moments of this tile, accumulated per lane: m[c][q] += w psi_c (o_2q, o_2q+1)
#pragma unroll
        for (int c = 0; c < 5; c++) {
            const float w = __ldg(A.wpsi + ((int64_t)vt * 5 + c) * kWarp + lane);
            const unsigned long long ww = pack2(w, w);
#pragma unroll
            for (int q = 0; q < NQ; q++)
                m[c][q] = ffma2(ww, pack2(o[2 * q], 2 * q + 1 < NP ? o[2 * q + 1] : 0.f), m[c][q]);
        }
        if (vl + 1 < vl1) {
#pragma unroll
            for (int i = 0; i < NP; i++) {
                f[i] = nf[i];
                acc[i] = nacc[i];
            }
        }
    }

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
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(m[c][q]));
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

template <int N1, int MODE>
__global__ void __launch_bounds__(kWarp *kWarpsPerCta) k_stage1d(const StageArgs A)
{
    stage1d_task<N1, MODE>(A, blockIdx.x, A.ops);
}

// Batched line-element stages: one persistent launch over the tasks of many independent problems
// (each with its own arguments, degree, mesh, velocity grid and task count). CTAs take tasks from an
// atomic counter; a binary search over the task prefix sums finds the problem. The degree selects the
// body; the FR operators of each degree come from constant memory.
__global__ void __launch_bounds__(kWarp *kWarpsPerCta, 4)
    k_stage1d_batch(const StageArgs *__restrict__ args, const int *__restrict__ task_start, int n, int *counter)
{
    __shared__ int s_item;
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
        case 2: stage1d_task<2, 0>(A, task, c_ops1d[2]); break;
        case 3: stage1d_task<3, 0>(A, task, c_ops1d[3]); break;
        case 4: stage1d_task<4, 0>(A, task, c_ops1d[4]); break;
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
