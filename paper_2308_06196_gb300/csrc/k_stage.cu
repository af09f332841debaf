// k_stage.cu -- the fused SSP-RK3 stage kernel of the line-element (1-D in space, 3-D in velocity)
// form, FP32-split, its batched persistent variant, and the dispatch of all stage kernels.
//
// One task = a run of consecutive elements (at most 16 nodes) x a run of G velocity tiles (32
// velocities of one sign octant each), on one warp: lane l owns velocity l of the tile. The warp
// streams its tiles through two shared buffers with bulk asynchronous copies on its own mbarriers,
// one tile ahead, and shares no barrier with any other warp (see line_task).
//
// The stage never reads what another task of the same launch writes: it reads f_s (source), f^n,
// the BGK exponent table and the ghost table, and writes only its own part of the destination and
// of the partial-moment table. The destination may alias f^n (the last stage updates f^n in place).
#include <type_traits>
#include "stage_common.cuh"

namespace bgk {

// FR operators of the line kernel for each p + 1 (they depend on p only), read by the batched launch.
__constant__ Ops c_ops1d[kMaxN1 + 1];

// Elements per task of the line kernels: a run of K = 16 / N1 consecutive elements, so that a warp
// holds at most 16 nodes of every velocity of its tile.
template <int N1>
__host__ __device__ constexpr int line_run()
{
    return 16 / N1;
}

// Shared memory of one warp of the line kernels (bulk copies, the warp's own mbarriers). Per buffer
// b (tile parity): fs the run's f_s rows between the rows of its two outside neighbours (only the
// upwind one is copied; the right one's rows follow the run's last real element), fn its f^n rows,
// tab the tile's velocity table. The barriers come first, at the same place for every N1 (the batched
// launch steps problems of different degrees through one warp's storage).
template <int N1>
struct __align__(16) LineWarp {
    static constexpr int K = line_run<N1>(), NW = K * N1;
    unsigned long long bar[2];
    float fs[2][NW + 2 * N1][kWarp];
    float fn[2][NW][kWarp];
    float tab[2][5][kWarp];
    float par[(NW + 1) / 2][kParamStride][2];  // BGK exponents of the run's nodes by pair
};

#ifndef BGK_LINE_WARPS
#define BGK_LINE_WARPS 4  // warps (independent tasks) per CTA of the line kernels
#endif
#ifndef BGK_LINE_MINCTAS
#define BGK_LINE_MINCTAS 4
#endif

// One task of the line-element stage: the run of elements eb .. eb + ne - 1 x a run of G velocity
// tiles, on one warp with no barrier shared with other warps. Lane l owns velocity l of the tile. The
// next tile's f_s, f^n, upwind outside neighbour and velocity table are in flight (one bulk copy each,
// issued by lanes 0-3 on one mbarrier) while this tile is computed. Per tile the warp
//   1. forms every element's FR advection residual (Sec. 2.1, Eqs. 7-9) from its line and the upwind
//      trace: the neighbouring element's interpolant at the shared face (a run element's or the
//      staged outside neighbour's), or the Dirichlet ghost value at a boundary end;
//   2. evaluates the conservative Maxwellian g = 2^j exp2(a + sum_d (b_d m_d + q_d m_d^2)) of every node
//      (m = the exact centred grid index of the velocity) from the per-point exponent the Newton kernel
//      wrote (Sec. 2.1, text after Eq. 13), applies the BGK relaxation (Eq. 3), the Shu-Osher
//      combination of the stage (Sec. 2.2) and, if on, the positivity limiter (Eqs. 10-11); stores
//      f_{s+1};
//   3. transposes the output through the consumed f_s rows and accumulates the moments W psi f_{s+1}
//      (Eq. 2 with Eq. 12): lane = (row np = lane / 4 of every group of 8 nodes) x (velocity eighth
//      kg = lane % 4), running sums in registers, combined over the 4 lanes of a row at the end and
//      written as the task's FP32 partial; the Newton kernel sums the partials of all tasks exactly.
// MODE 0: full stage. MODE 1: moments of src only (no advection, no store). ph: the phase parity
// bits of the warp's two barriers, carried across the tasks a warp runs.
template <int N1, int MODE, bool VT>
__device__ __forceinline__ void line_task(const StageArgs &A, const int task, const Ops &op, LineWarp<N1> &sm,
                                          uint32_t &ph)
{
    constexpr int NP = N1;
    constexpr int K = LineWarp<N1>::K, NW = LineWarp<N1>::NW;
    constexpr int NH = (NW + 1) / 2;
    constexpr int NHR = (NW + 7) / 8;
    constexpr uint32_t kRow = kWarp * sizeof(float);
    const int lane = threadIdx.x & 31;
    const int E = A.mesh.nelem;
    const int nEB = (E + K - 1) / K;
    const int gl = task / nEB;
    const int eb = (task % nEB) * K;
    const int ne = min(K, E - eb);
    const int nr = ne * N1;  // real rows of the run
    const int vl0 = gl * A.G;
    const int vl1 = min(vl0 + A.G, A.nvt);
    int ec[3] = {eb, 0, 0};
    const int enL = upwind_neighbour(A.mesh, ec, 0, true);  // outside neighbours of the run
    ec[0] = eb + ne - 1;
    const int enR = upwind_neighbour(A.mesh, ec, 0, false);
    const bool has_fn = MODE == 0 && A.fn != nullptr;

    __syncwarp();  // the previous task of this warp is done with the exponents and both buffers
    if (MODE == 0) {
        const float *src = A.param + (int64_t)eb * NP * kParamStride;
        for (int q = lane; q < NH * 2 * kParamStride; q += kWarp) {
            const int c = q % kParamStride, s2 = (q / kParamStride) & 1, h = q / (2 * kParamStride);
            sm.par[h][c][s2] = __ldg(src + min(2 * h + s2, nr - 1) * kParamStride + c);
        }
    }
    const int64_t tstride = (int64_t)E * NP * kWarp;
    const float *runsrc = A.src + fidx(0, eb, 0, 0, E, NP);
    const float *fnsrc = has_fn ? A.fn + fidx(0, eb, 0, 0, E, NP) : nullptr;
    const uint32_t bar0 = smem_u32(&sm.bar[0]);
    // the copies of tile vl into buffer b: lane 0 announces the bytes, lanes 0-3 issue one copy each
    auto issue = [&](int vl, int b) {
        const bool left = (__ldg(A.toct + A.vt0 + vl) & 1) != 0;
        const int en = left ? enL : enR;
        const bool nb = MODE == 0 && en >= 0;
        const uint32_t bb = bar0 + 8u * (uint32_t)b;
        if (lane == 0)
            mbar_arrive_expect_tx(bb, (uint32_t)(nr * (has_fn ? 2 : 1) + (nb ? N1 : 0) + 5) * kRow);
        __syncwarp();
        if (lane == 0)
            bulk_g2s(smem_u32(&sm.fs[b][N1][0]), runsrc + vl * tstride, nr * kRow, bb);
        else if (lane == 1 && has_fn)
            bulk_g2s(smem_u32(&sm.fn[b][0][0]), fnsrc + vl * tstride, nr * kRow, bb);
        else if (lane == 2 && nb)
            bulk_g2s(smem_u32(&sm.fs[b][left ? 0 : N1 + nr][0]), A.src + fidx(vl, en, 0, 0, E, NP), N1 * kRow, bb);
        else if (lane == 3)
            bulk_g2s(smem_u32(&sm.tab[b][0][0]), A.vtab + (int64_t)(A.vt0 + vl) * 5 * kWarp, 5 * kRow, bb);
    };
    if (vl0 < vl1) {
        fence_proxy_async();
        issue(vl0, 0);
    }

    const int np = lane >> 2, kg = lane & 3;
    float msum[NHR][5];
#pragma unroll
    for (int h = 0; h < NHR; h++)
#pragma unroll
        for (int c = 0; c < 5; c++)
            msum[h][c] = 0.f;
    const bool viso = A.viso != 0;
    const float kb = A.kb;
    const float bdt = A.b * A.dt;
    const float cdt = -A.mesh.inv_h2[0] * bdt;

    for (int vl = vl0; vl < vl1; vl++) {
        const int b = (vl - vl0) & 1;
        if (vl + 1 < vl1) {  // buffer b ^ 1 was consumed by the previous tile (its moment pass)
            __syncwarp();
            fence_proxy_async();
            issue(vl + 1, b ^ 1);
        }
        mbar_wait(bar0 + 8u * (uint32_t)b, (ph >> b) & 1, A.err);
        ph ^= 1u << b;
        const int vt = A.vt0 + vl;
        const int slot = vt * kWarp + lane;
        float acc[NW];
        if (MODE == 0) {
            const bool left = (__ldg(A.toct + vt) & 1) != 0;
            const float m0 = sm.tab[b][0][lane], m1 = sm.tab[b][1][lane], m2 = sm.tab[b][2][lane];
            const float x0 = fmaf(A.vs[0], m0, A.vc[0]);
            const float cd = cdt * x0;
            const float gm = sm.tab[b][3][lane] != 0.f ? 1.f : 0.f;  // the padding mask
            const float cg = A.kg * gm;
            // 1. advection of every element of the run: acc = an f^n + kb f_s + cd (line sums). Every
            // element slot of the run is computed (those past a short run from stale rows, never stored),
            // and the inflow side is one test per tile, so the unrolled loops stay one basic block each.
            float gh = 0.f;  // the Dirichlet ghost value at the run's inflow end, where it is a boundary
            if (left ? enL < 0 : enR < 0)
                gh = __ldg(A.ghost + (left ? 0 : A.nslots) + slot);
            auto advect = [&](auto left_c) {
                constexpr bool LEFT = decltype(left_c)::value;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    float fl[N1], v[N1], sd[N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        fl[j] = sm.fs[b][N1 + k * N1 + j][lane];
                        v[j] = sm.fs[b][LEFT ? k * N1 + j : N1 + (k + 1) * N1 + j][lane];
                    }
                    const float tr = trace_line<N1, LEFT>(v, op);
                    const bool inner = LEFT ? (k > 0 || enL >= 0) : (k < ne - 1 || enR >= 0);
                    line_sums<N1, LEFT>(sd, fl, inner ? tr : gh, op);
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        const int r = k * N1 + j;
                        const float fr = sm.fn[b][r][lane];
                        const float fnv = has_fn ? fr : 0.f;
                        float kbi = kb;
                        if constexpr (VT)  // per-node weights, rounded so that kb + kg = b exactly
                            kbi = __fsub_rn(A.b, __fmul_rn(bdt, sm.par[r / 2][6][r % 2]));
                        acc[r] = fmaf(cd, sd[j], fmaf(A.an, fnv, kbi * fl[j]));
                    }
                }
            };
            if (left)
                advect(std::true_type{});
            else
                advect(std::false_type{});
            // 2. BGK source towards the conservative Maxwellian, two nodes at a time
            const float mm0 = m0 * m0, mm1 = m1 * m1, mm2 = m2 * m2, mms = mm0 + mm1 + mm2;
            const unsigned long long M0 = pack2(m0, m0), M1 = pack2(m1, m1), M2 = pack2(m2, m2);
            const unsigned long long U0 = viso ? pack2(mms, mms) : pack2(mm0, mm0);
            const unsigned long long U1 = viso ? U0 : pack2(mm1, mm1);
            const unsigned long long U2 = viso ? 0ull : pack2(mm2, mm2);
#pragma unroll
            for (int h = 0; h < NH; h++) {  // pairs past a short run: clamped exponents, never stored
                const float4 *pp = reinterpret_cast<const float4 *>(&sm.par[h][0][0]);
                const float4 p01 = pp[0], p23 = pp[1], p45 = pp[2], p67 = pp[3];  // (c, c+1) of both nodes
                const unsigned long long lin =
                    ffma2(pack2(p23.z, p23.w), M2,
                          ffma2(pack2(p23.x, p23.y), M1, ffma2(pack2(p01.z, p01.w), M0, pack2(p01.x, p01.y))));
                const unsigned long long ex =
                    ffma2(pack2(p45.x, p45.y), U0, ffma2(pack2(p45.z, p45.w), U1, ffma2(pack2(p67.x, p67.y), U2, lin)));
                float g[2];
                exp2_fp32x2(ex, pack2(p67.z, p67.w), g[0], g[1]);
#pragma unroll
                for (int s2 = 0; s2 < 2; s2++) {
                    const int r = 2 * h + s2;
                    if (r >= NW)
                        break;
                    float cgi = cg;
                    if constexpr (VT) {
                        const float kbi = __fsub_rn(A.b, __fmul_rn(bdt, s2 == 0 ? p67.x : p67.y));
                        cgi = __fsub_rn(A.b, kbi) * gm;
                    }
                    acc[r] = fmaf(cgi, g[s2], acc[r]);
                }
            }
            if (A.limiter) {
                // Zhang-Shu (Sec. 2.1, Eqs. 10-11): contract towards the element mean where a node
                // value of this velocity is negative
#pragma unroll
                for (int k = 0; k < K; k++) {  // (element slots past a short run: never stored)
                    float mean = 0.f, mn = acc[k * N1];
#pragma unroll
                    for (int j = 0; j < N1; j++) {
                        mean = fmaf(op.wq[j], acc[k * N1 + j], mean);
                        mn = fminf(mn, acc[k * N1 + j]);
                    }
                    if (mn < 0.f) {
                        const float beta = fminf(fabsf(mean / (mean - mn)), 1.f);
#pragma unroll
                        for (int j = 0; j < N1; j++)
                            acc[k * N1 + j] = fmaf(beta, acc[k * N1 + j] - mean, mean);
                    }
                }
            }
            float *dst = A.dst + fidx(vl, eb, 0, lane, E, NP);
#pragma unroll
            for (int r = 0; r < NW; r++)
                if (r < nr)
                    __stcs(dst + r * kWarp, acc[r]);
        } else {
#pragma unroll
            for (int r = 0; r < NW; r++)
                acc[r] = r < nr ? sm.fs[b][N1 + r][lane] : 0.f;
        }
        // 3. moments of the run's nodes of the stored values: the output transposed through the f_s
        // rows (every lane has read its own column of them), 4-float groups of row r rotated by r mod 8
        __syncwarp();
#pragma unroll
        for (int r = 0; r < NW; r++)
            if (r < nr)
                sm.fs[b][N1 + r][lane ^ (4 * (r & 7))] = acc[r];
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
                const int row = min(np + 8 * h, nr - 1);  // rows past the run: discarded below
                const float4 v = *reinterpret_cast<const float4 *>(&sm.fs[b][N1 + row][kk ^ (4 * (row & 7))]);
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
    }
    // partial moments of this task: combine the 4 velocity eighths of every row
    const int grp = A.group0 + gl;
#pragma unroll
    for (int h = 0; h < NHR; h++) {
        const int row = np + 8 * h;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            float x = msum[h][c];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (kg == 0 && row < nr)
                A.partial[((int64_t)grp * 5 + c) * A.npts + (int64_t)eb * NP + row] = x;
        }
    }
}

// Tasks of one line-element launch of A (the batch prefix sums use the same count).
template <int N1>
__host__ __device__ int line_tasks(const StageArgs &A)
{
    constexpr int K = line_run<N1>();
    return ((A.mesh.nelem + K - 1) / K) * ((A.nvt + A.G - 1) / A.G);
}

int stage1d_tasks(const StageArgs &A)
{
    switch (A.n1) {
    case 2: return line_tasks<2>(A);
    case 3: return line_tasks<3>(A);
    case 4: return line_tasks<4>(A);
    case 5: return line_tasks<5>(A);
    case 6: return line_tasks<6>(A);
    }
    return 0;
}

__device__ __forceinline__ void line_init_barriers(uint32_t bar0)
{
    if ((threadIdx.x & 31) == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8u, 1);
        fence_mbar_init();
    }
    __syncwarp();
}

template <int N1, int MODE>
__global__ void __launch_bounds__(kWarp *BGK_LINE_WARPS, BGK_LINE_MINCTAS) k_stage1d(const StageArgs A)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int w = threadIdx.x >> 5;
    const int task = blockIdx.x * BGK_LINE_WARPS + w;
    if (task >= line_tasks<N1>(A))  // no barrier below involves other warps
        return;
    LineWarp<N1> &sm = reinterpret_cast<LineWarp<N1> *>(smraw)[w];
    line_init_barriers(smem_u32(&sm.bar[0]));
    uint32_t ph = 0;
    if (MODE == 0 && A.vtau)
        line_task<N1, MODE, true>(A, task, A.ops, sm, ph);
    else
        line_task<N1, MODE, false>(A, task, A.ops, sm, ph);
}

// Batched line-element stages: one persistent launch per degree over the tasks of that degree's
// problems (each with its own arguments, mesh, velocity grid and task count), so every launch runs one
// body. The task table lists the tasks degree by degree; block = {counter, first task, end}: every warp
// takes tasks from the counter on its own, and one load from the table gives the task's problem and its
// task index there. The FR operators of each degree come from constant memory.
template <int N1>
__global__ void __launch_bounds__(kWarp *BGK_LINE_WARPS, BGK_LINE_MINCTAS)
    k_stage1d_batch(const StageArgs *__restrict__ args, const int2 *__restrict__ task_member, int *block)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    LineWarp<N1> &sm = reinterpret_cast<LineWarp<N1> *>(smraw)[w];
    line_init_barriers(smem_u32(&sm.bar[0]));
    uint32_t ph = 0;
    const int first = *reinterpret_cast<volatile int *>(block + 1);
    const int end = *reinterpret_cast<volatile int *>(block + 2);
    for (;;) {
        int item = 0;
        if (lane == 0)
            item = first + atomicAdd(block, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= end)
            break;
        const int2 tm = __ldg(task_member + item);  // (member, its task index)
        if (args[tm.x].vtau)
            line_task<N1, 0, true>(args[tm.x], tm.y, c_ops1d[N1], sm, ph);
        else
            line_task<N1, 0, false>(args[tm.x], tm.y, c_ops1d[N1], sm, ph);
    }
}

static_assert(BGK_LINE_WARPS * sizeof(LineWarp<5>) <= 48 * 1024 && BGK_LINE_WARPS * sizeof(LineWarp<4>) <= 48 * 1024,
              "the line kernels stay within the default dynamic shared memory");

// Copy the line operators of degree n1 - 1 into the constant table of the batched launches.
cudaError_t set_batch_ops(int n1, const Ops &op)
{
    return cudaMemcpyToSymbol(c_ops1d, &op, sizeof(Ops), (size_t)n1 * sizeof(Ops));
}

// The launch of degree n1 - 1: its counter is reset in the same stream before every launch (a captured
// memset node); the first task and the end next to it are written with the task table.
cudaError_t launch_stage1d_batch(int n1, const StageArgs *d_args, const int2 *d_task_member, int *d_block, int ctas,
                                 cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_block, 0, sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    switch (n1) {
    case 2: k_stage1d_batch<2><<<ctas, kWarp * BGK_LINE_WARPS, BGK_LINE_WARPS * sizeof(LineWarp<2>), s>>>(
        d_args, d_task_member, d_block); break;
    case 3: k_stage1d_batch<3><<<ctas, kWarp * BGK_LINE_WARPS, BGK_LINE_WARPS * sizeof(LineWarp<3>), s>>>(
        d_args, d_task_member, d_block); break;
    case 4: k_stage1d_batch<4><<<ctas, kWarp * BGK_LINE_WARPS, BGK_LINE_WARPS * sizeof(LineWarp<4>), s>>>(
        d_args, d_task_member, d_block); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// CTAs of the persistent launch of degree n1 - 1: every SM filled to the kernel's occupancy.
int stage1d_batch_ctas(int n1)
{
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (n1 == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage1d_batch<2>, kWarp * BGK_LINE_WARPS,
                                                      BGK_LINE_WARPS * sizeof(LineWarp<2>));
    else if (n1 == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage1d_batch<3>, kWarp * BGK_LINE_WARPS,
                                                      BGK_LINE_WARPS * sizeof(LineWarp<3>));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage1d_batch<4>, kWarp * BGK_LINE_WARPS,
                                                      BGK_LINE_WARPS * sizeof(LineWarp<4>));
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
    const int ctas = (line_tasks<N1>(A) + BGK_LINE_WARPS - 1) / BGK_LINE_WARPS;
    const size_t smem = BGK_LINE_WARPS * sizeof(LineWarp<N1>);
    if (mode == 0)
        k_stage1d<N1, 0><<<ctas, kWarp * BGK_LINE_WARPS, smem, s>>>(A);
    else
        k_stage1d<N1, 1><<<ctas, kWarp * BGK_LINE_WARPS, smem, s>>>(A);
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
        return cudaSuccess;  // the line kernels stay within the default dynamic shared memory
    } else if (dim == 2 && p >= 1 && p <= 3) {
        return cudaSuccess;  // the quadrilateral kernels use static shared memory only
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
