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
#include "stage_common.cuh"

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

cudaError_t prepare_stage3_p1();
cudaError_t prepare_stage3_p2();
cudaError_t prepare_stage3_p3();
cudaError_t launch_stage3_p1(const StageArgs &A, int mode, int oct, cudaStream_t s);
cudaError_t launch_stage3_p2(const StageArgs &A, int mode, int oct, cudaStream_t s);
cudaError_t launch_stage3_p3(const StageArgs &A, int mode, int oct, cudaStream_t s);

template <int N1>
static cudaError_t prepare_1d()
{
    const int smem = (int)sizeof(StageSmem<Geo<N1, 1>::NP>);
    cudaError_t err = cudaFuncSetAttribute(k_stage<N1, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_stage<N1, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return err;
}

template <int N1>
static cudaError_t launch_1d(const StageArgs &A, int mode, cudaStream_t s)
{
    const int nEB = (A.mesh.nelem + kWarpsPerCta - 1) / kWarpsPerCta;
    const int ngroups = (A.nvt + A.G - 1) / A.G;
    dim3 grid(nEB * ngroups), block(kWarp * kWarpsPerCta);
    const int smem = (int)sizeof(StageSmem<Geo<N1, 1>::NP>);
    if (mode == 0)
        k_stage<N1, 1, 0><<<grid, block, smem, s>>>(A);
    else
        k_stage<N1, 1, 1><<<grid, block, smem, s>>>(A);
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
    } else if (dim == 1) {
        switch (p) {
        case 1: return prepare_1d<2>();
        case 2: return prepare_1d<3>();
        case 3: return prepare_1d<4>();
        case 4: return prepare_1d<5>();
        case 5: return prepare_1d<6>();
        }
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
