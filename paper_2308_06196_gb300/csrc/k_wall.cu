// k_wall.cu -- diffuse-wall densities of one stage.
//
// For every wall face point (a face Gauss-Legendre point of a boundary element on a diffuse-wall
// face), the density of the incoming wall Maxwellian is chosen so that the net discrete mass flux
// through that point vanishes: rho_w = sum_{xi . n_out > 0} w |xi_n| f_trace / sum_{xi . n_out < 0}
// w |xi_n| M_w, where f_trace is the element's own interpolant at the face (the value the FR scheme
// lets out) and M_w the unit-density Maxwellian of the wall (the denominator is fixed per face and
// precomputed on the host). One CTA per face point: its warps take every fourth velocity tile, lanes
// run over the tile's outgoing velocities, and the warps' sums are added in a fixed order. T is the
// storage type of f (float or double); the quadrature weights and velocities are those the moments use
// (FP32 tables for the FP32 form). The all-FP64 form sums in FP64; the FP32-split form forms the terms
// in FP32 and sums them in double-float. On curved walls the normal changes from point to point: both
// sums are then taken per face point, over all velocities, with the outward unit normal of the point
// (in FP64). The walls of an unstructured mesh have a kernel of their own over their list.
#include "bgk_common.cuh"

namespace bgk {

// Sum of one face point's flux terms. The all-FP64 form accumulates in FP64; the FP32-split form forms
// each term in FP32 (the precision of the stage kernel's own outgoing flux) and accumulates it in
// double-float, the running FP32 sum and its exact two-sum errors, about 1e-12 relative over any number
// of terms at FP32 throughput.
template <typename T>
struct WallAcc {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ double val() const { return s; }
};
template <>
struct WallAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float x)
    {
        const float t = __fadd_rn(hi, x), bb = __fsub_rn(t, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
        hi = t;
    }
    __device__ double val() const { return (double)hi + (double)lo; }
};

constexpr int kWallWarps = 4;  // warps per face point: tiles vl = w, w + 4, ... of every chunk

// a double from every warp of the CTA, added in warp order (deterministic); the result in thread 0
__device__ __forceinline__ double wall_cta_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kWallWarps; q++)
            s += red[q];
    __syncthreads();
    return s;
}

// Both sums of a face point with its own outward unit normal n (curved walls and the walls of an
// unstructured mesh), in FP64: the outgoing flux of the element's trace along its normal line (nodes
// n0 + j stride of element e, its +1 end when side = 1) and the incoming flux of the unit-density wall
// Maxwellian ghost[g]. This warp takes tiles wq, wq + kWallWarps, ...; returns rho_w in thread 0.
template <typename T, typename W>
__device__ double curved_wall_density(const WallArgs &A, const W *w, const W *xi, const double *n, int e, int side,
                                      int n0, int stride, int g, double *red)
{
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int N1 = A.N1, NP = A.NP, E = A.mesh.nelem;
    double out = 0.0, in = 0.0;
    for (int c = 0; c < A.nchunks; c++) {
        const T *src = static_cast<const T *>(A.src[c]);
        for (int vl = wq; vl < A.nvt[c]; vl += kWallWarps) {
            const int slot = (A.vt0[c] + vl) * kWarp + lane;
            const double un = n[0] * (double)xi[slot] + n[1] * (double)xi[(int64_t)A.nslots + slot] +
                              n[2] * (double)xi[2 * (int64_t)A.nslots + slot];
            if (un > 0.0) {
                const T *b = src + fidx(vl, e, n0, lane, E, NP);
                double t = 0.0;
                for (int j = 0; j < N1; j++)
                    t += (side ? A.lp[j] : A.lm[j]) * (double)b[(int64_t)j * stride * kWarp];
                out += (double)w[slot] * un * t;
            } else if (un < 0.0) {
                in -= (double)w[slot] * un * (double)static_cast<const T *>(A.ghost)[(int64_t)g * A.nslots + slot];
            }
        }
    }
    out = wall_cta_sum(out, red);
    in = wall_cta_sum(in, red);
    return out / in;
}

// One CTA of kWallWarps warps per face point of the structured mesh (a whole CTA returns together).
template <typename T, typename W>
__global__ void __launch_bounds__(kWallWarps * 32) k_wall(const WallArgs A, const W *w, const W *xi)
{
    __shared__ double red[kWallWarps];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int N1 = A.N1, NQ = N1 * N1, NP = A.NP, E = A.mesh.nelem;
    int q = 0;  // the wall face of this CTA's face point
    while (q + 1 < A.nwf && (int)blockIdx.x >= A.wfstart[q + 1])
        q++;
    const int f = A.wf[q], gp = (int)blockIdx.x - A.wfstart[q];
    const int fe = gp / NQ, fnode = gp % NQ;
    const int d = f >> 1, side = f & 1;
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;  // the two in-face directions
    int ec[3];
    ec[d] = side ? A.mesh.ne[d] - 1 : 0;
    ec[o1] = fe % A.mesh.ne[o1];
    ec[o2] = fe / A.mesh.ne[o1];
    const int e = ec[0] + A.mesh.ne[0] * (ec[1] + A.mesh.ne[1] * ec[2]);
    int nc[3];
    nc[o1] = fnode % N1;
    nc[o2] = fnode / N1;
    nc[d] = 0;
    const int n0 = nc[0] + N1 * (nc[1] + N1 * nc[2]);
    const int stride = d == 0 ? 1 : (d == 1 ? N1 : NQ);
    if (A.wn) {  // curved wall: per-point normal, both sums here (FP64)
        const double *n = A.wn + (((int64_t)f * A.nfmax + fe) * NQ + fnode) * 4;
        const double rw = curved_wall_density<T, W>(A, w, xi, n, e, side, n0, stride, f, red);
        if (threadIdx.x == 0)
            static_cast<T *>(A.rhow)[((int64_t)f * A.nfmax + fe) * NQ + fnode] = (T)rw;
        return;
    }
    T l[kMaxN1];
#pragma unroll
    for (int j = 0; j < kMaxN1; j++)
        l[j] = sizeof(T) == 4 ? (T)(side ? A.lpf[j] : A.lmf[j]) : (T)(side ? A.lp[j] : A.lm[j]);
    WallAcc<T> acc;
    for (int c = 0; c < A.nchunks; c++) {
        const int oc = A.oct[c];
        if (oc < 8 && ((oc >> d) & 1) != side)
            continue;  // no outgoing velocity in this chunk
        const T *src = static_cast<const T *>(A.src[c]);
        // branch-free body (the term of a velocity that does not leave is selected away), so that the
        // unrolled iterations' loads are in flight together
#pragma unroll 4
        for (int vl = wq; vl < A.nvt[c]; vl += kWallWarps) {
            const int slot = (A.vt0[c] + vl) * kWarp + lane;
            const T xn = (T)xi[(int64_t)d * A.nslots + slot];
            const T *b = src + fidx(vl, e, n0, lane, E, NP);
            T t = T(0);  // the element's own trace, in the storage precision
#pragma unroll
            for (int j = 0; j < kMaxN1; j++)
                if (j < N1)
                    t += l[j] * b[(int64_t)j * stride * kWarp];
            const bool leaves = side ? xn > T(0) : xn < T(0);
            acc.add(leaves ? (T)w[slot] * (xn < T(0) ? -xn : xn) * t : T(0));
        }
    }
    const double sum = wall_cta_sum(acc.val(), red);
    if (threadIdx.x == 0)
        static_cast<T *>(A.rhow)[((int64_t)f * A.nfmax + fe) * NQ + fnode] = (T)(sum * A.inv_in[f]);
}

// The wall faces of an unstructured mesh (from its list, one CTA of kWallWarps warps per face point):
// the same zero-net-mass-flux density with the face point's own outward normal, both sums over all
// velocities.
template <typename T, typename W>
__global__ void __launch_bounds__(kWallWarps * 32) k_wall_list(const WallArgs A, const W *w, const W *xi)
{
    __shared__ double red[kWallWarps];
    const int N1 = A.N1, NQ = N1 * N1;
    const int idx = (int)blockIdx.x / NQ, fnode = (int)blockIdx.x % NQ;
    const int4 wf = A.wlist[idx];
    const int e = wf.x, d = wf.y >> 1, side = wf.y & 1, g = wf.z;
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    int nc[3];
    nc[o1] = fnode % N1;
    nc[o2] = fnode / N1;
    nc[d] = 0;
    const int n0 = nc[0] + N1 * (nc[1] + N1 * nc[2]);
    const int stride = d == 0 ? 1 : (d == 1 ? N1 : NQ);
    const double *n = A.wnu + ((int64_t)idx * NQ + fnode) * 4;
    const double rw = curved_wall_density<T, W>(A, w, xi, n, e, side, n0, stride, g, red);
    if (threadIdx.x == 0)
        static_cast<T *>(A.rhowu)[(int64_t)idx * NQ + fnode] = (T)rw;
}

cudaError_t launch_wall(const WallArgs &A, bool fp64, const void *w, const void *xi, cudaStream_t s)
{
    if (A.wlist) {  // unstructured mesh: its wall-face list, one CTA per face point
        const int blocks = A.nwall * A.N1 * A.N1;
        if (blocks == 0)
            return cudaSuccess;
        if (fp64)
            k_wall_list<double, double>
                <<<blocks, kWallWarps * 32, 0, s>>>(A, static_cast<const double *>(w), static_cast<const double *>(xi));
        else
            k_wall_list<float, float>
                <<<blocks, kWallWarps * 32, 0, s>>>(A, static_cast<const float *>(w), static_cast<const float *>(xi));
        return cudaGetLastError();
    }
    const int blocks = A.wfstart[A.nwf];  // one CTA per wall face point
    if (blocks == 0)
        return cudaSuccess;
    if (fp64)
        k_wall<double, double>
            <<<blocks, kWallWarps * 32, 0, s>>>(A, static_cast<const double *>(w), static_cast<const double *>(xi));
    else
        k_wall<float, float>
            <<<blocks, kWallWarps * 32, 0, s>>>(A, static_cast<const float *>(w), static_cast<const float *>(xi));
    return cudaGetLastError();
}

}  // namespace bgk
