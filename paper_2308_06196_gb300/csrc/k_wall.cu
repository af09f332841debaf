// k_wall.cu -- diffuse-wall densities of one stage.
//
// For every wall face point (a face Gauss-Legendre point of a boundary element on a diffuse-wall
// face), the density of the incoming wall Maxwellian is chosen so that the net discrete mass flux
// through that point vanishes: rho_w = sum_{xi . n_out > 0} w |xi_n| f_trace / sum_{xi . n_out < 0}
// w |xi_n| M_w, where f_trace is the element's own interpolant at the face (the value the FR scheme
// lets out) and M_w the unit-density Maxwellian of the wall (the denominator is fixed per face and
// precomputed on the host). One warp per face point; lanes run over the outgoing velocities of the
// stage source, accumulating in FP64. T is the storage type of f (float or double); the quadrature
// weights and velocities are those the moments use (FP32 tables for the FP32 form). On curved walls
// the normal changes from point to point: both sums are then taken per face point, over all
// velocities, with the outward unit normal of the point.
#include "bgk_common.cuh"

namespace bgk {

template <typename T, typename W>
__global__ void __launch_bounds__(256) k_wall(const WallArgs A, const W *w, const W *xi)
{
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int N1 = A.N1, NQ = N1 * N1, NP = A.NP, E = A.mesh.nelem;
    const int f = gw / (A.nfmax * NQ);
    if (f >= 6 || (A.inv_in[f] == 0.0 && !(A.wn && A.mesh.bc[f] == 2)))
        return;  // whole warp
    const int fe = (gw / NQ) % A.nfmax, fnode = gw % NQ;
    const int d = f >> 1, side = f & 1;
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;  // the two in-face directions
    if (fe >= A.mesh.ne[o1] * A.mesh.ne[o2])
        return;
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
    if (A.wn) {  // curved wall: per-point normal, both sums here
        const double *n = A.wn + (((int64_t)f * A.nfmax + fe) * NQ + fnode) * 4;
        double out = 0.0, in = 0.0;
        for (int c = 0; c < A.nchunks; c++) {
            const T *src = static_cast<const T *>(A.src[c]);
            for (int vl = 0; vl < A.nvt[c]; vl++) {
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
                    in -= (double)w[slot] * un * (double)static_cast<const T *>(A.ghost)[(int64_t)f * A.nslots + slot];
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            out += __shfl_xor_sync(0xffffffffu, out, o);
            in += __shfl_xor_sync(0xffffffffu, in, o);
        }
        if (lane == 0)
            static_cast<T *>(A.rhow)[((int64_t)f * A.nfmax + fe) * NQ + fnode] = (T)(out / in);
        return;
    }
    double sum = 0.0;
    for (int c = 0; c < A.nchunks; c++) {
        const int oc = A.oct[c];
        if (oc < 8 && ((oc >> d) & 1) != side)
            continue;  // no outgoing velocity in this chunk
        const T *src = static_cast<const T *>(A.src[c]);
        for (int vl = 0; vl < A.nvt[c]; vl++) {
            const int slot = (A.vt0[c] + vl) * kWarp + lane;
            const double xn = (double)xi[(int64_t)d * A.nslots + slot];
            if (side ? !(xn > 0.0) : !(xn < 0.0))
                continue;
            const T *b = src + fidx(vl, e, n0, lane, E, NP);
            double t = 0.0;
            for (int j = 0; j < N1; j++)
                t += (side ? A.lp[j] : A.lm[j]) * (double)b[(int64_t)j * stride * kWarp];
            sum += (double)w[slot] * fabs(xn) * t;
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0)
        static_cast<T *>(A.rhow)[((int64_t)f * A.nfmax + fe) * NQ + fnode] = (T)(sum * A.inv_in[f]);
}

// The wall faces of an unstructured mesh (from its list, one warp per face point): the same zero-net-
// mass-flux density with the face point's own outward normal, both sums over all velocities.
template <typename T, typename W>
__global__ void __launch_bounds__(256) k_wall_list(const WallArgs A, const W *w, const W *xi)
{
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int N1 = A.N1, NQ = N1 * N1, NP = A.NP, E = A.mesh.nelem;
    if (gw >= A.nwall * NQ)
        return;  // whole warp
    const int idx = gw / NQ, fnode = gw % NQ;
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
    double out = 0.0, in = 0.0;
    for (int c = 0; c < A.nchunks; c++) {
        const T *src = static_cast<const T *>(A.src[c]);
        for (int vl = 0; vl < A.nvt[c]; vl++) {
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
    for (int o = 16; o > 0; o >>= 1) {
        out += __shfl_xor_sync(0xffffffffu, out, o);
        in += __shfl_xor_sync(0xffffffffu, in, o);
    }
    if (lane == 0)
        static_cast<T *>(A.rhowu)[(int64_t)idx * NQ + fnode] = (T)(out / in);
}

cudaError_t launch_wall(const WallArgs &A, bool fp64, const void *w, const void *xi, cudaStream_t s)
{
    if (A.wlist) {  // unstructured mesh: its wall-face list
        const int64_t warps = (int64_t)A.nwall * A.N1 * A.N1;
        const int blocks = (int)((warps * kWarp + 255) / 256);
        if (fp64)
            k_wall_list<double, double>
                <<<blocks, 256, 0, s>>>(A, static_cast<const double *>(w), static_cast<const double *>(xi));
        else
            k_wall_list<float, float><<<blocks, 256, 0, s>>>(A, static_cast<const float *>(w), static_cast<const float *>(xi));
        return cudaGetLastError();
    }
    const int64_t warps = 6ll * A.nfmax * A.N1 * A.N1;
    const int blocks = (int)((warps * kWarp + 255) / 256);
    if (fp64)
        k_wall<double, double><<<blocks, 256, 0, s>>>(A, static_cast<const double *>(w), static_cast<const double *>(xi));
    else
        k_wall<float, float><<<blocks, 256, 0, s>>>(A, static_cast<const float *>(w), static_cast<const float *>(xi));
    return cudaGetLastError();
}

}  // namespace bgk
