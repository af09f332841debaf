// k_plain64.cu -- the plain all-FP64 form of the stage: f stored and advected in FP64, unfused.
//
// Per stage and velocity chunk, k64_stage computes every degree of freedom independently (thread per
// (tile, element, node, lane)): it reads the lines through its node and the upwind neighbour's lines
// from global memory, forms the FR derivative with the upwind flux (Sec. 2.1, Eqs. 7-9) in the
// textbook form sum_j D_ij xi f_j + (F_up - xi f_trace) g'_i, evaluates the conservative Maxwellian
// with an FP64 exponential (Sec. 2, Eq. 4) and combines the Shu-Osher stage. k64_moments then sums
// the FP64 moments of the stage output over all chunks (warp per point), and the shared Newton kernel
// solves for the next Maxwellian from those FP64 moments. It is the straightforward comparison form:
// no fusion, no FP32, no shared-memory tiling.
#include <algorithm>

#include "bgk_common.cuh"

namespace bgk {

// The exterior trace at face (d, side) of element e for the face point fp of the line whose own first
// node is i0 (stride along d): the neighbour's interpolant at the shared face (structured grid or the
// connectivity table), or the face's ghost (times the wall density on a diffuse wall).
__device__ double exterior64(const Stage64Args &A, int vl, int e, const int ec[3], int d, int side, int fp, int i0,
                             int lane, int slot)
{
    const int N1 = A.N1, NQ = N1 * N1, E = A.mesh.nelem, NP = A.NP;
    const int stride = d == 0 ? 1 : (d == 1 ? N1 : NQ);
    int en, g, base, str, wall = -1;
    bool hi;  // the neighbour's shared face is its +1 end
    if (A.ftab) {
        const int4 t = A.ftab[(int64_t)e * 6 + 2 * d + side];
        en = t.x;
        g = -1 - t.x;
        str = t.y;
        hi = t.z != 0;
        wall = t.w;
        base = A.fbase[((int64_t)e * 6 + 2 * d + side) * NQ + fp];
    } else {
        int nc[3] = {ec[0], ec[1], ec[2]};
        nc[d] += side ? 1 : -1;
        g = 2 * d + side;
        en = -1;
        if (nc[d] < 0 || nc[d] >= A.mesh.ne[d]) {
            if (A.mesh.bc[g] == 0)
                nc[d] = (nc[d] + A.mesh.ne[d]) % A.mesh.ne[d];
        }
        if (nc[d] >= 0 && nc[d] < A.mesh.ne[d])
            en = nc[0] + A.mesh.ne[0] * (nc[1] + A.mesh.ne[1] * nc[2]);
        str = stride;
        hi = side == 0;
        base = i0;
    }
    if (en < 0) {
        double up = A.ghost[(int64_t)g * A.nslots + slot];
        if (A.ftab) {
            if (wall >= 0)  // a wall face of the unstructured mesh
                up *= A.rhowu[(int64_t)wall * NQ + fp];
        } else if (A.mesh.bc[g] == 2) {
            up *= A.rhow[((int64_t)g * A.nfmax + face_elem(A.mesh, ec, d)) * NQ + fp];
        }
        return up;
    }
    double t = 0.0;
    for (int j = 0; j < N1; j++)
        t += (hi ? A.ops.lp[j] : A.ops.lm[j]) * A.src[fidx(vl, en, base + j * str, lane, E, NP)];
    return t;
}

// Curvilinear residual of one degree of freedom (node i of element e, one velocity): per direction the
// nodal fluxes F_j = (Ja^d(node_j) . xi) f_j along the line, D F, and the FR corrections with the upwind
// common fluxes of the shared face normals at both ends; -(sum over directions) / J.
__device__ double curved_residual64(const Stage64Args &A, int vl, int e, int i, int lane, int slot, const int ec[3],
                                    const int ic[3], const double xi[3])
{
    const int N1 = A.N1, NQ = N1 * N1, E = A.mesh.nelem, NP = A.NP;
    double R = 0.0;
    for (int d = 0; d < 3; d++) {
        const int stride = d == 0 ? 1 : (d == 1 ? N1 : NQ);
        const int i0 = i - ic[d] * stride;
        const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
        const int fp = ic[o1] + N1 * ic[o2];
        double dsum = 0.0, FL = 0.0, FR = 0.0, fL = 0.0, fR = 0.0;
        for (int j = 0; j < N1; j++) {
            const int node = i0 + j * stride;
            const double *ja = A.ja + (((int64_t)e * NP + node) * 3 + d) * 3;
            const double fj = A.src[fidx(vl, e, node, lane, E, NP)];
            const double Fj = (ja[0] * xi[0] + ja[1] * xi[1] + ja[2] * xi[2]) * fj;
            dsum += A.ops.D[ic[d]][j] * Fj;
            FL += A.ops.lm[j] * Fj;
            FR += A.ops.lp[j] * Fj;
            fL += A.ops.lm[j] * fj;
            fR += A.ops.lp[j] * fj;
        }
        const double *nL = A.fnm + ((((int64_t)e * 3 + d) * 2 + 0) * NQ + fp) * 3;
        const double *nR = A.fnm + ((((int64_t)e * 3 + d) * 2 + 1) * NQ + fp) * 3;
        const double uL = nL[0] * xi[0] + nL[1] * xi[1] + nL[2] * xi[2];
        const double uR = nR[0] * xi[0] + nR[1] * xi[1] + nR[2] * xi[2];
        const double FIL = uL > 0.0 ? uL * exterior64(A, vl, e, ec, d, 0, fp, i0, lane, slot) : uL * fL;
        const double FIR = uR < 0.0 ? uR * exterior64(A, vl, e, ec, d, 1, fp, i0, lane, slot) : uR * fR;
        R -= dsum + (FIL - FL) * A.ops.gl[ic[d]] + (FIR - FR) * A.ops.gr[ic[d]];
    }
    return R * A.ijac[(int64_t)e * NP + i];
}

__global__ void __launch_bounds__(256) k64_stage(const Stage64Args A)
{
    const int NP = A.NP, N1 = A.N1, E = A.mesh.nelem, dim = A.mesh.dim;
    const int64_t n = (int64_t)A.nvt * E * NP * kWarp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int i = (int)((q / kWarp) % NP);
        const int e = (int)((q / ((int64_t)kWarp * NP)) % E);
        const int vl = (int)(q / ((int64_t)kWarp * NP * E));
        const int slot = (A.vt0 + vl) * kWarp + lane;
        const int ec[3] = {e % A.mesh.ne[0], (e / A.mesh.ne[0]) % A.mesh.ne[1], e / (A.mesh.ne[0] * A.mesh.ne[1])};
        const int ic[3] = {i % N1, (i / N1) % N1, i / (N1 * N1)};
        const double fs = A.src[q];
        double R = 0.0;
        double xi[3];
        for (int d = 0; d < 3; d++)
            xi[d] = A.xi[d * A.nslots + slot];
        if (A.ja) {  // curvilinear hexahedra: the reference-space flux (Ja^d . xi) f over J
            R = curved_residual64(A, vl, e, i, lane, slot, ec, ic, xi);
            goto have_R;
        }
        for (int d = 0; d < dim; d++) {
            const double a = xi[d];
            const bool left = a >= 0.0;
            const int stride = d == 0 ? 1 : (d == 1 ? N1 : N1 * N1);
            const int i0 = i - ic[d] * stride;  // node of this line at position 0
            double dsum = 0.0, tr = 0.0;
            for (int j = 0; j < N1; j++) {
                const double fj = A.src[fidx(vl, e, i0 + j * stride, lane, E, NP)];
                dsum += A.ops.D[ic[d]][j] * fj;
                tr += (left ? A.ops.lm[j] : A.ops.lp[j]) * fj;
            }
            // upwind neighbour (periodic wrap) or the ghost value of a Dirichlet face
            int nc[3] = {ec[0], ec[1], ec[2]};
            nc[d] += left ? -1 : 1;
            double up;
            if (nc[d] < 0 || nc[d] >= A.mesh.ne[d]) {
                const int fc = 2 * d + (left ? 0 : 1);
                if (A.mesh.bc[fc] != 0) {
                    up = A.ghost[fc * A.nslots + slot];
                    if (A.mesh.bc[fc] == 2) {  // diffuse wall: density of this face point
                        const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
                        const int fnode = ic[o1] + N1 * ic[o2];
                        up *= A.rhow[((int64_t)fc * A.nfmax + face_elem(A.mesh, ec, d)) * N1 * N1 + fnode];
                    }
                    goto have_up;
                }
                nc[d] = (nc[d] + A.mesh.ne[d]) % A.mesh.ne[d];
            }
            {
                const int en = nc[0] + A.mesh.ne[0] * (nc[1] + A.mesh.ne[1] * nc[2]);
                up = 0.0;
                for (int j = 0; j < N1; j++)
                    up += (left ? A.ops.lp[j] : A.ops.lm[j]) * A.src[fidx(vl, en, i0 + j * stride, lane, E, NP)];
            }
        have_up:
            const double corr = (left ? A.ops.gl[ic[d]] : A.ops.gr[ic[d]]) * (a * up - a * tr);
            R -= (2.0 / A.h[d]) * (a * dsum + corr);
        }
    have_R:
        // conservative Maxwellian of this point, BGK relaxation and the Shu-Osher combination
        const double *p = A.par + ((int64_t)e * NP + i) * 5;
        const double r2 = (xi[0] - p[1]) * (xi[0] - p[1]) + (xi[1] - p[2]) * (xi[1] - p[2]) + (xi[2] - p[3]) * (xi[2] - p[3]);
        const double g = A.gmask[slot] * p[0] * exp(-r2 * p[4]);
        double src = (g - fs) * (A.itau ? A.itau[(int64_t)e * NP + i] : A.inv_tau);
        if (A.fpar) {  // body-force source g (q0 + q . xi + q4 |xi|^2)
            const double *q = A.fpar + ((int64_t)e * NP + i) * 5;
            src += g * (q[0] + q[1] * xi[0] + q[2] * xi[1] + q[3] * xi[2] + q[4] * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]));
        }
        double out = A.b * (fs + A.dt * (R + src));
        if (A.fn)
            out += A.an * A.fn[q];
        A.dst[q] = out;
    }
}

__global__ void __launch_bounds__(256) k64_moments(const Moments64Args A)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= A.npts)
        return;
    const int e = warp / A.NP, i = warp % A.NP;
    double m[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < A.nchunks; c++)
        for (int vl = 0; vl < A.nvt[c]; vl++) {
            const double v = A.base[c][fidx(vl, e, i, lane, A.E, A.NP)];
            const double *w = A.wpsi + ((int64_t)(A.vt0[c] + vl) * kWarp + lane) * 5;
            for (int q = 0; q < 5; q++)
                m[q] += w[q] * v;
        }
    for (int q = 0; q < 5; q++) {
        double v = m[q];
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        m[q] = v;
    }
    if (lane < 5)
        A.Q[(int64_t)warp * 5 + lane] = m[lane];
}

// Sample the continuous Maxwellian of every point's primitive state into the FP64 layout.
__global__ void k64_init(double *f, const double *prim, const double *xi, const float *gmask, int nvt, int E, int NP,
                         int nslots, int vdim, int *err)
{
    const int64_t n = (int64_t)nvt * E * NP * kWarp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int pt = (int)((q / kWarp) % ((int64_t)E * NP));
        const int vt = (int)(q / ((int64_t)kWarp * NP * E));
        const int slot = vt * kWarp + lane;
        const double *s = prim + (int64_t)pt * 5;
        if (!(s[0] > 0.0) || !(s[4] > 0.0)) {
            if (lane == 0 && vt == 0)
                atomicOr(err, kErrDomain);
            f[q] = 0.0;
            continue;
        }
        double r2 = 0.0;
        for (int d = 0; d < vdim; d++) {  // m = 2: u_z and U_z take no part
            const double c = xi[d * nslots + slot] - s[1 + d];
            r2 += c * c;
        }
        f[q] = gmask[slot] * s[0] * pow(2.0 * 3.14159265358979323846 * s[4], -0.5 * vdim) * exp(-0.5 * r2 / s[4]);
    }
}

// f (device tiles, FP64) <-> host-order staging [pt - p0][k] (FP64)
__global__ void k64_convert(double *f, double *st, const int *slotk, int nvt, int E, int NP, int64_t nvel, int p0,
                            int npt, int to_device)
{
    const int64_t n = (int64_t)nvt * npt * kWarp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int pl = (int)((q / kWarp) % npt);
        const int vt = (int)(q / ((int64_t)kWarp * npt));
        const int k = slotk[vt * kWarp + lane];
        const int pt = p0 + pl;
        double &v = f[fidx(vt, pt / NP, pt % NP, lane, E, NP)];
        if (to_device)
            v = k < 0 ? 0.0 : st[(int64_t)pl * nvel + k];
        else if (k >= 0)
            st[(int64_t)pl * nvel + k] = v;
    }
}

static int grid_for(int64_t n, int threads) { return (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 32); }

// Zhang-Shu positivity limiter on the FP64 stage output (Sec. 2.1, Eqs. 10-11): thread per
// (tile, element, lane); the element mean uses the Gauss-Legendre weights of the nodes.
__global__ void __launch_bounds__(256) k64_limit(double *f, int nvt, int E, int NP, int N1, int dim, Ops64 ops,
                                                 const double *ijac)
{
    const int64_t n = (int64_t)nvt * E * kWarp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int64_t ve = q / kWarp;  // (tile, element)
        double *b = f + ve * NP * kWarp + lane;
        double mean = 0.0, wsum = 0.0, mn = b[0];
        for (int i = 0; i < NP; i++) {
            double w = ops.wq[i % N1];
            if (dim >= 2)
                w *= ops.wq[(i / N1) % N1];
            if (dim >= 3)
                w *= ops.wq[i / (N1 * N1)];
            if (ijac)  // curvilinear: the physical element's mean (weights W J)
                w /= ijac[(ve % E) * NP + i];
            const double v = b[(int64_t)i * kWarp];
            mean += w * v;
            wsum += w;
            mn = fmin(mn, v);
        }
        mean /= wsum;
        if (!(mn < 0.0))
            continue;
        const double beta = fmin(fabs(mean / (mean - mn)), 1.0);
        for (int i = 0; i < NP; i++)
            b[(int64_t)i * kWarp] = mean + beta * (b[(int64_t)i * kWarp] - mean);
    }
}

cudaError_t launch_limit64(double *f, int nvt, int E, int NP, int N1, int dim, const Ops64 &ops, const double *ijac,
                           cudaStream_t s)
{
    const int64_t n = (int64_t)nvt * E * kWarp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k64_limit<<<blocks, 256, 0, s>>>(f, nvt, E, NP, N1, dim, ops, ijac);
    return cudaGetLastError();
}

cudaError_t launch_stage64(const Stage64Args &A, cudaStream_t s)
{
    const int64_t n = (int64_t)A.nvt * A.mesh.nelem * A.NP * kWarp;
    k64_stage<<<grid_for(n, 256), 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_moments64(const Moments64Args &A, cudaStream_t s)
{
    k64_moments<<<(int)(((int64_t)A.npts * kWarp + 255) / 256), 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_init64(double *f, const double *prim, const double *xi, const float *gmask, int nvt, int E, int NP,
                          int nslots, int vdim, int *err, cudaStream_t s)
{
    const int64_t n = (int64_t)nvt * E * NP * kWarp;
    k64_init<<<grid_for(n, 256), 256, 0, s>>>(f, prim, xi, gmask, nvt, E, NP, nslots, vdim, err);
    return cudaGetLastError();
}

cudaError_t launch_convert64(bool to_device, double *f, double *st, const int *slotk, int nvt, int E, int NP,
                             int64_t nvel, int p0, int npt, cudaStream_t s)
{
    const int64_t n = (int64_t)nvt * npt * kWarp;
    k64_convert<<<grid_for(n, 256), 256, 0, s>>>(f, st, slotk, nvt, E, NP, nvel, p0, npt, to_device ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace bgk
