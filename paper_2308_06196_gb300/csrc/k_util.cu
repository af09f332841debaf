// k_util.cu -- set-up and data-movement kernels of libbgk: sampling the initial Maxwellian into the
// device layout, and converting f between the host order [point][velocity] (FP64) and the device
// tile layout f[vt][e][i][lane] (FP32).
#include "bgk_common.cuh"

namespace bgk {

// Sample the continuous Maxwellian (Sec. 2, Eq. 4, velocity dimension m = 3, or 2 when nz = 1: the
// one z node has factor 1 and U_z takes no part) of every point's primitive state into f. One CTA per
// element: the separable factors exp(-(xi_d - U_d)^2 / (2 theta)) of the element's points are tabulated
// once in shared memory as FP32 (the exponent in FP64, split into an integer power of two and a
// remainder in [-1/2, 1/2] whose 2^r is taken in FP32: within a few FP32 ulp at any exponent), then every
// (tile, node, lane) value is the product C * Ex * Ey * Ez. Writes 0 on padded slots.
// Q (when not null): the discrete moments (Eq. 2 with Eq. 12) of every point's sampled Maxwellian in
// FP64, from the 1-D trapezoid sums of its tabulated factors (the grid is a tensor product): they differ
// from the moments of the stored FP32 values only by the rounding of the products.
__device__ __forceinline__ float exp_split(double x)
{
    const double y = x * 1.4426950408889634;  // log2(e)
    const double n = rint(y);
    return ldexpf(exp2f((float)(y - n)), (int)n);
}

// Resident CTAs per SM the register allocation is sized for (4, 5 and 6 measured within 2 % of each other)
#ifndef BGK_INIT_MINCTAS
#define BGK_INIT_MINCTAS 5
#endif

__global__ void __launch_bounds__(256, BGK_INIT_MINCTAS)
    k_init_maxwellian(float *__restrict__ f, const double *__restrict__ prim, const float *__restrict__ mi,
                      const float *__restrict__ gmask, int nslots, int nvt, int E, int NP, int nx, int ny, int nz,
                      double v0x, double v0y, double v0z, double dvx, double dvy, double dvz, int *err,
                      double *__restrict__ Q, double *__restrict__ warm)
{
    const double hm = nz == 1 ? 1.0 : 1.5;  // m / 2
    extern __shared__ double ith[];          // [NP] -1 / (2 theta) of the element's points, then
    float *tab = reinterpret_cast<float *>(ith + NP);  // [NP][nx + ny + nz + 1]
    const int e = blockIdx.x;
    const int ntab = nx + ny + nz + 1;
    // per point: the normalisation rho (2 pi theta)^(-m/2) and -1 / (2 theta) (one division per point)
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        const double *s = prim + ((int64_t)e * NP + i) * 5;
        const double rho = s[0], th = s[4];
        const bool ok = rho > 0.0 && th > 0.0;
        if (!ok)
            atomicOr(err, kErrDomain);
        ith[i] = ok ? -0.5 / th : 0.0;
        const double C = rho * pow(2.0 * 3.14159265358979323846 * th, -hm);
        tab[i * ntab] = ok ? (float)C : 0.f;
        if (warm && ok) {  // the first Newton solve's start: this Maxwellian, (ln C, U, theta)
            double *wp = warm + ((int64_t)e * NP + i) * 5;
            wp[0] = log(C);
            wp[1] = s[1];
            wp[2] = s[2];
            wp[3] = nz == 1 ? 0.0 : s[3];
            wp[4] = th;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NP * (ntab - 1); q += blockDim.x) {
        const int i = q / (ntab - 1), t = 1 + q % (ntab - 1);
        const double *s = prim + ((int64_t)e * NP + i) * 5;
        const double a = ith[i];
        float v;
        if (t <= nx) {
            const double c = v0x + (t - 1) * dvx - s[1];
            v = exp_split(a * c * c);
        } else if (t <= nx + ny) {
            const double c = v0y + (t - 1 - nx) * dvy - s[2];
            v = exp_split(a * c * c);
        } else if (nz == 1) {
            v = 1.f;
        } else {
            const double c = v0z + (t - 1 - nx - ny) * dvz - s[3];
            v = exp_split(a * c * c);
        }
        tab[i * ntab + t] = a == 0.0 ? 0.f : v;
    }
    __syncthreads();
    if (Q)
        for (int i = threadIdx.x; i < NP; i += blockDim.x) {
            const float *t = tab + i * ntab;
            const int n[3] = {nx, ny, nz};
            const double v0[3] = {v0x, v0y, v0z}, dv[3] = {dvx, dvy, dvz};
            double S[3][3];
            int off = 1;
            for (int d = 0; d < 3; d++) {
                S[d][0] = S[d][1] = S[d][2] = 0.0;
                if (n[d] == 1) {  // the absent u_z: one node at 0 of unit weight
                    S[d][0] = (double)t[off];
                } else {
                    for (int k = 0; k < n[d]; k++) {
                        const double x = v0[d] + k * dv[d];
                        const double a = (k == 0 || k == n[d] - 1 ? 0.5 * dv[d] : dv[d]) * (double)t[off + k];
                        S[d][0] += a;
                        S[d][1] = fma(x, a, S[d][1]);
                        S[d][2] = fma(x * x, a, S[d][2]);
                    }
                }
                off += n[d];
            }
            const double C = (double)t[0];
            double *q = Q + ((int64_t)e * NP + i) * 5;
            q[0] = C * S[0][0] * S[1][0] * S[2][0];
            q[1] = C * S[0][1] * S[1][0] * S[2][0];
            q[2] = C * S[0][0] * S[1][1] * S[2][0];
            q[3] = C * S[0][0] * S[1][0] * S[2][1];
            q[4] = 0.5 * C * (S[0][2] * S[1][0] * S[2][0] + S[0][0] * S[1][2] * S[2][0] + S[0][0] * S[1][0] * S[2][2]);
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // the tile's table columns (1 + k_x, 1 + n_x + k_y, 1 + n_x + n_y + k_z) from the centred index table
    // (k_d = (m_d + n_d - 1) / 2, exact) and its mask; the next tile's are loaded while this one is written
    auto slot_cols = [&](int vt, int &cx, int &cy, int &cz, float &gm) {
        const int slot = vt * kWarp + lane;
        cx = 1 + __float2int_rn(0.5f * (__ldg(mi + slot) + (float)(nx - 1)));
        cy = 1 + nx + __float2int_rn(0.5f * (__ldg(mi + nslots + slot) + (float)(ny - 1)));
        cz = 1 + nx + ny + __float2int_rn(0.5f * (__ldg(mi + 2 * nslots + slot) + (float)(nz - 1)));
        gm = __ldg(gmask + slot);
    };
    int cx, cy, cz;
    float gm;
    slot_cols(0, cx, cy, cz, gm);
    for (int vt = 0; vt < nvt; vt++) {
        int nx_, ny_, nz_;
        float ngm;
        if (vt + 1 < nvt)
            slot_cols(vt + 1, nx_, ny_, nz_, ngm);
        float *dst = f + fidx(vt, e, 0, lane, E, NP);
#pragma unroll 4
        for (int i = w; i < NP; i += nw) {
            const float *t = tab + i * ntab;
            __stcs(dst + i * kWarp, gm * (t[0] * t[cx] * t[cy] * t[cz]));
        }
        if (vt + 1 < nvt) {
            cx = nx_;
            cy = ny_;
            cz = nz_;
            gm = ngm;
        }
    }
}

// f (device tiles, FP32) <- host-order staging [pt - p0][k] (FP64) for points [p0, p0 + npt)
__global__ void k_scatter_f(float *__restrict__ f, const double *__restrict__ st, const int *__restrict__ slotk,
                            int nvt, int E, int NP, int64_t nvel, int p0, int npt)
{
    const int64_t n = (int64_t)nvt * npt * kWarp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int pl = (int)((q / kWarp) % npt);
        const int vt = (int)(q / ((int64_t)kWarp * npt));
        const int k = __ldg(slotk + vt * kWarp + lane);
        const int pt = p0 + pl;
        f[fidx(vt, pt / NP, pt % NP, lane, E, NP)] = k < 0 ? 0.f : (float)st[(int64_t)pl * nvel + k];
    }
}

// host-order staging [pt - p0][k] (FP64) <- f (device tiles)
__global__ void k_gather_f(double *__restrict__ st, const float *__restrict__ f, const int *__restrict__ slotk,
                           int nvt, int E, int NP, int64_t nvel, int p0, int npt)
{
    const int64_t n = (int64_t)nvt * npt * kWarp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int pl = (int)((q / kWarp) % npt);
        const int vt = (int)(q / ((int64_t)kWarp * npt));
        const int k = __ldg(slotk + vt * kWarp + lane);
        if (k < 0)
            continue;
        const int pt = p0 + pl;
        st[(int64_t)pl * nvel + k] = (double)f[fidx(vt, pt / NP, pt % NP, lane, E, NP)];
    }
}

cudaError_t launch_init_maxwellian(float *f, const double *prim, const float *mi, const float *gmask, int nslots,
                                   int nvt, int E, int NP, const int n[3], const double v0[3], const double dv[3],
                                   int *err, double *Q, double *warm, cudaStream_t s)
{
    const int smem = NP * (int)sizeof(double) + NP * (n[0] + n[1] + n[2] + 1) * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_init_maxwellian, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    k_init_maxwellian<<<E, 256, smem, s>>>(f, prim, mi, gmask, nslots, nvt, E, NP, n[0], n[1], n[2], v0[0], v0[1],
                                           v0[2], dv[0], dv[1], dv[2], err, Q, warm);
    return cudaGetLastError();
}

// Largest |a - b| and |b| over the real slots of two distributions stored in the same tile layout
// (each FP32 or FP64): out[0], out[1] hold the bit patterns of the two non-negative doubles, which
// order like the unsigned integers (atomicMax).
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_f_distance(const TA *__restrict__ a, const TB *__restrict__ b,
                                                    const int *__restrict__ slotk, int64_t n, int per_tile,
                                                    unsigned long long *out)
{
    double d = 0.0, m = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(q % kWarp);
        const int vt = (int)(q / per_tile);
        if (__ldg(slotk + vt * kWarp + lane) < 0)
            continue;
        const double x = (double)a[q], y = (double)b[q];
        d = fmax(d, fabs(x - y));
        m = fmax(m, fabs(y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(d));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(m));
    }
}

cudaError_t launch_f_distance(const void *a, bool a64, const void *b, bool b64, const int *slotk, int nvt, int E,
                              int NP, unsigned long long *out, cudaStream_t s)
{
    const int64_t n = (int64_t)nvt * E * NP * kWarp;
    const int per_tile = E * NP * kWarp;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 16);
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess)
        return e;
    if (a64 && b64)
        k_f_distance<<<blocks, threads, 0, s>>>((const double *)a, (const double *)b, slotk, n, per_tile, out);
    else if (a64)
        k_f_distance<<<blocks, threads, 0, s>>>((const double *)a, (const float *)b, slotk, n, per_tile, out);
    else if (b64)
        k_f_distance<<<blocks, threads, 0, s>>>((const float *)a, (const double *)b, slotk, n, per_tile, out);
    else
        k_f_distance<<<blocks, threads, 0, s>>>((const float *)a, (const float *)b, slotk, n, per_tile, out);
    return cudaGetLastError();
}

cudaError_t launch_convert_f(bool to_device, float *f, double *st, const int *slotk, int nvt, int E, int NP,
                             int64_t nvel, int p0, int npt, cudaStream_t s)
{
    const int64_t n = (int64_t)nvt * npt * kWarp;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 64);
    if (to_device)
        k_scatter_f<<<blocks, threads, 0, s>>>(f, st, slotk, nvt, E, NP, nvel, p0, npt);
    else
        k_gather_f<<<blocks, threads, 0, s>>>(st, f, slotk, nvt, E, NP, nvel, p0, npt);
    return cudaGetLastError();
}

}  // namespace bgk
