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
__device__ __forceinline__ float exp_split(double x)
{
    const double y = x * 1.4426950408889634;  // log2(e)
    const double n = rint(y);
    return ldexpf(exp2f((float)(y - n)), (int)n);
}

__global__ void k_init_maxwellian(float *__restrict__ f, const double *__restrict__ prim, const float *__restrict__ mi,
                                  const float *__restrict__ gmask, int nslots, int nvt, int E, int NP, int nx, int ny,
                                  int nz, double v0x, double v0y, double v0z, double dvx, double dvy, double dvz,
                                  int *err)
{
    const double hm = nz == 1 ? 1.0 : 1.5;  // m / 2
    extern __shared__ float tab[];  // [NP][nx + ny + nz + 1]
    const int e = blockIdx.x;
    const int ntab = nx + ny + nz + 1;
    for (int q = threadIdx.x; q < NP * ntab; q += blockDim.x) {
        const int i = q / ntab, t = q % ntab;
        const double *s = prim + ((int64_t)e * NP + i) * 5;
        const double rho = s[0], th = s[4];
        if (!(rho > 0.0) || !(th > 0.0)) {
            tab[q] = 0.f;
            if (t == 0)
                atomicOr(err, kErrDomain);
            continue;
        }
        float v;
        if (t == 0) {
            v = (float)(rho * pow(2.0 * 3.14159265358979323846 * th, -hm));
        } else if (t <= nx) {
            const double c = v0x + (t - 1) * dvx - s[1];
            v = exp_split(-0.5 * c * c / th);
        } else if (t <= nx + ny) {
            const double c = v0y + (t - 1 - nx) * dvy - s[2];
            v = exp_split(-0.5 * c * c / th);
        } else if (nz == 1) {
            v = 1.f;
        } else {
            const double c = v0z + (t - 1 - nx - ny) * dvz - s[3];
            v = exp_split(-0.5 * c * c / th);
        }
        tab[q] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int vt = 0; vt < nvt; vt++) {
        // grid indices k_d = (m_d + n_d - 1) / 2 of the slot from the centred index table (exact)
        const int slot = vt * kWarp + lane;
        const int kx = __float2int_rn(0.5f * (__ldg(mi + slot) + (float)(nx - 1)));
        const int ky = __float2int_rn(0.5f * (__ldg(mi + nslots + slot) + (float)(ny - 1)));
        const int kz = __float2int_rn(0.5f * (__ldg(mi + 2 * nslots + slot) + (float)(nz - 1)));
        const float gm = __ldg(gmask + slot);
        for (int i = w; i < NP; i += nw) {
            const float *t = tab + i * ntab;
            const float v = gm * (t[0] * t[1 + kx] * t[1 + nx + ky] * t[1 + nx + ny + kz]);
            __stcs(f + fidx(vt, e, i, lane, E, NP), v);
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
                                   int *err, cudaStream_t s)
{
    const int smem = NP * (n[0] + n[1] + n[2] + 1) * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_init_maxwellian, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    k_init_maxwellian<<<E, 256, smem, s>>>(f, prim, mi, gmask, nslots, nvt, E, NP, n[0], n[1], n[2], v0[0], v0[1],
                                           v0[2], dv[0], dv[1], dv[2], err);
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
