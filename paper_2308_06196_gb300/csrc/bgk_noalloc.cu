// bgk_noalloc.cu -- bgk_equilibrium_noalloc: the moments + conservative-Maxwellian pass for callers
// that cannot allocate device memory.
//
// Why: some callers cannot call cudaMalloc at all -- for example code that runs inside another
// framework's memory pool or allocator hooks, under a strict no-allocation policy after start-up,
// or in a process that must not grow its device footprint after it has been sized. The regular
// path (bgk_create) allocates its own buffers, so those callers could not use it. This entry point
// allocates nothing: the caller passes device pointers for the input and the outputs, and the only
// scratch (the partial moment sums and the solver's private per-point table) lives in one
// file-scope __device__ array of fixed size. A device holds it from the moment this library's module
// is loaded there until the process exits; under lazy module loading (the CUDA default since 12.2)
// that is the first call of this entry point on the device, which is therefore the sizing point: a
// caller with a fixed footprint makes it during start-up. The call is synchronous (it reads the
// status word back), so it cannot be captured in a CUDA graph; on a capturing stream it returns
// BGK_EINVAL before enqueuing anything.
//
// Scratch layout (floats): [0, 64) status word, then partial sums [ngroups][5][npts], then the
// per-point exponent table [npts][8] written by the Newton kernel.
#include <cstdio>
#include <mutex>

#include "bgk.h"
#include "bgk_common.cuh"

namespace bgk {
cudaError_t launch_newton(const NewtonArgs &A, cudaStream_t s);
}
using namespace bgk;

namespace {

constexpr int64_t kScratchFloats = BGK_NOALLOC_SCRATCH_BYTES / 4;
constexpr int kGroupVel = 2048;   // velocities per partial-sum group
constexpr int kStatusFloats = 64; // status word region (keeps the partials 256-byte aligned)

static __device__ __align__(256) float g_scratch[kScratchFloats];

// Per-device address of g_scratch. Host code must not use the symbol itself: on the host it names
// a stand-in object, not device memory.
std::mutex g_mu;
float *g_ptr[256] = {nullptr};

// Partial grid-index moments sum_k W_k (1, m, sum_d r_d m_d^2) f[pt][k] (the basis of the Newton
// kernel's input, exact FP32 weights) over velocity group blockIdx.y of point blockIdx.x. f is in the
// host order [npts][N_v] with k = kx + nx (ky + ny kz).
__global__ void __launch_bounds__(256) k_noalloc_partials(const float *__restrict__ f, int npts, int nx, int ny,
                                                          int nz, float ry, float rz, float *partial)
{
    const int pt = blockIdx.x, g = blockIdx.y;
    const int64_t nvel = (int64_t)nx * ny * nz;
    const int64_t k0 = (int64_t)g * kGroupVel;
    const int64_t k1 = min(k0 + kGroupVel, nvel);
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const int kx = (int)(k % nx), ky = (int)((k / nx) % ny), kz = (int)(k / ((int64_t)nx * ny));
        const float W = (float)(end_factor(kx, nx) * end_factor(ky, ny) * end_factor(kz, nz));
        const float mx = (float)(2 * kx - (nx - 1)), my = (float)(2 * ky - (ny - 1)), mz = (float)(2 * kz - (nz - 1));
        const float v = __ldg(f + (int64_t)pt * nvel + k);
        m[0] = fmaf(W, v, m[0]);
        m[1] = fmaf(W * mx, v, m[1]);
        m[2] = fmaf(W * my, v, m[2]);
        m[3] = fmaf(W * mz, v, m[3]);
        m[4] = fmaf(W * (mx * mx + ry * (my * my) + rz * (mz * mz)), v, m[4]);
    }
    __shared__ float red[8][5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        float v = m[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0)
            red[threadIdx.x >> 5][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++)
            v += red[w][threadIdx.x];
        partial[((int64_t)g * 5 + threadIdx.x) * npts + pt] = v;
    }
}

}  // namespace

extern "C" int bgk_equilibrium_noalloc(const float *d_f, int64_t npts, const bgk_vgrid *vg, double *d_Q,
                                       double *d_prim, void *stream)
{
    if (!d_f || !vg || !d_Q || !d_prim || npts < 1 || npts > (1 << 30))
        return BGK_EINVAL;
    const int vdim = vg->n[2] == 1 ? 2 : 3;  // n[2] = 1: the two-dimensional velocity space
    bool all_two = true;  // two nodes on every axis: the energy moment depends on the others
    for (int d = 0; d < vdim; d++) {
        if (vg->n[d] < 2 || vg->n[d] > 4096 || !(vg->hi[d] > vg->lo[d]))
            return BGK_EINVAL;
        all_two = all_two && vg->n[d] == 2;
    }
    if (all_two)
        return BGK_EINVAL;
    const int64_t nvel = (int64_t)vg->n[0] * vg->n[1] * vg->n[2];
    const int64_t ng64 = (nvel + kGroupVel - 1) / kGroupVel;
    if (ng64 > 65535) {
        fprintf(stderr, "bgk_equilibrium_noalloc: %lld velocities exceed the 65535 x %d velocity limit\n",
                (long long)nvel, kGroupVel);
        return BGK_EINVAL;
    }
    const int ngroups = (int)ng64;
    const int64_t need = kStatusFloats + npts * (5 * (int64_t)ngroups + kParamStride);
    if (need > kScratchFloats) {
        fprintf(stderr,
                "bgk_equilibrium_noalloc: %lld points x %lld velocities need %lld scratch bytes, more than the "
                "fixed %lld-byte scratch (max points for this grid: %lld)\n",
                (long long)npts, (long long)nvel, (long long)(need * 4), (long long)BGK_NOALLOC_SCRATCH_BYTES,
                (long long)((kScratchFloats - kStatusFloats) / (5 * (int64_t)ngroups + kParamStride)));
        return BGK_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
        return BGK_ECUDA;
    float *scr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            // once per device, with that device current
            float *p = nullptr;
            if (cudaGetSymbolAddress((void **)&p, g_scratch) != cudaSuccess || !p)
                return BGK_ECUDA;
            g_ptr[dev] = p;
        }
        scr = g_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess)
        return BGK_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) {
        fprintf(stderr, "bgk_equilibrium_noalloc: the call is synchronous and cannot be captured in a CUDA graph\n");
        return BGK_EINVAL;
    }
    int *status = reinterpret_cast<int *>(scr);
    float *partial = scr + kStatusFloats;
    float *param = partial + (int64_t)ngroups * 5 * npts;
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
        return BGK_ECUDA;
    double v0[3], dv[3];
    for (int d = 0; d < vdim; d++) {
        v0[d] = vg->lo[d];
        dv[d] = (vg->hi[d] - vg->lo[d]) / (vg->n[d] - 1);
    }
    if (vdim == 2) {  // one node at 0 of unit weight; dv[2] a placeholder equal to dv[0]
        v0[2] = 0.0;
        dv[2] = dv[0];
    }
    dim3 grid((unsigned)npts, (unsigned)ngroups);
    k_noalloc_partials<<<grid, 256, 0, s>>>(d_f, (int)npts, vg->n[0], vg->n[1], vg->n[2], index_r(dv[1], dv[0]),
                                            index_r(dv[2], dv[0]), partial);
    if (cudaGetLastError() != cudaSuccess)
        return BGK_ECUDA;
    NewtonArgs N{};
    N.partial = partial;
    N.ngroups = ngroups;
    N.npts = (int)npts;
    N.Q = d_Q;
    N.prim = d_prim;
    N.param = param;
    N.err = status;
    N.cold = 1;
    N.it32 = 2;
    N.it64 = 1;
    for (int d = 0; d < 3; d++)
        newton_axis(N, d, v0[d], dv[d], vg->n[d]);
    N.vdim = vdim;
    if (launch_newton(N, s) != cudaSuccess)
        return BGK_ECUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return BGK_ECUDA;
    if (h & kErrDomain)
        return BGK_EDOMAIN;
    if (h & kErrNewton)
        return BGK_ENEWTON;
    return BGK_OK;
}
