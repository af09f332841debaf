// stage_common.cuh -- device helpers shared by the stage kernels (line and hexahedron forms).
#pragma once
#include "bgk_common.cuh"

namespace bgk {

// fused multiply-add on two packed FP32 lanes (sm_100+): d = a * b + c, element-wise
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float sum2(unsigned long long v)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Upwind neighbour of element (ec) in direction d: returns its index, -1 when the face is a Dirichlet or
// diffuse-wall boundary (then the ghost table supplies the upwind value), or kHaloNeighbour when it is
// an exchange face (the neighbour is the element across it in the halo of that face).
constexpr int kHaloNeighbour = -2;
__device__ __forceinline__ int upwind_neighbour(const Mesh &m, const int ec[3], int d, bool left)
{
    int c[3] = {ec[0], ec[1], ec[2]};
    c[d] += left ? -1 : 1;
    if (c[d] < 0 || c[d] >= m.ne[d]) {
        const int b = m.bc[2 * d + (left ? 0 : 1)];
        if (b == 3)
            return kHaloNeighbour;
        if (b != 0)
            return -1;
        c[d] = (c[d] + m.ne[d]) % m.ne[d];
    }
    return c[0] + m.ne[0] * (c[1] + m.ne[1] * c[2]);
}

// The 1-D line computation shared by the three directions: for the line values fl (inflow end R,
// upwind trace T) returns s_i = sum_{j != R} Dm[i][j] (f_j - f_R) + g_i (T - f_R) for all nodes i
// (Dm = D - g (x) l, the derivative with the interior trace folded in; d f_i/dt gains cd * s_i).
template <int N1, bool LEFT>
__device__ __forceinline__ void line_sums(float (&s)[N1], const float (&fl)[N1], float T, const Ops &op)
{
    constexpr int R = LEFT ? 0 : N1 - 1;
    const float fr = fl[R];
    const float tr = T - fr;
    float G[N1];
#pragma unroll
    for (int j = 0; j < N1; j++)
        G[j] = fl[j] - fr;
#pragma unroll
    for (int i = 0; i < N1; i++) {
        float v = (LEFT ? op.gl[i] : op.gr[i]) * tr;
#pragma unroll
        for (int j = 0; j < N1; j++)
            if (j != R)
                v = fmaf(LEFT ? op.DL[i][j] : op.DR[i][j], G[j], v);
        s[i] = v;
    }
}

// line_sums with the jump tr = T - f_R at the inflow face given (see trace_jump)
template <int N1, bool LEFT>
__device__ __forceinline__ void line_sums_jump(float (&s)[N1], const float (&fl)[N1], float tr, const Ops &op)
{
    constexpr int R = LEFT ? 0 : N1 - 1;
    const float fr = fl[R];
    float G[N1];
#pragma unroll
    for (int j = 0; j < N1; j++)
        G[j] = fl[j] - fr;
#pragma unroll
    for (int i = 0; i < N1; i++) {
        float v = (LEFT ? op.gl[i] : op.gr[i]) * tr;
#pragma unroll
        for (int j = 0; j < N1; j++)
            if (j != R)
                v = fmaf(LEFT ? op.DL[i][j] : op.DR[i][j], G[j], v);
        s[i] = v;
    }
}

// The jump T - f_R between the upwind neighbour line v's trace (a left neighbour at its +1 end, a right
// one at its -1 end) and this line's inflow value fr, in difference form: (v_0 - f_R) + sum_{j>=1}
// l_j (v_j - v_0), exactly 0 when both lines hold one constant.
template <int N1, bool LEFT>
__device__ __forceinline__ float trace_jump(const float (&v)[N1], float fr, const Ops &op)
{
    float t = v[0] - fr;
#pragma unroll
    for (int j = 1; j < N1; j++)
        t = fmaf(LEFT ? op.lp[j] : op.lm[j], v[j] - v[0], t);
    return t;
}

// line_sums_jump and trace_jump on two lines at once (the two halves of packed FP32 pairs), for lines
// of one direction that share the operator: every step is one f32x2 instruction on both lines.
__device__ __forceinline__ unsigned long long dup2(float c) { return pack2(c, c); }

template <int N1, bool LEFT>
__device__ __forceinline__ unsigned long long trace_jump2(const unsigned long long (&v)[N1], unsigned long long fr,
                                                          const Ops &op)
{
    unsigned long long t = fsub2(v[0], fr);
#pragma unroll
    for (int j = 1; j < N1; j++)
        t = ffma2(dup2(LEFT ? op.lp[j] : op.lm[j]), fsub2(v[j], v[0]), t);
    return t;
}

template <int N1, bool LEFT>
__device__ __forceinline__ void line_sums_jump2(unsigned long long (&s)[N1], const unsigned long long (&fl)[N1],
                                                unsigned long long tr, const Ops &op)
{
    constexpr int R = LEFT ? 0 : N1 - 1;
    unsigned long long G[N1];
#pragma unroll
    for (int j = 0; j < N1; j++)
        G[j] = fsub2(fl[j], fl[R]);
#pragma unroll
    for (int i = 0; i < N1; i++) {
        unsigned long long v = fmul2(dup2(LEFT ? op.gl[i] : op.gr[i]), tr);
#pragma unroll
        for (int j = 0; j < N1; j++)
            if (j != R)
                v = ffma2(dup2(LEFT ? op.DL[i][j] : op.DR[i][j]), G[j], v);
        s[i] = v;
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

// 2^(x + j) in FP32 arithmetic for an integer j carried in the rounding constant kmagic = 1.5 * 2^23 + j
// (the BGK Maxwellian: j is the integer part of the point's exponent, x the velocity-dependent rest,
// so the FP32 rounding of x is relative to a small number). x = n + r with n = rint(x) (the low bits of
// x + kmagic hold n + j) and |r| <= 1/2; 2^r by a degree-6 polynomial fitted by weighted least squares
// to 2^r on [-1/2, 1/2] in FP64 (coefficients from exp2_fit.py, rounded to FP32); 2^(n + j) added to
// the exponent field. Relative error below 8e-8, with a mean over any unit interval of x below 1e-9:
// the mean matters, because every relaxation step moves the moments of f by (dt / tau) times the mean
// error of g, and the special-function unit's 2^x has a mean error near -5e-8. x is clamped at -100
// (g below 2^(j - 100), of no weight); |j| <= 20 keeps n + j inside the normal range.
__device__ __forceinline__ float exp2_fp32(float x, float kmagic)
{
    x = fmaxf(x, -100.0f);
    const float t = __fadd_rn(x, kmagic);
    const float r = __fsub_rn(x, __fsub_rn(t, kmagic));
    float p = 1.533757750e-04f;
    p = fmaf(p, r, 1.339985989e-03f);
    p = fmaf(p, r, 9.618519805e-03f);
    p = fmaf(p, r, 5.550329015e-02f);
    p = fmaf(p, r, 2.402264625e-01f);
    p = fmaf(p, r, 6.931471825e-01f);
    p = fmaf(p, r, 1.0f);
    // the low bits of t hold n + j (two's complement); shifting them into the exponent field scales
    return __int_as_float(__float_as_int(p) + (__float_as_int(t) << 23));
}

// exp2_fp32 of two values at once, every step on packed FP32 pairs (the same coefficients, duplicated).
// x holds the two arguments, kmagic their two rounding constants.
__device__ __forceinline__ void exp2_fp32x2(unsigned long long x, unsigned long long kmagic, float &y0, float &y1)
{
    float x0, x1;
    unpack2(x, x0, x1);
    const unsigned long long xc = pack2(fmaxf(x0, -100.0f), fmaxf(x1, -100.0f));
    const unsigned long long t = fadd2(xc, kmagic);
    const unsigned long long r = fsub2(xc, fsub2(t, kmagic));
    float t0, t1;
    unpack2(t, t0, t1);
    // the polynomial on the packed pair (coefficient pairs as 64-bit immediates)
    unsigned long long pp = pack2(1.533757750e-04f, 1.533757750e-04f);
    pp = ffma2(pp, r, pack2(1.339985989e-03f, 1.339985989e-03f));
    pp = ffma2(pp, r, pack2(9.618519805e-03f, 9.618519805e-03f));
    pp = ffma2(pp, r, pack2(5.550329015e-02f, 5.550329015e-02f));
    pp = ffma2(pp, r, pack2(2.402264625e-01f, 2.402264625e-01f));
    pp = ffma2(pp, r, pack2(6.931471825e-01f, 6.931471825e-01f));
    pp = ffma2(pp, r, pack2(1.0f, 1.0f));
    float p0, p1;
    unpack2(pp, p0, p1);
    y0 = __int_as_float(__float_as_int(p0) + (__float_as_int(t0) << 23));
    y1 = __int_as_float(__float_as_int(p1) + (__float_as_int(t1) << 23));
}

// Upwind trace of one neighbour line v (difference form, exact for a constant state): a left
// neighbour is evaluated at its +1 end (lp), a right neighbour at its -1 end (lm).
template <int N1, bool LEFT>
__device__ __forceinline__ float trace_line(const float (&v)[N1], const Ops &op)
{
    float t = 0.f;
#pragma unroll
    for (int j = 1; j < N1; j++)
        t = fmaf(LEFT ? op.lp[j] : op.lm[j], v[j] - v[0], t);
    return v[0] + t;
}

}  // namespace bgk

namespace bgk {

// ------------------------------------------------------------------------------------------------
// Bulk asynchronous copies (global -> this CTA's shared memory) completed on an mbarrier. One lane
// arms the barrier with the bytes it is about to copy and issues the copies; every lane that reads
// the data waits on the barrier's phase first. Source and destination are 16-byte aligned and every
// size is a multiple of 16 bytes (rows of 32 floats).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// makes barrier initialisations visible to the asynchronous (bulk-copy) proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier generic-proxy shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// the same with a suspend-time hint: a thread whose phase is not complete sleeps in hardware until it
// completes or hint_ns nanoseconds pass, instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of phase `parity`: one plain test, then up to 10^4 sleeping tries of
// at most 100 us each (about a second in all). After that the timeout bit of the status word is set,
// so that a copy that never lands cannot hang the GPU; the kernel carries on with whatever the buffer
// holds (its results are then void and the host reports BGK_ETIMEOUT).
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, int *err)
{
    if (mbar_try_wait(bar, parity))
        return;
    for (int i = 0; i < 10000; i++)
        if (mbar_try_wait_sleep(bar, parity, 100000u))
            return;
    if (err)
        atomicOr(err, kErrTimeout);
}

}  // namespace bgk
