// k_newton.cu -- per-point discretely-conservative Maxwellian (Sec. 2.1, text after Eq. 13).
//
// For every spatial point the kernel
//   1. sums the FP32 partial moments of all velocity tasks exactly (double-float accumulation) and
//      maps these grid-index moments to Q = sum_k w_k psi_k f_k in FP64 (Eq. 2 with the trapezoid
//      operator of Eq. 12),
//   2. finds the Maxwellian g at a perturbed state whose discrete moments equal Q. On the tensor
//      velocity grid with tensor trapezoid weights, g factors into 1-D Gaussians, so every moment
//      and every Jacobian entry sum_k w g psi psi^T is a product of 1-D sums S_d^m = sum_k w c^m A
//      (m <= 4). The unknowns are the log-linear coefficients alpha of g = exp(alpha . psi~) in the
//      velocity c = (xi - V) / s centred and scaled by the starting state (V, s^2), which keeps the
//      5 x 5 Jacobian well conditioned.
//        - FP32 Newton iterations (closed-form Jacobian) bring alpha to FP32 accuracy;
//        - FP64 refinement: the residual is evaluated in FP64 (the 1-D Gaussians by an exact
//          product recurrence outward from their peak, relative to the peak value: one FP64
//          exponential per axis, one for the ratio factor of equally spaced axes, and one for
//          alpha_0 with the three peak values) and
//          corrected with the FP32 Jacobian, which contracts the error by ~1e-6 per refinement.
//   3. writes Q, the perturbed state (rho', U', theta') used as the next warm start, and the FP32
//      exponent g = exp2(a + sum_d (b_d m_d + q_d m_d^2)) in the centred grid index m of the velocity
//      (exact in FP32), which the stage kernel evaluates per velocity.
// Points with rho <= 0, theta <= 0 or NaN moments set the domain bit of the status word; a Newton
// correction that stays large sets the Newton bit. No thread waits on another.
#include "bgk_common.cuh"

namespace bgk {

// exact FP32 two-sum: s + e = a + b
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Solve J x = r (5 x 5) by Gaussian elimination in T; returns false when a pivot vanishes. J is the
// Hessian sum_k w g psi psi^T of a strictly convex function (symmetric positive definite), so
// elimination without pivoting is stable and every index stays compile-time (registers only).
template <typename T>
__device__ __forceinline__ bool solve5(T (&J)[5][5], T (&r)[5], T (&x)[5])
{
#pragma unroll
    for (int c = 0; c < 5; c++) {
        if (!(J[c][c] > T(0)))
            return false;
        const T inv = T(1) / J[c][c];
#pragma unroll
        for (int q = c + 1; q < 5; q++) {
            const T m = J[q][c] * inv;
#pragma unroll
            for (int k = c + 1; k < 5; k++)
                J[q][k] -= m * J[c][k];
            r[q] -= m * r[c];
        }
    }
#pragma unroll
    for (int q = 4; q >= 0; q--) {
        T s = r[q];
#pragma unroll
        for (int k = q + 1; k < 5; k++)
            s -= J[q][k] * x[k];
        x[q] = s / J[q][q];
    }
    return true;
}

// Moments M[g psi~] (5) and, when J is non-null, the Jacobian M[g psi~ psi~^T] from the 1-D sums
// S[d][m] = sum_k w_k c_k^m A_d(c_k), scaled by e0 = exp(alpha_0).
template <typename T>
__device__ __forceinline__ void assemble(const T (&S)[3][5], T e0, T (&M)[5], T (*J)[5])
{
    const T p0 = S[0][0] * S[1][0] * S[2][0];
    const T a01 = S[1][0] * S[2][0], a02 = S[0][0] * S[2][0], a12 = S[0][0] * S[1][0];
    const T o0[3] = {a01, a02, a12};  // product of the S0 of the other two axes
    M[0] = e0 * p0;
#pragma unroll
    for (int d = 0; d < 3; d++)
        M[1 + d] = e0 * S[d][1] * o0[d];
    const T m4 = T(0.5) * (S[0][2] * o0[0] + S[1][2] * o0[1] + S[2][2] * o0[2]);
    M[4] = e0 * m4;
    if (!J)
        return;
    J[0][0] = M[0];
#pragma unroll
    for (int d = 0; d < 3; d++)
        J[0][1 + d] = J[1 + d][0] = M[1 + d];
    J[0][4] = J[4][0] = M[4];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        J[1 + d][1 + d] = e0 * S[d][2] * o0[d];
#pragma unroll
        for (int q = d + 1; q < 3; q++) {
            const int f = 3 - d - q;
            J[1 + d][1 + q] = J[1 + q][1 + d] = e0 * S[d][1] * S[q][1] * S[f][0];
        }
        // M[g c_d |c|^2 / 2]
        T s = S[d][3] * o0[d];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            if (q == d)
                continue;
            const int f = 3 - d - q;
            s += S[d][1] * S[q][2] * S[f][0];
        }
        J[1 + d][4] = J[4][1 + d] = e0 * T(0.5) * s;
    }
    T s4 = S[0][4] * o0[0] + S[1][4] * o0[1] + S[2][4] * o0[2];
    s4 += T(2) * (S[0][2] * S[1][2] * S[2][0] + S[0][2] * S[2][2] * S[1][0] + S[1][2] * S[2][2] * S[0][0]);
    J[4][4] = e0 * T(0.25) * s4;
}

// 1-D sums in FP32: A(c) = exp(ad c - (beta/2) c^2) on c_k = c0 + k h, trapezoid weights dv (ends /2);
// an axis with one node (no u_z, m = 2) has the single weight 1.
__device__ __forceinline__ void sums32(float ad, float beta, float c0, float h, int n, float dv, float (&S)[5])
{
    if (n == 1) {
        const float t = __expf(c0 * fmaf(-0.5f * beta, c0, ad));
        S[0] = t;
        S[1] = t * c0;
        S[2] = S[1] * c0;
        S[3] = S[2] * c0;
        S[4] = S[3] * c0;
        return;
    }
    for (int m = 0; m < 5; m++)
        S[m] = 0.f;
    for (int k = 0; k < n; k++) {
        const float c = fmaf((float)k, h, c0);
        float t = __expf(c * fmaf(-0.5f * beta, c, ad));
        if (k == 0 || k == n - 1)
            t *= 0.5f;
        S[0] += t;
        t *= c;
        S[1] += t;
        t *= c;
        S[2] += t;
        t *= c;
        S[3] += t;
        t *= c;
        S[4] += t;
    }
    for (int m = 0; m < 5; m++)
        S[m] *= dv;
}

// 1-D sums in FP64 up to m = 2, exponentials by the exact product recurrence from the peak:
// q(k) = ad c_k - beta/2 c_k^2 is quadratic in k, so A(k+1)/A(k) = exp(q1 + q2 (2k+1)) and the ratio
// itself changes by the constant factor exp(2 q2). Values decay away from the peak, so the products
// underflow gracefully instead of overflowing.
template <int M>
__device__ __forceinline__ void sums64(double ad, double beta, double c0, double h, int n, double dv, double (&S)[M])
{
    if (n == 1) {  // one node of unit weight (no u_z, m = 2)
        double t = exp(c0 * fma(-0.5 * beta, c0, ad));
#pragma unroll
        for (int m = 0; m < M; m++, t *= c0)
            S[m] = t;
        return;
    }
    const double q1 = (ad - beta * c0) * h, q2 = -0.5 * beta * h * h;
    int kp = (int)rintf((float)(-q1) / (float)(2.0 * q2));
    kp = kp < 0 ? 0 : (kp > n - 1 ? n - 1 : kp);
    const double cp = fma((double)kp, h, c0);
    const double Ap = exp(cp * fma(-0.5 * beta, cp, ad));
    const double E2 = exp(2.0 * q2);
    const double rp = exp(q1 + q2 * (2.0 * kp + 1.0));
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
    // upward from the peak (inclusive); unit weights, the trapezoid ends are corrected below
    double A = Ap, r = rp, c = cp, Aend = Ap, cend = cp;
    for (int k = kp; k < n; k++) {
        s0 += A;
        s1 = fma(c, A, s1);
        s2 = fma(c * c, A, s2);
        if (M > 3) {
            s3 = fma(c * c * c, A, s3);
            s4 = fma(c * c * c * c, A, s4);
        }
        Aend = A;
        cend = c;
        A *= r;
        r *= E2;
        c += h;
    }
    // downward from the peak (exclusive): A(k-1) = A(k) d(k), d(k) = E2 / r(k), d(k-1) = d(k) E2
    A = Ap;
    c = cp;
    double dk = E2 / rp, A0 = Ap, c0e = cp;
    for (int k = kp - 1; k >= 0; k--) {
        A *= dk;
        dk *= E2;
        c -= h;
        s0 += A;
        s1 = fma(c, A, s1);
        s2 = fma(c * c, A, s2);
        if (M > 3) {
            s3 = fma(c * c * c, A, s3);
            s4 = fma(c * c * c * c, A, s4);
        }
        A0 = A;
        c0e = c;
    }
    // trapezoid: half weight at both ends (k = 0 and k = n - 1)
    s0 -= 0.5 * (A0 + Aend);
    s1 -= 0.5 * (c0e * A0 + cend * Aend);
    s2 -= 0.5 * (c0e * c0e * A0 + cend * cend * Aend);
    S[0] = s0 * dv;
    S[1] = s1 * dv;
    S[2] = s2 * dv;
    if constexpr (M > 3) {
        s3 -= 0.5 * (c0e * c0e * c0e * A0 + cend * cend * cend * Aend);
        s4 -= 0.5 * (c0e * c0e * c0e * c0e * A0 + cend * cend * cend * cend * Aend);
        S[3] = s3 * dv;
        S[4] = s4 * dv;
    }
}

// Double-float (FP32 pair) arithmetic for the refinement's 1-D sums: about 2^-47 relative per operation,
// at FP32 throughput (GB300's FP64 rate is 1/60 of its FP32 rate). Every operation is an explicitly
// rounded intrinsic, so nothing is contracted or reassociated.
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl df_from(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_val(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // the exact rounding error of p
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const float s = __fadd_rn(a.hi, b.hi);  // two-sum of the high parts
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float r = __fadd_rn(s, e);
    return {r, __fsub_rn(e, __fsub_rn(r, s))};
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
// a * b for a float b
__device__ __forceinline__ dfl df_mulf(dfl a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ dfl df_scale(dfl a, float b) { return {a.hi * b, a.lo * b}; }  // b a power of two
// a / b: the FP32 quotient of the high parts, corrected once with the double-float remainder
__device__ __forceinline__ dfl df_div(dfl a, dfl b)
{
    const float r = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const dfl t = df_sub(a, df_mulf(b, q1));
    const float q2 = __fmul_rn(t.hi, r);
    const float s = __fadd_rn(q1, q2);
    return {s, __fsub_rn(q2, __fsub_rn(s, q1))};
}

// e^x in double-float FP32 arithmetic, relative error about 1e-14 for |x| <= 10 (checked against a
// 60-digit reference over [-10, 10]; the refinement's arguments are the log-ratios of neighbouring
// Gaussian nodes and the peak value, all well inside). x = n ln 2 + r with n = rint(x / ln 2) and
// |r| <= ln 2 / 2: ln 2 in three FP32 parts, the first with 12 significant bits so that n ln2_1 and
// x - n ln2_1 are exact; e^r by its Taylor series to degree 11 (truncation below 1e-15 at |r| = 0.35),
// Horner in double-float with the coefficients 1/k! as FP32 pairs; the result scaled by 2^n. Larger
// arguments take the FP64 exponential.
__device__ __forceinline__ dfl df_exp(dfl x)
{
    if (!(fabsf(x.hi) <= 10.f))
        return df_from(exp((double)x.hi + (double)x.lo));
    constexpr float kLn2a = 6.931152344e-01f, kLn2b = 3.194618330e-05f, kLn2c = 1.646594970e-12f;
    constexpr float kCh[12] = {1.0f, 1.0f, 0.5f, 0.1666666716337204f, 0.0416666679084301f, 0.008333333767950535f,
                               0.0013888889225199819f, 0.00019841270113829523f, 2.4801587642286904e-05f,
                               2.7557318844628753e-06f, 2.755731998149713e-07f, 2.5052107943679403e-08f};
    constexpr float kCl[12] = {0.0f, 0.0f, 0.0f, -4.967053879312289e-09f, -1.2417634698280722e-09f,
                               -4.34617203337595e-10f, -3.3631094437103215e-11f, -2.725596874933456e-12f,
                               -3.40699609366682e-13f, 3.793571224297229e-14f, -7.575112209051195e-15f,
                               4.4176230446483665e-16f};
    const float n = rintf(x.hi * 1.44269504089f);
    const float t = __fmaf_rn(-n, kLn2a, x.hi);  // exact
    dfl r = df_add({t, 0.f}, {x.lo, 0.f});
    r = df_add(r, df_mulf({-kLn2b, -kLn2c}, n));
    dfl p = {kCh[11], kCl[11]};
#pragma unroll
    for (int k = 10; k >= 0; k--)
        p = df_add(df_mul(p, r), {kCh[k], kCl[k]});
    const float sc = __int_as_float(((int)n + 127) << 23);  // 2^n, |n| <= 15
    return {p.hi * sc, p.lo * sc};
}

// The refinement's 1-D sums S0..S2 of one axis in double-float, relative to the peak node: returns
// ln A(kp) = q(kp) and S_m / A(kp) (sums64<3>'s recurrence). Every moment and Jacobian entry is a
// product of one 1-D sum per axis, so the three peak values join exp(alpha_0) in one exponential. The
// ratio factor E2 = exp(-beta h^2) comes from the caller (one exponential for all axes of equal
// spacing); the first ratio exp(q1 + q2 (2 kp + 1)) is one exponential per axis; the downward ratio
// E2 / rp a division. Relative error about 1e-13, far below what one refinement with the FP32 Jacobian
// needs.
__device__ __forceinline__ dfl sums_dd(dfl ad, dfl beta, dfl c0, dfl h, int n, dfl dv, dfl E2, dfl (&S)[3])
{
    if (n == 1) {  // one node of unit weight (no u_z, m = 2)
        S[0] = {1.f, 0.f};
        S[1] = c0;
        S[2] = df_mul(c0, c0);
        return df_mul(c0, df_sub(ad, df_mulf(df_mul(beta, c0), 0.5f)));
    }
    const dfl q1 = df_mul(df_sub(ad, df_mul(beta, c0)), h);
    const dfl q2 = df_mulf(df_mul(beta, df_mul(h, h)), -0.5f);
    int kp = (int)rintf(-q1.hi / (2.f * q2.hi));
    kp = kp < 0 ? 0 : (kp > n - 1 ? n - 1 : kp);
    const dfl cp = df_add(c0, df_mulf(h, (float)kp));
    const dfl rp = df_exp(df_add(q1, df_mulf(q2, (float)(2 * kp + 1))));
    const dfl hm = df_neg(h);
    dfl s0 = {0.f, 0.f}, s1 = {0.f, 0.f}, s2 = {0.f, 0.f};
    // upward from the peak (inclusive, value 1); unit weights, the trapezoid ends are corrected below
    dfl Ak = {1.f, 0.f}, r = rp, c = cp, Aend = Ak, cend = c;
    for (int k = kp; k < n; k++) {
        const dfl cA = df_mul(c, Ak);
        s0 = df_add(s0, Ak);
        s1 = df_add(s1, cA);
        s2 = df_add(s2, df_mul(c, cA));
        Aend = Ak;
        cend = c;
        Ak = df_mul(Ak, r);
        r = df_mul(r, E2);
        c = df_add(c, h);
    }
    // downward from the peak (exclusive): A(k-1) = A(k) d(k), d(k) = E2 / r(k), d(k-1) = d(k) E2
    Ak = {1.f, 0.f};
    c = cp;
    dfl dk = df_div(E2, rp), A0 = Ak, c0e = c;
    for (int k = kp - 1; k >= 0; k--) {
        Ak = df_mul(Ak, dk);
        dk = df_mul(dk, E2);
        c = df_add(c, hm);
        const dfl cA = df_mul(c, Ak);
        s0 = df_add(s0, Ak);
        s1 = df_add(s1, cA);
        s2 = df_add(s2, df_mul(c, cA));
        A0 = Ak;
        c0e = c;
    }
    // trapezoid: half weight at both ends (k = 0 and k = n - 1)
    const dfl xa0 = df_mul(c0e, A0), xae = df_mul(cend, Aend);
    S[0] = df_mul(df_sub(s0, df_scale(df_add(A0, Aend), 0.5f)), dv);
    S[1] = df_mul(df_sub(s1, df_scale(df_add(xa0, xae), 0.5f)), dv);
    S[2] = df_mul(df_sub(s2, df_scale(df_add(df_mul(c0e, xa0), df_mul(cend, xae)), 0.5f)), dv);
    return df_mul(cp, df_sub(ad, df_mulf(df_mul(beta, cp), 0.5f)));
}

// The moments M[g psi~] (5) of assemble() from double-float 1-D sums S[d][0..2], scaled by e0.
__device__ __forceinline__ void assemble_dd(const dfl (&S)[3][3], dfl e0, dfl (&M)[5])
{
    const dfl o0[3] = {df_mul(S[1][0], S[2][0]), df_mul(S[0][0], S[2][0]), df_mul(S[0][0], S[1][0])};
    M[0] = df_mul(e0, df_mul(S[0][0], o0[0]));
#pragma unroll
    for (int d = 0; d < 3; d++)
        M[1 + d] = df_mul(e0, df_mul(S[d][1], o0[d]));
    const dfl m4 = df_add(df_add(df_mul(S[0][2], o0[0]), df_mul(S[1][2], o0[1])), df_mul(S[2][2], o0[2]));
    M[4] = df_mul(e0, df_scale(m4, 0.5f));
}

__device__ __forceinline__ void newton_point(const NewtonArgs &A, const int pt)
{

    // 1. moments: exact sum of the FP32 partials (or the FP64 moments of the all-FP64 form)
    double Q[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        if (A.Qin) {
            Q[c] = A.Qin[(int64_t)pt * 5 + c];
            continue;
        }
        float hi = 0.f, lo = 0.f;
        const float *p = A.partial + (int64_t)c * A.npts + pt;
        for (int g = 0; g < A.ngroups; g++) {
            float s, e;
            two_sum(hi, __ldg(p + (int64_t)g * 5 * A.npts), s, e);
            hi = s;
            lo += e;
        }
        Q[c] = (double)hi + (double)lo;
    }
    if (!A.Qin) {  // the FP32 kernels sum in the grid-index basis
        const double mu[5] = {Q[0], Q[1], Q[2], Q[3], Q[4]};
        index_to_moments(mu, A.v0, A.dv, A.n, Q);
    }
#pragma unroll
    for (int c = 0; c < 5; c++)
        A.Q[(int64_t)pt * 5 + c] = Q[c];

    const double rho = Q[0], irho = 1.0 / rho;
    const double u[3] = {Q[1] * irho, Q[2] * irho, Q[3] * irho};
    const double hm = 0.5 * A.vdim;  // E = rho |U|^2 / 2 + (m / 2) rho theta
    const double thc = (Q[4] * irho - 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2])) * (A.vdim == 2 ? 1.0 : 2.0 / 3.0);
    float *par = A.param + (int64_t)pt * kParamStride;
    if (!(rho > 0.0) || !(thc > 0.0) || !isfinite(rho) || !isfinite(thc)) {
        atomicOr(A.err, kErrDomain);
        par[0] = -1e30f;  // g = 0 at this point
        for (int c = 1; c < kParamStride; c++)
            par[c] = 0.f;
        par[7] = kExp2Magic;
        if (A.param64)
            for (int c = 0; c < 5; c++)
                A.param64[(int64_t)pt * 5 + c] = 0.0;
        return;
    }

    // 2. starting state (V, s^2) and target moments in the centred, scaled basis psi~ = (1, c, |c|^2/2)
    double V[3] = {u[0], u[1], u[2]}, th0 = thc, rh0 = rho;
    bool warm = false;
    double lnc0 = 0.0;  // warm start in the lnC form: alpha_0 of the centred basis directly
    if (!A.cold && !A.continuous) {
        const double *pp = A.prim + (int64_t)pt * 5;
        if ((A.lnc_form || pp[0] > 0.0) && pp[4] > 0.0 && isfinite(pp[0] + pp[1] + pp[2] + pp[3] + pp[4])) {
            rh0 = pp[0];
            lnc0 = pp[0];
            V[0] = pp[1];
            V[1] = pp[2];
            V[2] = pp[3];
            th0 = pp[4];
            warm = true;
        }
    }
    const double is = rsqrt(th0), s = th0 * is;
    double Qt[5];
    Qt[0] = Q[0];
    for (int d = 0; d < 3; d++)
        Qt[1 + d] = (Q[1 + d] - Q[0] * V[d]) * is;
    Qt[4] = (Q[4] - (V[0] * Q[1] + V[1] * Q[2] + V[2] * Q[3]) + 0.5 * Q[0] * (V[0] * V[0] + V[1] * V[1] + V[2] * V[2])) * is * is;

    // alpha = (alpha_0, a_1, a_2, a_3, -beta): g = exp(alpha_0 + a . c - beta |c|^2 / 2)
    double al[5] = {warm && A.lnc_form ? lnc0 : log(rh0) - hm * log(2.0 * 3.14159265358979323846 * th0), 0.0, 0.0,
                    0.0, -1.0};
    // the grid in the centred, scaled basis, c_k = c0 + k h: in double-float FP32 pairs (the grid's own
    // pairs come with the arguments), with FP32 high parts for the FP32 iterations
    dfl c0d[3], hd[3], dvd[3];
    {
        const dfl isd = df_from(is);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            dvd[d] = {A.dvh[d], A.dvl[d]};
            c0d[d] = df_mul(df_sub({A.v0h[d], A.v0l[d]}, df_from(V[d])), isd);
            hd[d] = df_mul(dvd[d], isd);
        }
    }

    // the ablation (continuous Maxwellian of Q) stops here: alpha = the starting state itself
    double corr = 0.0;
    if (!A.continuous) {
        // FP32 Newton iterations until the step is below FP32 resolution (it32 minimum, 30 maximum), all
        // in FP32: the steps accumulate in da and are added to the FP64 alpha once at the end
        float J[5][5];
        bool haveJ = false;
        const int it32min = warm ? A.it32 : max(A.it32, 4);
        // the targets, grid and starting alpha as double-float pairs (the refinement's operands); their
        // high parts are the FP32 loop's (alpha_1..3 = 0 and alpha_4 = -1 are exact)
        dfl ald[5], Qd[5];
    #pragma unroll
        for (int m = 0; m < 5; m++) {
            ald[m] = m == 0 ? df_from(al[0]) : dfl{(float)al[m], 0.f};
            Qd[m] = df_from(Qt[m]);
        }
        float a0[5], da[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Qf[5], c0f[3], hf[3], dvf[3];
    #pragma unroll
        for (int m = 0; m < 5; m++) {
            a0[m] = ald[m].hi;
            Qf[m] = Qd[m].hi;
        }
    #pragma unroll
        for (int d = 0; d < 3; d++) {
            c0f[d] = c0d[d].hi;
            hf[d] = hd[d].hi;
            dvf[d] = dvd[d].hi;
        }
        for (int it = 0; it < 30; it++) {
            float S[3][5];
    #pragma unroll
            for (int d = 0; d < 3; d++)
                sums32(a0[1 + d] + da[1 + d], -(a0[4] + da[4]), c0f[d], hf[d], A.n[d], dvf[d], S[d]);
            float M[5];
            assemble<float>(S, expf(a0[0] + da[0]), M, J);
            haveJ = true;
            if (A.vdim == 2) {  // no u_z: the a_3 row and column vanish; keep a_3 = 0
                J[3][3] = 1.f;
                M[3] = Qf[3];
            }
            float r[5], dx[5], Jw[5][5];
    #pragma unroll
            for (int m = 0; m < 5; m++) {
                r[m] = Qf[m] - M[m];
    #pragma unroll
                for (int q = 0; q < 5; q++)
                    Jw[m][q] = J[m][q];
            }
            if (!solve5<float>(Jw, r, dx)) {
                haveJ = false;
                break;
            }
            // keep the Gaussian decaying: halve the step while beta would drop below 0.05
            float lam = 1.f;
            while (-(a0[4] + da[4] + lam * dx[4]) < 0.05f && lam > 1e-3f)
                lam *= 0.5f;
            float step = 0.f;
    #pragma unroll
            for (int m = 0; m < 5; m++) {
                da[m] += lam * dx[m];
                step = fmaxf(step, fabsf(lam * dx[m]));
            }
            if (it + 1 >= it32min && step < 2e-6f)
                break;
        }
    #pragma unroll
        for (int m = 0; m < 5; m++)
            ald[m] = df_add(ald[m], {da[m], 0.f});
        if (!haveJ) {
            atomicOr(A.err, kErrNewton);
            return;
        }

        // Refinements to FP64 accuracy with the FP32 Jacobian of the last iteration, until the correction
        // is at FP64 resolution (it64 minimum, 4 maximum). The residual Q - M(alpha) is formed in
        // double-float FP32 arithmetic (about 1e-13 relative): alpha, the targets and the grid in FP32
        // pairs, the 1-D Gaussian sums by the product recurrence, the exponentials by df_exp. GB300's
        // FP64 rate is 1/60 of its FP32 rate, and the same residual in FP64 took 58 % of this kernel.
        const int it64min = warm ? A.it64 : max(A.it64, 2);
        for (int it = 0; it < 4; it++) {
            dfl S[3][3], E2[3], lnp = {0.f, 0.f};
            const dfl beta = df_neg(ald[4]);
    #pragma unroll
            for (int d = 0; d < 3; d++)
                E2[d] = d > 0 && hd[d].hi == hd[d - 1].hi && hd[d].lo == hd[d - 1].lo
                            ? E2[d - 1]
                            : df_exp(df_mul(ald[4], df_mul(hd[d], hd[d])));
    #pragma unroll
            for (int d = 0; d < 3; d++)
                lnp = df_add(lnp, sums_dd(ald[1 + d], beta, c0d[d], hd[d], A.n[d], dvd[d], E2[d], S[d]));
            dfl M[5];
            assemble_dd(S, df_exp(df_add(ald[0], lnp)), M);  // the peaks' factors with alpha_0
            if (A.vdim == 2)
                M[3] = Qd[3];
            // the residual, solved with the FP32 Jacobian in FP32: the correction only needs FP32
            // relative accuracy (iterative refinement)
            float r[5], dx[5], Jw[5][5];
    #pragma unroll
            for (int m = 0; m < 5; m++) {
                const dfl t = df_sub(Qd[m], M[m]);
                r[m] = t.hi + t.lo;
    #pragma unroll
                for (int q = 0; q < 5; q++)
                    Jw[m][q] = J[m][q];
            }
            if (!solve5<float>(Jw, r, dx)) {
                atomicOr(A.err, kErrNewton);
                return;
            }
            float cf = 0.f;
    #pragma unroll
            for (int m = 0; m < 5; m++) {
                ald[m] = df_add(ald[m], {dx[m], 0.f});
                cf = fmaxf(cf, fabsf(dx[m]));
            }
            corr = cf;
            // the FP32 Jacobian contracts the error by ~1e-6 per refinement: after a correction below
            // 1e-6 the residual is at FP64 resolution
            if (it + 1 >= it64min && cf < 1e-6f)
                break;
        }
    #pragma unroll
        for (int m = 0; m < 5; m++)
            al[m] = df_val(ald[m]);
    }
    const double beta = -al[4];
    if (!(beta > 0.0) || !isfinite(al[0] + al[1] + al[2] + al[3]) || corr >= 1e-6) {
        atomicOr(A.err, kErrNewton);
        return;
    }

    // 3. outputs: perturbed state and the stage kernel's exponent in the raw velocity
    const double a[3] = {al[1], al[2], al[3]};
    const double ib = 1.0 / beta;
    const double thp = th0 * ib;  // s^2 / beta
    double Up[3];
    for (int d = 0; d < 3; d++)
        Up[d] = V[d] + s * a[d] * ib;
    const double lnC = al[0] + 0.5 * (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) * ib;  // ln(rho' (2 pi theta')^-m/2)
    double *pp = A.prim + (int64_t)pt * 5;
    pp[0] = A.lnc_form ? lnC : exp(lnC) * pow(2.0 * 3.14159265358979323846 * thp, hm);
    pp[1] = Up[0];
    pp[2] = Up[1];
    pp[3] = Up[2];
    pp[4] = thp;
    // stage-kernel exponent in the centred grid index m (xi_d = c_d + s_d m_d, c_d the grid centre,
    // s_d half the spacing): log2 g = L2E (lnC - |xi - U'|^2 / (2 theta'))
    //   = A + sum_d b_d m_d + sum_d q_d m_d^2, e_d = c_d - U'_d,
    //   A = L2E (lnC - |e|^2 / (2 theta')), b_d = -L2E e_d s_d / theta', q_d = -L2E s_d^2 / (2 theta').
    // The index is exact in FP32, so the kernel evaluates the Maxwellian of the exact discrete velocity
    // set. A = j + a with j = rint(A) carried exactly in the rounding constant of the kernel's 2^x and
    // a in [-1/2, 1/2]; on grids with one spacing q is written as two FP32 parts. Left in FP32, the
    // roundings of A and q would scale every g of the point alike (a moment error near 1e-7 per
    // solve, which the relaxation accumulates); split, they are below 1e-8.
    const double L2E = 1.4426950408889634;
    const double it2 = beta * is * is;  // 1 / theta' = beta / s^2
    double e2 = 0.0;
    for (int d = 0; d < 3; d++) {
        const double sd = 0.5 * A.dv[d];
        const double ed = A.v0[d] + (A.n[d] - 1) * sd - Up[d];
        e2 += ed * ed;
        par[1 + d] = (float)(-L2E * ed * sd * it2);
    }
    const double Aexp = L2E * (lnC - 0.5 * e2 * it2);
    const double j = fmin(20.0, fmax(-20.0, rint(Aexp)));
    par[0] = (float)(Aexp - j);
    if (A.dv[0] == A.dv[1] && A.dv[0] == A.dv[2]) {
        const double q = -0.5 * L2E * (0.25 * A.dv[0] * A.dv[0]) * it2;
        const float qh = (float)q;
        par[4] = qh;
        par[5] = (float)(q - (double)qh);
        par[6] = 0.f;
    } else {
        for (int d = 0; d < 3; d++)
            par[4 + d] = (float)(-0.5 * L2E * (0.25 * A.dv[d] * A.dv[d]) * it2);
    }
    par[7] = kExp2Magic + (float)j;
    if (A.mu_ref > 0.0) {  // variable collision time of this point's state: 1/tau = rho theta / mu(theta)
        const double itau = rho * thc / (A.mu_ref * pow(thc, A.mu_omega));
        par[6] = (float)itau;
        if (A.itau64)
            A.itau64[pt] = itau;
    }
    // body force: source S = g (beta . psi~) with M[g psi~ psi~^T] beta = M[S psi~] =
    // (0, rho F / s, rho (U - V) . F / s^2), whose raw moments are (0, rho F, rho U . F); written as
    // the polynomial q0 + q . xi + q4 |xi|^2 in the raw velocity
    if (A.force[0] != 0.0 || A.force[1] != 0.0 || A.force[2] != 0.0) {
        double S[3][5];
#pragma unroll
        for (int d = 0; d < 3; d++)
            sums64<5>(al[1 + d], -al[4], df_val(c0d[d]), df_val(hd[d]), A.n[d], A.dv[d], S[d]);
        double M[5], J[5][5], r[5], b[5];
        assemble<double>(S, exp(al[0]), M, J);
        r[0] = 0.0;
        double uf = 0.0;
        for (int d = 0; d < 3; d++) {
            r[1 + d] = rho * A.force[d] * is;
            uf += (u[d] - V[d]) * A.force[d];
        }
        r[4] = rho * uf * is * is;
        float *fp = A.fpar + (int64_t)pt * kParamStride;
        if (!solve5<double>(J, r, b)) {
            atomicOr(A.err, kErrNewton);
            return;
        }
        double q[5];
        q[0] = b[0] - (b[1] * V[0] + b[2] * V[1] + b[3] * V[2]) * is +
               0.5 * b[4] * (V[0] * V[0] + V[1] * V[1] + V[2] * V[2]) * is * is;
        for (int d = 0; d < 3; d++)
            q[1 + d] = b[1 + d] * is - b[4] * V[d] * is * is;
        q[4] = 0.5 * b[4] * is * is;
        for (int m = 0; m < 5; m++)
            fp[m] = (float)q[m];
        if (A.fpar64)
            for (int m = 0; m < 5; m++)
                A.fpar64[(int64_t)pt * 5 + m] = q[m];
    }
    if (A.param64) {
        double *p64 = A.param64 + (int64_t)pt * 5;
        p64[0] = exp(lnC);
        p64[1] = Up[0];
        p64[2] = Up[1];
        p64[3] = Up[2];
        p64[4] = 0.5 * it2;
    }
}

// Resident CTAs of 128 threads per SM the register allocation is sized for. The solve is bound by the
// latency of its FP32 and FP64 chains and by the FP64 pipe, which more resident warps keep busier:
// 8 CTAs (64 registers, spilling to L1) run the 262,144-point solves of the planar and Taylor-Green
// workloads 10-17 % faster than 4 (128 registers); the batched solve, whose arguments come from
// global memory, runs best at 4.
#ifndef BGK_NEWTON_MINCTAS
#define BGK_NEWTON_MINCTAS 8
#endif
#ifndef BGK_NEWTON_BATCH_MINCTAS
#define BGK_NEWTON_BATCH_MINCTAS 4
#endif

__global__ void __launch_bounds__(128, BGK_NEWTON_MINCTAS) k_newton(const NewtonArgs A)
{
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    if (pt < A.npts)
        newton_point(A, pt);
}

// Batched solve over the points of many independent problems: thread per point, the problem found
// by a binary search over the point prefix sums pt_start[0..n].
__global__ void __launch_bounds__(128, BGK_NEWTON_BATCH_MINCTAS) k_newton_batch(const NewtonArgs *__restrict__ args,
                                                      const int *__restrict__ pt_start, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pt_start[n])
        return;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pt_start[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    newton_point(args[lo], g - pt_start[lo]);
}

cudaError_t launch_newton_batch(const NewtonArgs *d_args, const int *d_pt_start, int n, int total_pts,
                                cudaStream_t s)
{
    const int threads = 128;
    k_newton_batch<<<(total_pts + threads - 1) / threads, threads, 0, s>>>(d_args, d_pt_start, n);
    return cudaGetLastError();
}

cudaError_t launch_newton(const NewtonArgs &A, cudaStream_t s)
{
    const int threads = 128;
    k_newton<<<(A.npts + threads - 1) / threads, threads, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace bgk
