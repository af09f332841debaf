// bgk_common.cuh -- device-side data structures shared by the libbgk kernels and the host planner.
//
// Device layout of the distribution function (FP32-split form):
//   f[vt][e][i][lane]   vt   = 32-velocity tile (velocities of one sign octant, padded to 32),
//                       e    = element (x fastest), i = node in the element (x fastest),
//                       lane = velocity within the tile.
// A warp owns one (element, run of tiles) task; lane l holds velocity l of the tile, so every
// global load or store of one node is one coalesced 128-byte line.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bgk {

constexpr int kWarp = 32;
constexpr int kWarpsPerCta = 4;   // elements per CTA in the stage kernel
constexpr int kMaxN1 = 8;         // nodes per direction (p <= 7)
constexpr int kParamStride = 8;   // floats per point in the BGK parameter table
constexpr float kExp2Magic = 12582912.0f;  // 1.5 * 2^23, the rounding constant of the stage kernels' 2^x

// error bits of the device status word
constexpr int kErrDomain = 1;
constexpr int kErrNewton = 2;
constexpr int kErrTimeout = 4;  // a bounded device wait (an asynchronous copy's barrier) gave up

// FR reference operators on [-1, 1] in FP32 (Sec. 2.1, Eqs. 7-9), merged for the upwind side:
//   left inflow  (xi_d > 0): d_i = sum_{j>=1} DL[i][j] (f_j - f_0) + gl[i] (t_up - f_0)
//   right inflow (xi_d < 0): d_i = sum_{j<=p-1} DR[i][j] (f_j - f_p) + gr[i] (t_up - f_p)
// where DL = D - gl (x) lm, DR = D - gr (x) lp (the interior trace folded into the derivative),
// t_up is the upwind neighbour's trace (lp on its nodes for a left neighbour, lm for a right one).
struct Ops {
    float DL[kMaxN1][kMaxN1];
    float DR[kMaxN1][kMaxN1];
    float DM[kMaxN1][kMaxN1];  // D - gl (x) lm - gr (x) lp: both interior traces folded in (curvilinear)
    float gl[kMaxN1], gr[kMaxN1];
    float lm[kMaxN1], lp[kMaxN1];
    float wq[kMaxN1];    // Gauss-Legendre weights / 2 (they sum to 1): the element mean of the limiter
};

struct Mesh {
    int dim;
    int ne[3];          // elements per direction (1 for unused directions)
    int nelem;
    int bc[6];          // boundary kind per face (2*d + side)
    float inv_h2[3];    // 2 / h_d
};

// One launch of the fused stage kernel over one velocity chunk.
struct StageArgs {
    const float *src;    // f_s of this chunk: [nvt_chunk][E][NP][32]
    const float *fn;     // f^n of this chunk (same layout), null in stage 1
    float *dst;          // stage output of this chunk (may alias fn: in-place update of f^n)
    const float *mi;     // [3][nslots] centred grid index m_d = 2 k_d - (n_d - 1) of every device slot
                         // (an integer, exact in FP32): xi_d = vc[d] + vs[d] m_d
    const float *wpsi;   // [nvt][5][32] w * (1, xi, |xi|^2/2), 0 on padded slots
    const float *vtab;   // [nvt][5][32] m_x, m_y, m_z, W, W sum_d r_d m_d^2 (rows 1 and 5 of the index-basis
                         // weights): the per-tile velocity table of the staged hexahedral kernel
    const float *gmask;  // [nslots] 1 for real velocities, 0 for padding
    const unsigned char *toct;  // [nvt] sign octant of every tile (bit d: xi_d >= 0)
    const float *ghost;  // [6][nslots] Dirichlet ghost values (sampled Maxwellian), or null
    const float *param;  // [n_x][8] BGK exponent of every point in the grid index m:
                         //   g = 2^j exp2(a + sum_d b_d m_d + e),  j integer,
                         // (a, b_x, b_y, b_z, p4, p5, p6, kExp2Magic + j) with, when viso (one spacing
                         // on all axes), e = p4 |m|^2 + p5 |m|^2 (p4 + p5 = q in two FP32 parts, p6 = 0),
                         // otherwise e = p4 m_x^2 + p5 m_y^2 + p6 m_z^2
    const float *rhow;   // [6][nfmax][N1^2] diffuse-wall density per wall face point, or null
    const float *fpar;   // [n_x][8] body-force source polynomial q0..q4: S = g (q0 + q.xi + q4|xi|^2), or null
    int nfmax;           // face elements per face slot of rhow
    float vc[3], vs[3];  // velocity grid centre and half spacing per axis
    int viso;            // 1: one velocity spacing on all axes
    float *partial;      // [ngroups_total][5][n_x] moment partial sums of the stage output
    Ops ops;
    Mesh mesh;
    int n1;              // nodes per direction (p + 1)
    int vt0;             // first global tile of the chunk
    int nvt;             // tiles in the chunk
    int G;               // tiles per warp task
    int group0;          // global index of the chunk's first task group
    int nslots;          // total device velocity slots (= nvt_total * 32)
    int npts;            // n_x
    float an, b;         // Shu-Osher coefficients: out = an f^n + b (f_s + dt L(f_s))
    float dt, inv_tau;
    int limiter;         // 1: Zhang-Shu positivity limiter on the stage output (Sec. 2.1, Eqs. 10-11)
    int vtau;            // 1: per-point 1/tau in param slot 6 (variable collision time, one spacing only)
    float kb, kg;        // b (1 - dt / tau) and b dt / tau: the weights of f_s and of the Maxwellian.
                         // Rounded so that an + b = 1 and kb + kg = b hold exactly in FP32, so a state
                         // equal to f^n and to its Maxwellian is kept up to unbiased rounding.
    // curvilinear hexahedra (null on the affine mesh):
    const float4 *met;   // [E][NP][3] metric rows Ja^d (d = 0, 1, 2) of every node; .w of row 0 and row 2
                         // = 1/J, .w of row 1 = W J (tensor Gauss-Legendre weight / 8 times J)
    const float4 *fnm;   // [E][3][2][N1^2] shared contravariant face normal N (direction, low/high side,
                         // face point); N . xi > 0 is flow towards +r_d
    const float *iwj;    // [E] 1 / sum_i W_i J_i (the limiter's element mean over the physical element)
    // unstructured connectivity (null: the structured element grid), per element and local face 2d+side:
    const int4 *ftab;    // [E][6] (neighbour element or -1 - g for the ghost of face g, node stride of the
                         // neighbour's normal axis, side of its shared face (1: its +1 end), index of
                         // the face in the wall list when it is a diffuse wall, else -1)
    const float *rhowu;  // [nwall][N1^2] wall densities of the unstructured mesh's wall faces, or null
    const unsigned char *fbase;  // [E][6][N1^2] the neighbour's first node on the line through each face point
    int *err;            // device status word (atomicOr of the kErr* bits)
    // exchange faces (x faces shared with a neighbouring subdomain): the neighbours' element layers next
    // to the lo and hi x faces, [nvt_total][eface][NP][32] (face element = y + ne_y z), or null
    const float *halo[2];
    int eface;           // elements on an x face (ne_y ne_z)
};

struct NewtonArgs {
    const float *partial;  // [ngroups][5][n_x]
    double force[3];       // body force per unit mass (zero: no force source)
    float *fpar;           // [n_x][8] force polynomial of the stage kernel (out, when force != 0)
    double *fpar64;        // [n_x][5] force polynomial in FP64 (out, all-FP64 form), or null
    const double *Qin;     // [n_x][5] FP64 moments; when set, used instead of the partial sums
    double *param64;       // [n_x][5] (C, U'x, U'y, U'z, 1/(2 theta')) of g in FP64, or null
    int ngroups;
    int npts;
    double *Q;             // [n_x][5] moments (out)
    double *prim;          // [n_x][5] perturbed state rho', U', theta' (in: warm start, out); with lnc_form
                           // slot 0 holds lnC = ln(rho' (2 pi theta')^(-m/2)) instead of rho'
    int lnc_form;          // 1: prim in the lnC form above (no logarithm or exponential per solve)
    float *param;          // [n_x][8] stage-kernel exponent (out)
    int *err;              // status word (atomicOr)
    int cold;              // 1: ignore prim and start from the continuous state of Q
    int continuous;        // 1: no solve, g = the continuous Maxwellian of Q (ablation)
    double mu_ref, mu_omega;  // mu_ref > 0: 1/tau = P / (mu_ref theta^omega) per point (Sec. 2, Eq. 5),
                              // written to param slot 6 (FP32 kernels) and to itau64 (FP64 form)
    double *itau64;           // [n_x] 1/tau of the plain FP64 form, or null
    int it32;              // FP32 Newton iterations
    int it64;              // FP64 refinements
    // 1-D velocity grids: xi_k = v0[d] + k dv[d], k < n[d]; trapezoid weights. An axis with one node
    // (n[2] = 1: the two-dimensional velocity space, m = 2) has v0 = 0 and unit weight, and its dv is
    // the x spacing (a placeholder that keeps the one-spacing forms of the exponent).
    double v0[3], dv[3];
    float v0h[3], v0l[3], dvh[3], dvl[3];  // v0 and dv as double-float pairs (hi + lo)
    int n[3];
    int vdim;              // velocity dimension m: 3, or 2 (no u_z, E = rho |U|^2 / 2 + rho theta)
};

// Axis d of the Newton solve's velocity grid: first node v0, spacing dv, n nodes (with the FP32 pairs).
inline void newton_axis(NewtonArgs &N, int d, double v0, double dv, int n)
{
    N.v0[d] = v0;
    N.dv[d] = dv;
    N.n[d] = n;
    N.v0h[d] = (float)v0;
    N.v0l[d] = (float)(v0 - (double)N.v0h[d]);
    N.dvh[d] = (float)dv;
    N.dvl[d] = (float)(dv - (double)N.dvh[d]);
}

// FR reference operators in FP64 for the plain all-FP64 form (Sec. 2.1, Eqs. 7-9).
struct Ops64 {
    double D[kMaxN1][kMaxN1];
    double lm[kMaxN1], lp[kMaxN1];
    double gl[kMaxN1], gr[kMaxN1];
    double wq[kMaxN1];  // Gauss-Legendre weights / 2
};

// One launch of the plain FP64 stage kernel over one velocity chunk (thread per degree of freedom).
struct Stage64Args {
    const double *src, *fn;
    double *dst;
    const double *xi;      // [3][nslots]
    const double *ghost;   // [6][nslots]
    const double *par;     // [n_x][5] (C, U', 1/(2 theta')) of the conservative Maxwellian
    const double *rhow;    // [6][nfmax][N1^2] diffuse-wall densities, or null
    const double *fpar;    // [n_x][5] body-force polynomial, or null
    int nfmax;
    const float *gmask;    // [nslots]
    Ops64 ops;
    Mesh mesh;
    double h[3];
    int N1, NP;
    int vt0, nvt, nslots;
    double an, b, dt, inv_tau;
    const double *itau;    // [n_x] per-point 1/tau (variable collision time), or null: inv_tau
    // curvilinear hexahedra (null on the affine mesh): the metric rows Ja^d of every node [n_x][3][3]
    // with 1/J [n_x], the shared face normals [E][3][2][N1^2][3], and the unstructured connectivity
    // (the FP32 form's tables: int4 [E][6] and the neighbour's first node per face point), or null
    const double *ja, *ijac, *fnm;
    const int4 *ftab;
    const unsigned char *fbase;
    const double *rhowu;   // [nwall][N1^2] wall densities of the unstructured mesh's wall faces, or null
};

// FP64 moments of the stage output over all chunks (warp per point).
struct Moments64Args {
    const double *base[9];  // chunk output bases
    int vt0[9], nvt[9];
    int nchunks;
    const double *wpsi;     // [nslots][5] w psi in FP64
    int E, NP, npts;
    double *Q;              // [n_x][5]
};

// Diffuse-wall densities of one stage (Sec. 2.1 boundary reading: zero net discrete mass flux through
// every wall face point): rho_w = sum_{out} w |xi_n| f_trace / sum_{in} w |xi_n| M_w.
struct WallArgs {
    const void *src[9];    // stage source of every chunk (float or double)
    int vt0[9], nvt[9], oct[9];
    int nchunks;
    int nslots;
    double inv_in[6];      // 1 / sum_{in} w |xi_n| M_w per face (0: not a wall)
    Mesh mesh;
    int N1, NP, nfmax;
    double lm[kMaxN1], lp[kMaxN1];
    float lmf[kMaxN1], lpf[kMaxN1];  // the same in FP32 (the FP32-split form's traces)
    // the structured mesh's wall faces: nwf faces wf[q], whose face points are CTAs wfstart[q] ..
    // wfstart[q + 1] - 1 of the launch
    int nwf, wf[6], wfstart[7];
    void *rhow;            // out: float or double [6][nfmax][N1^2]
    // curved walls (FP32-split form): the outward unit normal of every wall face point, [6][nfmax][N1^2][4]
    // (FP64), or null on affine faces; with it both sums run per face point over all velocities, the
    // incoming one with the unit-density wall Maxwellian ghost[6][nslots]
    const double *wn;
    const void *ghost;     // float or double, as the storage type of f
    // walls of an unstructured mesh: the list of wall faces (element, local face 2d+side, boundary class
    // g, 0), their outward unit normals [nwall][N1^2][4] and the densities out [nwall][N1^2]
    const int4 *wlist;
    int nwall;
    const double *wnu;
    void *rhowu;
};

// Moment weights of the FP32 stage kernels in the grid-index basis. With W = w / (dv_x dv_y dv_z)
// (1, 1/2, 1/4 or 1/8 on the trapezoid grid) and m_d = 2 k_d - (n_d - 1) the centred index
// (xi_d = c_d + s_d m_d, s_d = dv_d / 2), the kernels accumulate
//   mu = sum_k W_k (1, m_x, m_y, m_z, r_x m_x^2 + r_y m_y^2 + r_z m_z^2) f_k,  r_d = (s_d / s_x)^2 in FP32,
// whose weights are exact FP32 numbers (r_d = 1 on grids with one spacing), so the only FP32 error of
// the moments is the summation's. index_to_moments turns mu into Q = sum_k w_k psi_k f_k (Eq. 2).
// Trapezoid end factor of index k on an axis of n nodes: 1/2 at both ends, 1 inside; 1 on an axis with
// a single node (the absent u_z of the two-dimensional velocity space).
__host__ __device__ inline double end_factor(int k, int n) { return n > 1 && (k == 0 || k == n - 1) ? 0.5 : 1.0; }

__host__ __device__ inline float index_r(double dv_d, double dv_x)
{
    return (float)((dv_d / dv_x) * (dv_d / dv_x));
}

__host__ __device__ inline void index_to_moments(const double (&mu)[5], const double v0[3], const double dv[3],
                                                 const int n[3], double (&Q)[5])
{
    // cell volume of the axes that have a spacing (an axis with one node has unit weight)
    const double V = dv[0] * dv[1] * (n[2] > 1 ? dv[2] : 1.0), s0 = 0.5 * dv[0];
    double cs = 0.0, cm = 0.0;
    Q[0] = V * mu[0];
    for (int d = 0; d < 3; d++) {
        const double sd = 0.5 * dv[d], cd = v0[d] + (n[d] - 1) * sd;
        Q[1 + d] = V * (cd * mu[0] + sd * mu[1 + d]);
        cs += cd * cd;
        cm += cd * sd * mu[1 + d];
    }
    Q[4] = 0.5 * V * (cs * mu[0] + 2.0 * cm + s0 * s0 * mu[4]);
}

// Index of the face element of element (ec) on face direction d: the two other coordinates.
__host__ __device__ inline int face_elem(const Mesh &m, const int ec[3], int d)
{
    return d == 0 ? ec[1] + m.ne[1] * ec[2] : (d == 1 ? ec[0] + m.ne[0] * ec[2] : ec[0] + m.ne[0] * ec[1]);
}

__host__ __device__ inline int64_t fidx(int vt_local, int e, int i, int lane, int E, int NP)
{
    return (((int64_t)vt_local * E + e) * NP + i) * kWarp + lane;
}

}  // namespace bgk
