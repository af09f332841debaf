// bgk_api.cu -- the C ABI of libbgk (include/bgk.h): host planning, FR operators, buffers, the
// SSP-RK3 launch sequence and its CUDA graph.
//
// Memory plan of the FP32-split form. Velocities are grouped into chunks (one per sign octant by
// default). f^n lives in one full array A; stage outputs rotate through a pool of (chunks + 1)
// chunk-sized slots:
//   stage 1: chunk c reads A[c]                      -> writes slot c
//   stage 2: chunk c reads slot c (+ A[c])           -> writes slot c-1 (slot C for c = 0)
//   stage 3: chunk c reads its stage-2 slot (+ A[c]) -> writes A[c] in place
// A stage reads neighbours only inside its own chunk, and chunks run in order on one stream, so a
// slot is rewritten only after the launch that read it has finished. Memory = A + (C+1)/C arrays.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bgk.h"
#include "bgk_common.cuh"

namespace bgk {
cudaError_t launch_stage(const StageArgs &A, int p, int mode, int oct, cudaStream_t s);
cudaError_t prepare_stage(int dim, int p);
cudaError_t launch_newton(const NewtonArgs &A, cudaStream_t s);
cudaError_t launch_newton_batch(const NewtonArgs *d_args, const int *d_pt_start, int n, int total_pts,
                                cudaStream_t s);
cudaError_t launch_stage1d_batch(int n1, const StageArgs *d_args, const int2 *d_task_member, int *d_block,
                                 int ctas, cudaStream_t s);
cudaError_t set_batch_ops(int n1, const Ops &op);
int stage1d_tasks(const StageArgs &A);
int stage1d_batch_ctas(int n1);
cudaError_t launch_init_maxwellian(float *f, const double *prim, const float *mi, const float *gmask, int nslots,
                                   int nvt, int E, int NP, const int n[3], const double v0[3], const double dv[3],
                                   int *err, double *Q, double *warm, cudaStream_t s);
cudaError_t launch_convert_f(bool to_device, float *f, double *st, const int *slotk, int nvt, int E, int NP,
                             int64_t nvel, int p0, int npt, cudaStream_t s);
cudaError_t launch_stage64(const Stage64Args &A, cudaStream_t s);
cudaError_t launch_limit64(double *f, int nvt, int E, int NP, int N1, int dim, const Ops64 &ops, const double *ijac,
                           cudaStream_t s);
cudaError_t launch_wall(const WallArgs &A, bool fp64, const void *w, const void *xi, cudaStream_t s);
cudaError_t launch_moments64(const Moments64Args &A, cudaStream_t s);
cudaError_t launch_init64(double *f, const double *prim, const double *xi, const float *gmask, int nvt, int E, int NP,
                          int nslots, int vdim, int *err, cudaStream_t s);
cudaError_t launch_convert64(bool to_device, double *f, double *st, const int *slotk, int nvt, int E, int NP,
                             int64_t nvel, int p0, int npt, cudaStream_t s);
cudaError_t launch_f_distance(const void *a, bool a64, const void *b, bool b64, const int *slotk, int nvt, int E,
                              int NP, unsigned long long *out, cudaStream_t s);
}  // namespace bgk

using namespace bgk;

namespace {

const double kPi = 3.14159265358979323846;
const int kMinTuneG = 2;  // shortest task (tiles per warp task) the autotuner tries

struct Chunk {
    int vt0, nvt, group0, ngroups;
    int oct;  // sign octant of every tile (bit d: xi_d >= 0), 8 when the chunk mixes octants
};

// Gauss-Legendre nodes and weights on [-1, 1]: Newton on P_n with P_n' = n (x P_n - P_{n-1}) / (x^2 - 1).
void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; i++) {
        double z = -cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16)
                break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Lagrange basis value at y, barycentric weights lam.
double lag(int n, const double *x, const double *lam, int j, double y)
{
    double num = lam[j] / (y - x[j]), den = 0.0;
    for (int k = 0; k < n; k++)
        den += lam[k] / (y - x[k]);
    return num / den;
}

// FR operators (Sec. 2.1, Eqs. 7-9) for the stage kernel, built in FP64 and rounded to FP32:
// barycentric derivative matrix with the negative-sum diagonal, end interpolants, and the DG lift
// (Radau correction) derivatives g_L'(x_i) = -l_i(-1) / W_i, g_R'(x_i) = l_i(1) / W_i.
void build_ops(int p, Ops &op, Ops64 &o64, double *xg_out)
{
    const int n = p + 1;
    double x[kMaxN1], W[kMaxN1], lam[kMaxN1], D[kMaxN1][kMaxN1], lm[kMaxN1], lp[kMaxN1], gl[kMaxN1], gr[kMaxN1];
    gauss_legendre(n, x, W);
    for (int j = 0; j < n; j++) {
        lam[j] = 1.0;
        for (int k = 0; k < n; k++)
            if (k != j)
                lam[j] /= (x[j] - x[k]);
    }
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i)
                continue;
            D[i][j] = (lam[j] / lam[i]) / (x[i] - x[j]);
            s += D[i][j];
        }
        D[i][i] = -s;
    }
    for (int j = 0; j < n; j++) {
        lm[j] = n == 1 ? 1.0 : lag(n, x, lam, j, -1.0);
        lp[j] = n == 1 ? 1.0 : lag(n, x, lam, j, 1.0);
    }
    for (int i = 0; i < n; i++) {
        gl[i] = -lm[i] / W[i];
        gr[i] = lp[i] / W[i];
    }
    memset(&op, 0, sizeof(op));
    memset(&o64, 0, sizeof(o64));
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++)
            o64.D[i][j] = D[i][j];
        o64.lm[i] = lm[i];
        o64.lp[i] = lp[i];
        o64.gl[i] = gl[i];
        o64.gr[i] = gr[i];
        o64.wq[i] = 0.5 * W[i];
    }
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            op.DL[i][j] = (float)(D[i][j] - gl[i] * lm[j]);
            op.DR[i][j] = (float)(D[i][j] - gr[i] * lp[j]);
            op.DM[i][j] = (float)(D[i][j] - gl[i] * lm[j] - gr[i] * lp[j]);
        }
        op.gl[i] = (float)gl[i];
        op.gr[i] = (float)gr[i];
        op.lm[i] = (float)lm[i];
        op.lp[i] = (float)lp[i];
        op.wq[i] = (float)(0.5 * W[i]);
        xg_out[i] = x[i];
    }
}

// Continuous Maxwellian (Eq. 4) in velocity dimension m (3, or 2: u_z and U_z take no part).
double maxwell(int m, double rho, const double *U, double th, double vx, double vy, double vz)
{
    double r2 = (vx - U[0]) * (vx - U[0]) + (vy - U[1]) * (vy - U[1]);
    if (m == 3)
        r2 += (vz - U[2]) * (vz - U[2]);
    return rho * pow(2.0 * kPi * th, -0.5 * m) * exp(-0.5 * r2 / th);
}

}  // namespace

struct bgk_ctx {
    // problem
    int dim = 0, p = 0, N1 = 0, NP = 0;
    int ne[3] = {1, 1, 1};
    int E = 0;
    int64_t npts = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    double bcs[30] = {0};
    int nv[3] = {0, 0, 0};
    double vlo[3] = {0, 0, 0}, dv[3] = {0, 0, 0};
    int vdim = 3;  // velocity dimension m: 3, or 2 when nv[2] = 1 (dv[2] then holds dv[0] as a placeholder)
    int64_t nvel = 0;
    double tau = 0;
    bgk_opts opts{};
    double xg[kMaxN1] = {0};
    // velocity plan
    int nvt = 0, nslots = 0, G = 1, ngroups = 0, max_groups = 0;
    std::vector<int> slotk;
    std::vector<unsigned char> toct_h;  // sign octant of every tile
    std::vector<Chunk> chunks;
    int64_t chunk_floats = 0;  // floats per pool slot
    // device buffers
    float *fA = nullptr, *pool = nullptr;
    float *xi = nullptr, *mi = nullptr, *wpsi = nullptr, *gmask = nullptr, *ghost = nullptr;
    float *vtab = nullptr;  // [nvt][5][32]: m_x, m_y, m_z, W and W sum_d r_d m_d^2 of every slot, by tile
    int *slotk_d = nullptr;
    unsigned char *toct = nullptr;
    float *partial = nullptr, *param = nullptr;
    // all-FP64 form
    int prec = BGK_FP32_SPLIT;
    double *fA64 = nullptr, *pool64 = nullptr, *xi64 = nullptr, *wpsi64 = nullptr, *ghost64 = nullptr, *par64 = nullptr;
    // diffuse walls and body force
    bool has_wall = false, has_force = false;
    // exchange faces (x faces shared with a neighbouring subdomain): the halos, [nvt][E_face][NP][32]
    bool has_exchange = false;
    int64_t halo_floats = 0;
    float *halo_own[2] = {nullptr, nullptr};   // library-owned halos (zeros until bgk_set_halo)
    const float *halo[2] = {nullptr, nullptr}; // the halos the stage kernel reads (lo, hi x face)
    double force[3] = {0, 0, 0};
    double inv_in[6] = {0, 0, 0, 0, 0, 0};
    int nfmax = 0;
    float *rhow32 = nullptr, *fpar32 = nullptr, *w32 = nullptr;
    double *rhow64 = nullptr, *fpar64 = nullptr, *w64 = nullptr;
    Ops64 ops64{};
    double *Q = nullptr, *prim = nullptr, *prim_in = nullptr;
    double *itau64 = nullptr;  // per-point 1/tau of the FP64 form (variable collision time)
    // curvilinear hexahedra (bgk_set_geometry)
    float4 *met = nullptr, *fnm = nullptr;
    float *iwj = nullptr;
    double *wn64 = nullptr;  // outward unit normals of the curved wall face points [6][nfmax][N1^2][4]
    double *ja64 = nullptr, *ijac64 = nullptr, *fnm64 = nullptr;  // the same metric in FP64 (all-FP64 form)
    // unstructured connectivity (bgk_set_connectivity): host tables [E][6] and their device form
    std::vector<int> cnbr, cface, corient;
    int4 *ftab = nullptr;
    unsigned char *fbase = nullptr;
    // diffuse walls of an unstructured mesh: the list of its wall faces (element, local face, class, 0),
    // each face's index in it (or -1) by element and local face, normals and wall densities
    std::vector<int4> wlist_h;
    std::vector<int> wall_idx;
    int4 *wlist = nullptr;
    double *wnu = nullptr;
    float *rhowu32 = nullptr;
    double *rhowu64 = nullptr;
    std::vector<double> geom;  // node coordinates [n_x][3]
    double curv_smax = 0.0;    // max over nodes and velocities of sum_d |Ja^d . xi| / (2 J)
    int *err = nullptr;
    int64_t bytes = 0;
    Ops ops{};
    Mesh mesh{};
    int64_t esize = 4;  // bytes per stored value of f
    // execution
    cudaStream_t stream = nullptr, own = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double gdt = -1.0;
    std::string last;
    int sticky = 0;
    // timing
    bool timing = false;
    struct Ev {
        cudaEvent_t a, b;
        int kind;  // 0 stage, 1 newton
        double bytes;
    };
    std::vector<Ev> evs;
    size_t nev = 0;
};

namespace {

int fail(bgk_ctx *c, int code, const std::string &msg)
{
    if (c)
        c->last = msg;
    return code;
}

int cuda_fail(bgk_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, BGK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                       \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess)                         \
            return cuda_fail(c, e_, #call);            \
    } while (0)

template <typename T>
cudaError_t dalloc(bgk_ctx *c, T **p, size_t n)
{
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e == cudaSuccess)
        c->bytes += (int64_t)(n * sizeof(T));
    return e;
}

StageArgs stage_args(bgk_ctx *c, const Chunk &ch)
{
    StageArgs A{};
    A.mi = c->mi;
    A.toct = c->toct;
    for (int d = 0; d < 3; d++) {
        A.vc[d] = (float)(c->vlo[d] + 0.5 * (c->nv[d] - 1) * c->dv[d]);
        A.vs[d] = (float)(0.5 * c->dv[d]);
    }
    A.viso = c->dv[0] == c->dv[1] && c->dv[0] == c->dv[2];
    A.wpsi = c->wpsi;
    A.vtab = c->vtab;
    A.gmask = c->gmask;
    A.ghost = c->ghost;
    A.param = c->param;
    A.rhow = c->rhow32;
    A.fpar = c->fpar32;
    A.nfmax = c->nfmax;
    A.partial = c->partial;
    A.ops = c->ops;
    A.mesh = c->mesh;
    A.n1 = c->N1;
    A.vt0 = ch.vt0;
    A.nvt = ch.nvt;
    A.G = c->G;
    A.group0 = ch.group0;
    A.nslots = c->nslots;
    A.npts = (int)c->npts;
    A.inv_tau = (float)(1.0 / c->tau);
    A.limiter = c->opts.limiter != 0;
    A.vtau = c->opts.mu_ref > 0.0;
    A.met = c->met;
    A.fnm = c->fnm;
    A.iwj = c->iwj;
    A.ftab = c->ftab;
    A.fbase = c->fbase;
    A.rhowu = c->rhowu32;
    A.err = c->err;
    A.halo[0] = c->halo[0];
    A.halo[1] = c->halo[1];
    A.eface = c->ne[1] * c->ne[2];
    return A;
}

// Shu-Osher stage st (0, 1, 2) of step dt in FP32: b = 1, 1/4, 2/3 and an = 1 - b (exact), the
// Maxwellian weight kg = b dt / tau and kb = b - kg, rounded so that kb + kg = b exactly (Sterbenz's
// lemma makes b - kg or b - kb exact for dt / tau <= 2). With inexact sums a state equal to f^n and
// to its Maxwellian would gain the sum's rounding (about 3e-8 for 1/3 + 2/3) at every stage.
void stage_coeffs(StageArgs &A, int st, double dt, double tau)
{
    static const float bb[3] = {1.f, 0.25f, (float)(2.0 / 3.0)};
    const float b = bb[st];
    A.b = b;
    A.an = 1.f - b;
    A.dt = (float)dt;
    A.inv_tau = (float)(1.0 / tau);
    const float kg0 = (float)((double)b * dt / tau);
    const float kb = b - kg0;
    A.kb = kb;
    A.kg = b - kb;
}

float *chunk_ptr(bgk_ctx *c, float *base, int vt0) { return base + (int64_t)vt0 * c->E * c->NP * kWarp; }

NewtonArgs newton_args(bgk_ctx *c, int cold)
{
    NewtonArgs N{};
    N.partial = c->partial;
    N.ngroups = c->ngroups;
    N.npts = (int)c->npts;
    N.Q = c->Q;
    N.prim = c->prim;
    N.lnc_form = 1;  // bgk_equilibrium turns lnC into rho' on the host
    N.param = c->param;
    N.err = c->err;
    N.cold = cold;
    N.continuous = c->opts.maxwellian == BGK_MAXWELLIAN_CONTINUOUS;
    N.mu_ref = c->opts.mu_ref;
    N.mu_omega = c->opts.mu_omega;
    N.itau64 = c->itau64;
    N.it32 = c->opts.newton_max_it > 0 ? c->opts.newton_max_it : 2;
    N.it64 = 1;
    if (c->prec == BGK_FP64) {  // FP64 moments from k64_moments; FP64 Maxwellian parameters out
        N.Qin = c->Q;
        N.param64 = c->par64;
    }
    for (int d = 0; d < 3; d++)
        N.force[d] = c->force[d];
    N.fpar = c->fpar32;
    N.fpar64 = c->fpar64;
    for (int d = 0; d < 3; d++)
        newton_axis(N, d, c->vlo[d], c->dv[d], c->nv[d]);
    N.vdim = c->vdim;
    return N;
}

void ev_begin(bgk_ctx *c, int kind, double bytes)
{
    if (!c->timing)
        return;
    if (c->nev == c->evs.size()) {
        bgk_ctx::Ev ev{};
        cudaEventCreate(&ev.a);
        cudaEventCreate(&ev.b);
        c->evs.push_back(ev);
    }
    bgk_ctx::Ev &ev = c->evs[c->nev];
    ev.kind = kind;
    ev.bytes = bytes;
    cudaEventRecord(ev.a, c->stream);
}

void ev_end(bgk_ctx *c)
{
    if (!c->timing)
        return;
    cudaEventRecord(c->evs[c->nev].b, c->stream);
    c->nev++;
}

double *chunk_ptr64(bgk_ctx *c, double *base, int vt0) { return base + (int64_t)vt0 * c->E * c->NP * kWarp; }

Moments64Args moments64_args(bgk_ctx *c)
{
    Moments64Args M{};
    M.nchunks = (int)c->chunks.size();
    M.wpsi = c->wpsi64;
    M.E = c->E;
    M.NP = c->NP;
    M.npts = (int)c->npts;
    M.Q = c->Q;
    return M;
}

// Moments of the state f^n and its conservative Maxwellian (after bgk_set_state / bgk_set_f). have_q:
// Q was formed with the state (the initial sampling's separable moments) and the Newton solve starts
// from the sampled Maxwellian itself; otherwise a moments pass over f and a cold solve.
int prologue(bgk_ctx *c, cudaStream_t s, bool have_q = false)
{
    if (c->prec == BGK_FP64) {
        Moments64Args M = moments64_args(c);
        for (int q = 0; q < M.nchunks; q++) {
            M.base[q] = chunk_ptr64(c, c->fA64, c->chunks[q].vt0);
            M.vt0[q] = c->chunks[q].vt0;
            M.nvt[q] = c->chunks[q].nvt;
        }
        CK(launch_moments64(M, s));
        CK(launch_newton(newton_args(c, 1), s));
        return BGK_OK;
    }
    if (have_q) {  // after bgk_set_state: the moments and the warm start are the sampled Maxwellian's
        NewtonArgs N = newton_args(c, 0);
        N.Qin = c->Q;
        CK(launch_newton(N, s));
        return BGK_OK;
    }
    for (const Chunk &ch : c->chunks) {
        StageArgs A = stage_args(c, ch);
        A.src = chunk_ptr(c, c->fA, ch.vt0);
        CK(launch_stage(A, c->p, 1, ch.oct, s));
    }
    CK(launch_newton(newton_args(c, 1), s));
    return BGK_OK;
}

// Diffuse-wall densities of the stage whose chunk sources are src[q].
int enqueue_wall(bgk_ctx *c, const std::vector<const void *> &src, cudaStream_t s)
{
    if (!c->has_wall)
        return BGK_OK;
    WallArgs W{};
    W.nchunks = (int)c->chunks.size();
    for (int q = 0; q < W.nchunks; q++) {
        W.src[q] = src[q];
        W.vt0[q] = c->chunks[q].vt0;
        W.nvt[q] = c->chunks[q].nvt;
        W.oct[q] = c->chunks[q].oct;
    }
    W.nslots = c->nslots;
    for (int q = 0; q < 6; q++)
        W.inv_in[q] = c->inv_in[q];
    W.mesh = c->mesh;
    W.N1 = c->N1;
    W.NP = c->NP;
    W.nfmax = c->nfmax;
    for (int j = 0; j < c->N1; j++) {
        W.lm[j] = c->ops64.lm[j];
        W.lp[j] = c->ops64.lp[j];
        W.lmf[j] = (float)c->ops64.lm[j];
        W.lpf[j] = (float)c->ops64.lp[j];
    }
    const bool f64 = c->prec == BGK_FP64;
    W.rhow = f64 ? (void *)c->rhow64 : (void *)c->rhow32;
    W.wn = c->wn64;  // curved walls
    W.nwf = 0;
    W.wfstart[0] = 0;
    for (int f = 0; f < 6; f++) {
        if (c->inv_in[f] == 0.0 && !(c->wn64 && c->mesh.bc[f] == BGK_BC_DIFFUSE_WALL))
            continue;
        const int d = f >> 1, o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
        W.wf[W.nwf] = f;
        W.wfstart[W.nwf + 1] = W.wfstart[W.nwf] + c->mesh.ne[o1] * c->mesh.ne[o2] * c->N1 * c->N1;
        W.nwf++;
    }
    W.ghost = f64 ? (const void *)c->ghost64 : (const void *)c->ghost;
    if (!c->wlist_h.empty()) {  // walls of an unstructured mesh: their own list instead of the grid's faces
        W.wlist = c->wlist;
        W.nwall = (int)c->wlist_h.size();
        W.wnu = c->wnu;
        W.rhowu = f64 ? (void *)c->rhowu64 : (void *)c->rhowu32;
    }
    CK(launch_wall(W, f64, f64 ? (const void *)c->w64 : (const void *)c->w32,
                   f64 ? (const void *)c->xi64 : (const void *)c->xi, s));
    return BGK_OK;
}

// One SSP-RK3 step of the plain all-FP64 form: per stage, the unfused stage kernel over every chunk,
// the FP64 moments of all chunk outputs, then the Newton solve.
int enqueue_step64(bgk_ctx *c, double dt, cudaStream_t s, const std::vector<int> &slot1,
                   const std::vector<int> &slot2)
{
    static const double an[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double bb[3] = {1.0, 0.25, 2.0 / 3.0};
    const int C = (int)c->chunks.size();
    for (int st = 0; st < 3; st++) {
        Moments64Args M = moments64_args(c);
        if (c->has_wall) {
            std::vector<const void *> srcs(C);
            for (int q = 0; q < C; q++) {
                double *Aq = chunk_ptr64(c, c->fA64, c->chunks[q].vt0);
                srcs[q] = st == 0 ? (const void *)Aq
                                  : (const void *)(c->pool64 + (int64_t)(st == 1 ? slot1[q] : slot2[q]) * c->chunk_floats);
            }
            int rc = enqueue_wall(c, srcs, s);
            if (rc)
                return rc;
        }
        for (int q = 0; q < C; q++) {
            const Chunk &ch = c->chunks[q];
            double *Aq = chunk_ptr64(c, c->fA64, ch.vt0);
            double *s1 = c->pool64 + (int64_t)slot1[q] * c->chunk_floats;
            double *s2 = c->pool64 + (int64_t)slot2[q] * c->chunk_floats;
            Stage64Args A{};
            A.src = st == 0 ? Aq : (st == 1 ? s1 : s2);
            A.fn = st == 0 ? nullptr : Aq;
            A.dst = st == 0 ? s1 : (st == 1 ? s2 : Aq);
            A.xi = c->xi64;
            A.ghost = c->ghost64;
            A.par = c->par64;
            A.rhow = c->rhow64;
            A.fpar = c->fpar64;
            A.nfmax = c->nfmax;
            A.gmask = c->gmask;
            A.ops = c->ops64;
            A.mesh = c->mesh;
            for (int d = 0; d < 3; d++)
                A.h[d] = c->h[d];
            A.N1 = c->N1;
            A.NP = c->NP;
            A.vt0 = ch.vt0;
            A.nvt = ch.nvt;
            A.nslots = c->nslots;
            A.an = an[st];
            A.b = bb[st];
            A.dt = dt;
            A.inv_tau = 1.0 / c->tau;
            A.itau = c->itau64;
            A.ja = c->ja64;  // curvilinear hexahedra (null on the affine mesh)
            A.ijac = c->ijac64;
            A.fnm = c->fnm64;
            A.ftab = c->ftab;
            A.fbase = c->fbase;
            A.rhowu = c->rhowu64;
            int64_t real = 0;
            for (int v = ch.vt0 * kWarp; v < (ch.vt0 + ch.nvt) * kWarp; v++)
                real += c->slotk[v] >= 0;
            ev_begin(c, 0, (double)real * c->npts * sizeof(double) * (st == 0 ? 2 : 3));
            CK(launch_stage64(A, s));
            if (c->opts.limiter)
                CK(launch_limit64(A.dst, ch.nvt, c->E, c->NP, c->N1, c->dim, c->ops64, c->ijac64, s));
            ev_end(c);
            M.base[q] = A.dst;
            M.vt0[q] = ch.vt0;
            M.nvt[q] = ch.nvt;
        }
        ev_begin(c, 1, 0.0);
        CK(launch_moments64(M, s));
        CK(launch_newton(newton_args(c, 0), s));
        ev_end(c);
    }
    return BGK_OK;
}

int enqueue_stage(bgk_ctx *c, double dt, int st, cudaStream_t s);

// One SSP-RK3 step: three stages, each over all chunks, each followed by the Newton solve.
int enqueue_step(bgk_ctx *c, double dt, cudaStream_t s)
{
    const int C = (int)c->chunks.size();
    std::vector<int> slot1(C), slot2(C);
    for (int q = 0; q < C; q++) {
        slot1[q] = q;
        slot2[q] = q == 0 ? C : q - 1;
    }
    if (c->prec == BGK_FP64)
        return enqueue_step64(c, dt, s, slot1, slot2);
    for (int st = 0; st < 3; st++) {
        int rc = enqueue_stage(c, dt, st, s);
        if (rc)
            return rc;
    }
    return BGK_OK;
}

// Pool slots of the FP32-split stage outputs: chunk q's stage-1 output in slot q, its stage-2 output in
// slot q - 1 (slot C for chunk 0), which chunk q - 1 has read by then.
void stage_slots(const bgk_ctx *c, std::vector<int> &slot1, std::vector<int> &slot2)
{
    const int C = (int)c->chunks.size();
    slot1.resize(C);
    slot2.resize(C);
    for (int q = 0; q < C; q++) {
        slot1[q] = q;
        slot2[q] = q == 0 ? C : q - 1;
    }
}

// The source of stage st (0, 1, 2) of chunk q (FP32-split form): f^n, the stage-1 or the stage-2 output.
float *stage_source(bgk_ctx *c, int q, int st)
{
    std::vector<int> slot1, slot2;
    stage_slots(c, slot1, slot2);
    if (st == 0)
        return chunk_ptr(c, c->fA, c->chunks[q].vt0);
    return c->pool + (int64_t)(st == 1 ? slot1[q] : slot2[q]) * c->chunk_floats;
}

// Stage st of one SSP-RK3 step of the FP32-split form: the wall densities of the stage source, the stage
// kernel over every chunk, the Newton solve of the stage output.
int enqueue_stage(bgk_ctx *c, double dt, int st, cudaStream_t s)
{
    const int C = (int)c->chunks.size();
    std::vector<int> slot1, slot2;
    stage_slots(c, slot1, slot2);
    {
        if (c->has_wall) {
            std::vector<const void *> srcs(C);
            for (int q = 0; q < C; q++) {
                float *Aq = chunk_ptr(c, c->fA, c->chunks[q].vt0);
                srcs[q] = st == 0 ? (const void *)Aq
                                  : (const void *)(c->pool + (int64_t)(st == 1 ? slot1[q] : slot2[q]) * c->chunk_floats);
            }
            int rc = enqueue_wall(c, srcs, s);
            if (rc)
                return rc;
        }
        for (int q = 0; q < C; q++) {
            const Chunk &ch = c->chunks[q];
            StageArgs A = stage_args(c, ch);
            float *Aq = chunk_ptr(c, c->fA, ch.vt0);
            float *s1 = c->pool + (int64_t)slot1[q] * c->chunk_floats;
            float *s2 = c->pool + (int64_t)slot2[q] * c->chunk_floats;
            if (st == 0) {
                A.src = Aq;
                A.fn = nullptr;
                A.dst = s1;
            } else if (st == 1) {
                A.src = s1;
                A.fn = Aq;
                A.dst = s2;
            } else {
                A.src = s2;
                A.fn = Aq;
                A.dst = Aq;
            }
            stage_coeffs(A, st, dt, c->tau);
            int64_t real = 0;
            for (int v = ch.vt0 * kWarp; v < (ch.vt0 + ch.nvt) * kWarp; v++)
                real += c->slotk[v] >= 0;
            ev_begin(c, 0, (double)real * c->npts * sizeof(float) * (st == 0 ? 2 : 3));
            CK(launch_stage(A, c->p, 0, ch.oct, s));
            ev_end(c);
        }
        ev_begin(c, 1, 0.0);
        CK(launch_newton(newton_args(c, 0), s));
        ev_end(c);
    }
    return BGK_OK;
}

int read_status(bgk_ctx *c)
{
    int e = 0;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    c->sticky |= e;
    if (c->sticky & kErrDomain)
        return fail(c, BGK_EDOMAIN, "non-physical state (rho <= 0, theta <= 0 or NaN) met on the device");
    if (c->sticky & kErrNewton)
        return fail(c, BGK_ENEWTON, "conservative-Maxwellian Newton solve did not converge at some point");
    if (c->sticky & kErrTimeout)
        return fail(c, BGK_ETIMEOUT, "a bounded device wait for an asynchronous copy gave up");
    return BGK_OK;
}

}  // namespace

extern "C" {

const char *bgk_last_error(const bgk_ctx *c) { return c ? c->last.c_str() : "null context"; }

void bgk_destroy(bgk_ctx *c)
{
    if (!c)
        return;
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    if (c->gexec)
        cudaGraphExecDestroy(c->gexec);
    for (auto &ev : c->evs) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    void *bufs[] = {c->fA, c->pool, c->xi, c->mi, c->vtab, c->toct, c->wpsi, c->gmask, c->ghost, c->slotk_d, c->partial,
                    c->param, c->Q, c->prim, c->prim_in, c->err, c->fA64, c->pool64, c->xi64,
                    c->wpsi64, c->ghost64, c->par64, c->rhow32, c->fpar32, c->w32, c->rhow64,
                    c->fpar64, c->w64, c->itau64, c->met, c->fnm, c->iwj, c->ftab, c->fbase, c->wn64,
                    c->ja64, c->ijac64, c->fnm64, c->wlist, c->wnu, c->rhowu32, c->rhowu64,
                    c->halo_own[0], c->halo_own[1]};
    for (void *b : bufs)
        if (b)
            cudaFree(b);
    if (c->own)
        cudaStreamDestroy(c->own);
    delete c;
}

int bgk_create(const bgk_mesh *mesh, int p, const bgk_vgrid *vg, double tau, const bgk_opts *opts, bgk_ctx **out)
{
    if (!out)
        return BGK_EINVAL;
    *out = nullptr;
    if (!mesh || !vg)
        return BGK_EINVAL;
    bgk_ctx *c = new bgk_ctx();
    auto bail = [&](int code, const std::string &msg) {
        c->last = msg;
        fprintf(stderr, "bgk_create: %s\n", msg.c_str());
        bgk_destroy(c);
        return code;
    };
    if (opts)
        c->opts = *opts;
    if (c->opts.precision != BGK_FP32_SPLIT && c->opts.precision != BGK_FP64)
        return bail(BGK_EINVAL, "precision must be BGK_FP32_SPLIT or BGK_FP64");
    if (c->opts.mu_ref > 0.0 && !(std::isfinite(c->opts.mu_ref) && std::isfinite(c->opts.mu_omega)))
        return bail(BGK_EINVAL, "mu_ref and mu_omega must be finite");
    if (c->opts.maxwellian != BGK_MAXWELLIAN_CONSERVATIVE && c->opts.maxwellian != BGK_MAXWELLIAN_CONTINUOUS)
        return bail(BGK_EINVAL, "maxwellian must be BGK_MAXWELLIAN_CONSERVATIVE or BGK_MAXWELLIAN_CONTINUOUS");
    c->prec = c->opts.precision;
    c->esize = c->prec == BGK_FP64 ? 8 : 4;
    c->dim = mesh->dim;
    if (c->dim < 1 || c->dim > 3)
        return bail(BGK_EINVAL, "dim must be 1, 2 or 3");
    if (p < 1 || (c->dim >= 2 && p > 3) || (c->dim == 1 && p > 5))
        return bail(BGK_EINVAL, "p must be in [1, 3] (dim 2, 3) or [1, 5] (dim 1)");
    if (!(tau > 0.0) || !std::isfinite(tau))
        return bail(BGK_EINVAL, "tau must be positive and finite");
    for (int d = 0; d < 3; d++) {
        c->force[d] = c->opts.body_force[d];
        if (!std::isfinite(c->force[d]))
            return bail(BGK_EINVAL, "body force must be finite");
        c->has_force = c->has_force || c->force[d] != 0.0;
    }
    if (c->has_force && c->dim != 3)
        return bail(BGK_EINVAL, "the body-force source is built for hexahedral meshes (dim = 3)");
    c->p = p;
    c->N1 = p + 1;
    c->NP = c->dim == 1 ? c->N1 : (c->dim == 2 ? c->N1 * c->N1 : c->N1 * c->N1 * c->N1);
    int64_t E = 1;
    for (int d = 0; d < 3; d++) {
        if (d < c->dim) {
            c->ne[d] = mesh->nelem[d];
            c->lo[d] = mesh->lo[d];
            c->hi[d] = mesh->hi[d];
            if (c->ne[d] < 1 || !(c->hi[d] > c->lo[d]))
                return bail(BGK_EINVAL, "bad mesh extent");
            for (int s = 0; s < 2; s++) {
                const int b = mesh->bc[d][s];
                if (b != BGK_BC_PERIODIC && b != BGK_BC_DIRICHLET && b != BGK_BC_DIFFUSE_WALL &&
                    b != BGK_BC_EXCHANGE)
                    return bail(BGK_EINVAL, "unknown boundary kind");
                if (b == BGK_BC_EXCHANGE && (d != 0 || c->dim != 3 || c->prec != BGK_FP32_SPLIT))
                    return bail(BGK_EINVAL, "exchange faces are built for the x faces of hexahedral meshes in the "
                                            "FP32-split form");
                if (b == BGK_BC_EXCHANGE)
                    c->has_exchange = true;
                if (b == BGK_BC_DIFFUSE_WALL && c->dim != 3)
                    return bail(BGK_EINVAL, "diffuse walls are built for hexahedral meshes (dim = 3)");
                if (b == BGK_BC_DIFFUSE_WALL)
                    c->has_wall = true;
                c->bc[2 * d + s] = b;
                for (int q = 0; q < 5; q++)
                    c->bcs[(2 * d + s) * 5 + q] = mesh->bc_state[d][s][q];
            }
            if ((c->bc[2 * d] == BGK_BC_PERIODIC) != (c->bc[2 * d + 1] == BGK_BC_PERIODIC))
                return bail(BGK_EINVAL, "periodic faces must come in pairs");
        }
        c->h[d] = (c->hi[d] - c->lo[d]) / c->ne[d];
        E *= c->ne[d];
    }
    if (E * c->NP > INT32_MAX / 2)
        return bail(BGK_EINVAL, "too many points");
    c->E = (int)E;
    c->npts = E * c->NP;
    c->vdim = vg->n[2] == 1 ? 2 : 3;
    if (c->vdim == 2 && c->dim > 2)
        return bail(BGK_EINVAL, "a two-dimensional velocity space (n[2] = 1) needs dim <= 2");
    for (int d = 0; d < c->vdim; d++) {
        if (vg->n[d] < 2 || vg->n[d] > 4096 || !(vg->hi[d] > vg->lo[d]))
            return bail(BGK_EINVAL, "bad velocity grid");
        c->nv[d] = vg->n[d];
        c->vlo[d] = vg->lo[d];
        c->dv[d] = (vg->hi[d] - vg->lo[d]) / (vg->n[d] - 1);
    }
    bool all_two = true;  // on two nodes every function of xi_d is affine in xi_d, so with two on every
    for (int d = 0; d < c->vdim; d++)  // axis |xi|^2 is a combination of 1 and xi: E is not independent
        all_two = all_two && vg->n[d] == 2;
    if (all_two)
        return bail(BGK_EINVAL, "the velocity grid needs 3 or more nodes on some axis (with 2 on every axis "
                                "the energy moment depends on the others and the Maxwellian is not unique)");
    if (c->vdim == 2) {  // the absent u_z axis: one node at 0 of unit weight
        c->nv[2] = 1;
        c->vlo[2] = 0.0;
        c->dv[2] = c->dv[0];
    }
    if (c->opts.mu_ref > 0.0 && c->prec == BGK_FP32_SPLIT && !(c->dv[0] == c->dv[1] && c->dv[0] == c->dv[2]))
        return bail(BGK_EINVAL, "a variable collision time needs one velocity spacing on all axes (FP32-split form)");
    c->nvel = (int64_t)c->nv[0] * c->nv[1] * c->nv[2];
    c->tau = tau;
    build_ops(p, c->ops, c->ops64, c->xg);

    // velocity plan: octants (sign of each component; xi = 0 goes with the positive side)
    std::vector<int> idx[3][2];
    for (int d = 0; d < 3; d++)
        for (int k = 0; k < c->nv[d]; k++)
            idx[d][c->vlo[d] + k * c->dv[d] >= 0.0 ? 1 : 0].push_back(k);
    for (int o = 0; o < 8; o++) {
        const auto &X = idx[0][o & 1], &Y = idx[1][(o >> 1) & 1], &Z = idx[2][(o >> 2) & 1];
        const int64_t n = (int64_t)X.size() * Y.size() * Z.size();
        if (n == 0)
            continue;
        Chunk ch{};
        ch.oct = o;
        ch.vt0 = (int)(c->slotk.size() / kWarp);
        std::vector<int> ks;
        ks.reserve(n);
        for (int kz : Z)
            for (int ky : Y)
                for (int kx : X)
                    ks.push_back(kx + c->nv[0] * (ky + c->nv[1] * kz));
        if (c->dim == 3 && c->nv[0] > 1 && c->nv[1] > 1 && c->nv[2] > 1) {
            // velocities with one component small against another first: on curved hexahedra these are
            // the ones whose flow may enter an element through the face its octant does not make upwind
            // (a face normal tilted against the small component), so they fill a few tiles of their own
            // instead of a few lanes of every tile. Affine meshes are indifferent to the order.
            auto ratio = [&](int k) {
                double a[3];
                const int kk[3] = {k % c->nv[0], (k / c->nv[0]) % c->nv[1], k / (c->nv[0] * c->nv[1])};
                for (int d = 0; d < 3; d++)
                    a[d] = std::fabs(c->vlo[d] + kk[d] * c->dv[d]);
                double r = 1e300;
                for (int d = 0; d < 3; d++) {
                    const double other = std::max(a[(d + 1) % 3], a[(d + 2) % 3]);
                    if (other > 0.0)
                        r = std::min(r, a[d] / other);
                }
                return r;
            };
            std::vector<double> key(ks.size());
            std::vector<int> order(ks.size());
            for (size_t i = 0; i < ks.size(); i++) {
                key[i] = ratio(ks[i]);
                order[i] = (int)i;
            }
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
            for (int i : order)
                c->slotk.push_back(ks[i]);
        } else {
            c->slotk.insert(c->slotk.end(), ks.begin(), ks.end());
        }
        while (c->slotk.size() % kWarp)
            c->slotk.push_back(-1);
        ch.nvt = (int)(c->slotk.size() / kWarp) - ch.vt0;
        c->toct_h.insert(c->toct_h.end(), ch.nvt, (unsigned char)o);
        c->chunks.push_back(ch);
    }
    c->nvt = (int)(c->slotk.size() / kWarp);
    c->nslots = c->nvt * kWarp;
    if (c->opts.chunks == 1 && c->chunks.size() > 1) {
        Chunk all{0, c->nvt, 0, 0, 8};
        c->chunks.assign(1, all);
    }
    int maxc = 0;
    for (auto &ch : c->chunks)
        maxc = std::max(maxc, ch.nvt);
    // tiles per warp task: enough tasks for ~32 resident warps per SM, at most 8 tiles
    if (c->opts.vtiles_per_task > 0)
        c->G = c->opts.vtiles_per_task;
    else {
        const int64_t tasks1 = (int64_t)maxc * E;
        c->G = (int)std::max<int64_t>(1, std::min<int64_t>(8, tasks1 / (152 * 32)));
    }
    c->ngroups = 0;
    for (auto &ch : c->chunks) {
        ch.group0 = c->ngroups;
        ch.ngroups = (ch.nvt + c->G - 1) / c->G;
        c->ngroups += ch.ngroups;
    }
    // the partial-moment table is sized for the shortest task the autotuner tries
    c->max_groups = 0;
    for (auto &ch : c->chunks)
        c->max_groups += (ch.nvt + std::min(c->G, kMinTuneG) - 1) / std::min(c->G, kMinTuneG);
    c->chunk_floats = (int64_t)maxc * E * c->NP * kWarp;

    // mesh descriptor
    c->mesh.dim = c->dim;
    c->mesh.nelem = c->E;
    for (int d = 0; d < 3; d++) {
        c->mesh.ne[d] = c->ne[d];
        c->mesh.inv_h2[d] = (float)(2.0 / c->h[d]);
    }
    for (int q = 0; q < 6; q++)
        c->mesh.bc[q] = c->bc[q];

    // memory check before any allocation
    const int64_t fA = (int64_t)c->nvt * E * c->NP * kWarp;
    const int64_t need = (fA + (int64_t)(c->chunks.size() + 1) * c->chunk_floats) * c->esize +
                         (int64_t)c->max_groups * 5 * c->npts * 4 + c->npts * (5 * 8 * 3 + kParamStride * 4) +
                         (int64_t)c->nslots * 4 * 25 +
                         (c->has_exchange ? 2 * (int64_t)c->nvt * c->ne[1] * c->ne[2] * c->NP * kWarp * 4 : 0);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
        return bail(BGK_ECUDA, "cudaMemGetInfo failed (no CUDA device?)");
    if ((double)need > 0.97 * (double)free_b)
        return bail(BGK_ENOMEM, "configuration needs " + std::to_string(need >> 20) + " MiB, only " +
                                    std::to_string(free_b >> 20) + " MiB free");
    for (int q = 0; q < 6; q++)
        if (q / 2 < c->dim && c->bc[q] == BGK_BC_DIRICHLET && !(c->bcs[q * 5] > 0.0 && c->bcs[q * 5 + 4] > 0.0))
            return bail(BGK_EINVAL, "Dirichlet state needs rho > 0 and T > 0");

#define AL(ptr, n)                                                        \
    if (dalloc(c, &(ptr), (size_t)(n)) != cudaSuccess)                    \
        return bail(BGK_ENOMEM, std::string("cudaMalloc failed: ") + #ptr);
    if (c->prec == BGK_FP64) {
        AL(c->fA64, fA);
        AL(c->pool64, (c->chunks.size() + 1) * c->chunk_floats);
        AL(c->xi64, 3 * c->nslots);
        AL(c->wpsi64, 5 * c->nslots);
        AL(c->ghost64, 6 * c->nslots);
        AL(c->par64, c->npts * 5);
        if (c->opts.mu_ref > 0.0)
            AL(c->itau64, c->npts);
    } else {
        AL(c->fA, fA);
        AL(c->pool, (c->chunks.size() + 1) * c->chunk_floats);
    }
    AL(c->xi, 3 * c->nslots);
    AL(c->mi, 3 * c->nslots);
    AL(c->toct, c->nvt);
    AL(c->wpsi, 5 * c->nslots);
    AL(c->vtab, 5 * c->nslots);
    if (c->has_exchange) {  // halos of the exchange faces, zero until bgk_set_halo
        c->halo_floats = (int64_t)c->nvt * c->ne[1] * c->ne[2] * c->NP * kWarp;
        for (int f = 0; f < 2; f++)
            if (c->bc[f] == BGK_BC_EXCHANGE) {
                AL(c->halo_own[f], c->halo_floats);
                c->halo[f] = c->halo_own[f];
            }
    }
    AL(c->gmask, c->nslots);
    AL(c->ghost, 6 * c->nslots);
    AL(c->slotk_d, c->nslots);
    c->nfmax = std::max(c->ne[1] * c->ne[2], std::max(c->ne[0] * c->ne[2], c->ne[0] * c->ne[1]));
    if (c->has_wall) {
        if (c->prec == BGK_FP64) {
            AL(c->rhow64, 6ll * c->nfmax * c->N1 * c->N1);
            AL(c->w64, c->nslots);
        } else {
            AL(c->rhow32, 6ll * c->nfmax * c->N1 * c->N1);
            AL(c->w32, c->nslots);
        }
    }
    if (c->has_force) {
        AL(c->fpar32, c->npts * kParamStride);
        if (c->prec == BGK_FP64)
            AL(c->fpar64, c->npts * 5);
    }
    AL(c->partial, (int64_t)c->max_groups * 5 * c->npts);
    AL(c->param, c->npts * kParamStride);
    AL(c->Q, c->npts * 5);
    AL(c->prim, c->npts * 5);
    AL(c->prim_in, c->npts * 5);
    AL(c->err, 1);
#undef AL
    // velocity tables
    std::vector<float> xi(3 * c->nslots), mi(3 * c->nslots), wpsi(5 * c->nslots), gm(c->nslots), gh(6 * c->nslots, 0.f);
    std::vector<float> vtab(5 * c->nslots);
    std::vector<double> xi64(3 * c->nslots), wpsi64(5 * c->nslots), gh64(6 * c->nslots, 0.0), w64h(c->nslots);
    std::vector<float> w32h(c->nslots);
    double win[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < c->nslots; s++) {
        int k = c->slotk[s];
        const bool real = k >= 0;
        if (!real) {  // padding: a copy of the tile's first velocity, zero weight, no relaxation
            k = c->slotk[(s / kWarp) * kWarp];
        }
        const int kk[3] = {k % c->nv[0], (k / c->nv[0]) % c->nv[1], k / (c->nv[0] * c->nv[1])};
        double v[3], w = 1.0;
        for (int d = 0; d < 3; d++) {
            v[d] = c->vlo[d] + kk[d] * c->dv[d];
            if (c->nv[d] > 1)
                w *= end_factor(kk[d], c->nv[d]) * c->dv[d];
            xi[d * c->nslots + s] = (float)v[d];
            xi64[d * c->nslots + s] = v[d];
            mi[d * c->nslots + s] = (float)(2 * kk[d] - (c->nv[d] - 1));
        }
        if (!real)
            w = 0.0;
        const int vt = s / kWarp, l = s % kWarp;
        const double ps[5] = {1.0, v[0], v[1], v[2], 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])};
        // FP32 kernels: exact index-basis weights W (1, m, sum_d r_d m_d^2) (see index_to_moments)
        double W = real ? 1.0 : 0.0, m[3], mr = 0.0;
        for (int d = 0; d < 3; d++) {
            W *= end_factor(kk[d], c->nv[d]);
            m[d] = 2.0 * kk[d] - (c->nv[d] - 1);
            mr += (double)index_r(c->dv[d], c->dv[0]) * m[d] * m[d];
        }
        const double pi[5] = {1.0, m[0], m[1], m[2], mr};
        for (int q = 0; q < 5; q++) {
            wpsi[((int64_t)vt * 5 + q) * kWarp + l] = (float)(W * pi[q]);
            wpsi64[(int64_t)s * 5 + q] = w * ps[q];
        }
        for (int d = 0; d < 3; d++)
            vtab[((int64_t)vt * 5 + d) * kWarp + l] = (float)m[d];
        vtab[((int64_t)vt * 5 + 3) * kWarp + l] = (float)(W * pi[0]);
        vtab[((int64_t)vt * 5 + 4) * kWarp + l] = (float)(W * pi[4]);
        gm[s] = real ? 1.f : 0.f;
        w32h[s] = (float)w;
        w64h[s] = w;
        for (int q = 0; q < 6; q++)
            if (q / 2 < c->dim && (c->bc[q] == BGK_BC_DIRICHLET || c->bc[q] == BGK_BC_DIFFUSE_WALL) && real) {
                // Dirichlet: the prescribed Maxwellian; diffuse wall: the unit-density wall Maxwellian
                const double *st = c->bcs + 5 * q;
                const double rho = c->bc[q] == BGK_BC_DIRICHLET ? st[0] : 1.0;
                gh64[q * c->nslots + s] = maxwell(c->vdim, rho, st + 1, st[4], v[0], v[1], v[2]);
                gh[q * c->nslots + s] = (float)gh64[q * c->nslots + s];
                if (c->bc[q] == BGK_BC_DIFFUSE_WALL) {
                    const double un = (q & 1) ? v[q / 2] : -v[q / 2];  // xi . n_out
                    if (un < 0.0)
                        win[q] += w * (-un) * gh64[q * c->nslots + s];
                }
            }
    }
    for (int q = 0; q < 6; q++)
        c->inv_in[q] = (c->bc[q] == BGK_BC_DIFFUSE_WALL && win[q] > 0.0) ? 1.0 / win[q] : 0.0;
    cudaError_t rc;
    if ((c->w32 && (rc = cudaMemcpy(c->w32, w32h.data(), w32h.size() * 4, cudaMemcpyHostToDevice))) ||
        (c->w64 && (rc = cudaMemcpy(c->w64, w64h.data(), w64h.size() * 8, cudaMemcpyHostToDevice))) ||
        (rc = cudaMemcpy(c->xi, xi.data(), xi.size() * 4, cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->mi, mi.data(), mi.size() * 4, cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->toct, c->toct_h.data(), c->toct_h.size(), cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->wpsi, wpsi.data(), wpsi.size() * 4, cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->vtab, vtab.data(), vtab.size() * 4, cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->gmask, gm.data(), gm.size() * 4, cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->ghost, gh.data(), gh.size() * 4, cudaMemcpyHostToDevice)) ||
        (rc = cudaMemcpy(c->slotk_d, c->slotk.data(), c->slotk.size() * 4, cudaMemcpyHostToDevice)) ||
        (c->prec == BGK_FP64 &&
         ((rc = cudaMemcpy(c->xi64, xi64.data(), xi64.size() * 8, cudaMemcpyHostToDevice)) ||
          (rc = cudaMemcpy(c->wpsi64, wpsi64.data(), wpsi64.size() * 8, cudaMemcpyHostToDevice)) ||
          (rc = cudaMemcpy(c->ghost64, gh64.data(), gh64.size() * 8, cudaMemcpyHostToDevice)) ||
          (rc = cudaMemset(c->fA64, 0, fA * 8)) || (rc = cudaMemset(c->par64, 0, c->npts * 5 * 8)))) ||
        (c->prec != BGK_FP64 && (rc = cudaMemset(c->fA, 0, fA * 4))) || (rc = cudaMemset(c->err, 0, 4)) ||
        (rc = cudaMemset(c->prim, 0, c->npts * 5 * 8)) || (rc = cudaMemset(c->param, 0, c->npts * kParamStride * 4)))
        return bail(BGK_ECUDA, std::string("device set-up copy failed: ") + cudaGetErrorString(rc));
    // the set-up memsets may still run on the legacy stream, which work on a non-blocking stream
    // (the context's own, or the caller's) does not wait for: finish them here
    if ((rc = cudaDeviceSynchronize()) != cudaSuccess)
        return bail(BGK_ECUDA, std::string("device set-up failed: ") + cudaGetErrorString(rc));
    if (prepare_stage(c->dim, p) != cudaSuccess)
        return bail(BGK_ECUDA, "stage kernel attribute set-up failed");
    if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess)
        return bail(BGK_ECUDA, "stream creation failed");
    c->stream = c->own;
    *out = c;
    return BGK_OK;
}

int bgk_set_stream(bgk_ctx *c, void *stream)
{
    if (!c)
        return BGK_EINVAL;
    c->stream = stream ? (cudaStream_t)stream : c->own;
    return BGK_OK;
}

int bgk_info(const bgk_ctx *c, int64_t *npoints, int64_t *nvel, int64_t *ndof, int64_t *device_bytes)
{
    if (!c)
        return BGK_EINVAL;
    if (npoints)
        *npoints = c->npts;
    if (nvel)
        *nvel = c->nvel;
    if (ndof)
        *ndof = c->npts * c->nvel;
    if (device_bytes)
        *device_bytes = c->bytes;
    return BGK_OK;
}

int bgk_points(const bgk_ctx *c, double *x)
{
    if (!c || !x)
        return BGK_EINVAL;
    if (!c->geom.empty()) {
        std::copy(c->geom.begin(), c->geom.end(), x);
        return BGK_OK;
    }
    for (int64_t pt = 0; pt < c->npts; pt++) {
        const int e = (int)(pt / c->NP), i = (int)(pt % c->NP);
        const int ec[3] = {e % c->ne[0], (e / c->ne[0]) % c->ne[1], e / (c->ne[0] * c->ne[1])};
        const int ic[3] = {i % c->N1, (i / c->N1) % c->N1, i / (c->N1 * c->N1)};
        for (int d = 0; d < 3; d++)
            x[pt * 3 + d] = d < c->dim ? c->lo[d] + (ec[d] + 0.5 * (c->xg[ic[d]] + 1.0)) * c->h[d] : 0.0;
    }
    return BGK_OK;
}

static int set_state_impl(bgk_ctx *c, const double *prim, cudaMemcpyKind kind)
{
    CK(cudaMemcpyAsync(c->prim_in, prim, c->npts * 5 * sizeof(double), kind, c->stream));
    if (c->prec == BGK_FP64)
        CK(launch_init64(c->fA64, c->prim_in, c->xi64, c->gmask, c->nvt, c->E, c->NP, c->nslots, c->vdim, c->err,
                         c->stream));
    else
        CK(launch_init_maxwellian(c->fA, c->prim_in, c->mi, c->gmask, c->nslots, c->nvt, c->E, c->NP, c->nv, c->vlo,
                                  c->dv, c->err, c->Q, c->prim, c->stream));
    return prologue(c, c->stream, c->prec != BGK_FP64);
}

int bgk_set_state(bgk_ctx *c, const double *prim)
{
    if (!c || !prim)
        return BGK_EINVAL;
    int rc = set_state_impl(c, prim, cudaMemcpyHostToDevice);
    if (rc)
        return rc;
    return read_status(c);
}

int bgk_set_state_device(bgk_ctx *c, const double *d_prim)
{
    if (!c || !d_prim)
        return BGK_EINVAL;
    return set_state_impl(c, d_prim, cudaMemcpyDeviceToDevice);
}

static int convert_impl(bgk_ctx *c, double *f, bool in)
{
    const int64_t per_pt = c->nvel * (int64_t)sizeof(double);
    int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(c->npts, (256ll << 20) / per_pt));
    double *st = nullptr;
    CK(cudaMalloc(&st, chunk * per_pt));
    int rc = BGK_OK;
    for (int64_t p0 = 0; p0 < c->npts && rc == BGK_OK; p0 += chunk) {
        const int64_t n = std::min(chunk, c->npts - p0);
        cudaError_t e = cudaSuccess;
        if (in) {
            e = cudaMemcpyAsync(st, f + p0 * c->nvel, n * per_pt, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = c->prec == BGK_FP64
                        ? launch_convert64(true, c->fA64, st, c->slotk_d, c->nvt, c->E, c->NP, c->nvel, (int)p0,
                                           (int)n, c->stream)
                        : launch_convert_f(true, c->fA, st, c->slotk_d, c->nvt, c->E, c->NP, c->nvel, (int)p0,
                                           (int)n, c->stream);
        } else {
            e = c->prec == BGK_FP64
                    ? launch_convert64(false, c->fA64, st, c->slotk_d, c->nvt, c->E, c->NP, c->nvel, (int)p0, (int)n,
                                       c->stream)
                    : launch_convert_f(false, c->fA, st, c->slotk_d, c->nvt, c->E, c->NP, c->nvel, (int)p0, (int)n,
                                       c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(f + p0 * c->nvel, st, n * per_pt, cudaMemcpyDeviceToHost, c->stream);
        }
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            rc = cuda_fail(c, e, "f conversion");
    }
    cudaFree(st);
    return rc;
}

int bgk_set_f(bgk_ctx *c, const double *f)
{
    if (!c || !f)
        return BGK_EINVAL;
    int rc = convert_impl(c, const_cast<double *>(f), true);
    if (rc)
        return rc;
    rc = prologue(c, c->stream);
    if (rc)
        return rc;
    return read_status(c);
}

int bgk_get_f(bgk_ctx *c, double *f)
{
    if (!c || !f)
        return BGK_EINVAL;
    return convert_impl(c, f, false);
}

int bgk_f_distance(bgk_ctx *a, bgk_ctx *b, double *max_abs_diff, double *max_abs_b)
{
    if (!a || !b || !max_abs_diff || !max_abs_b)
        return BGK_EINVAL;
    if (a->E != b->E || a->NP != b->NP || a->nvt != b->nvt || a->nvel != b->nvel || a->slotk != b->slotk)
        return fail(a, BGK_EINVAL, "bgk_f_distance: the two contexts have different meshes or velocity plans");
    bgk_ctx *c = a;  // errors are reported on a
    // both contexts' work before the comparison: b's stream first, then a's, which runs the kernel
    CK(cudaStreamSynchronize(b->stream));
    unsigned long long *d = nullptr, h[2] = {0, 0};
    CK(cudaMalloc(&d, sizeof(h)));
    cudaError_t e = launch_f_distance(a->prec == BGK_FP64 ? (const void *)a->fA64 : (const void *)a->fA,
                                      a->prec == BGK_FP64, b->prec == BGK_FP64 ? (const void *)b->fA64 : (const void *)b->fA,
                                      b->prec == BGK_FP64, a->slotk_d, a->nvt, a->E, a->NP, d, a->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, a->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(a->stream);
    cudaFree(d);
    if (e != cudaSuccess)
        return cuda_fail(a, e, "bgk_f_distance");
    std::memcpy(max_abs_diff, &h[0], sizeof(double));
    std::memcpy(max_abs_b, &h[1], sizeof(double));
    return BGK_OK;
}

int bgk_halo_floats(const bgk_ctx *c, int64_t *nfloats)
{
    if (!c || !nfloats)
        return BGK_EINVAL;
    *nfloats = c->halo_floats;
    return BGK_OK;
}

int bgk_set_halo(bgk_ctx *c, int face, const float *d_halo)
{
    if (!c || face < 0 || face > 1)
        return BGK_EINVAL;
    if (c->bc[face] != BGK_BC_EXCHANGE)
        return fail(c, BGK_EINVAL, "bgk_set_halo: the face is not an exchange face");
    c->halo[face] = d_halo ? d_halo : c->halo_own[face];
    return BGK_OK;
}

int bgk_halo_pack(bgk_ctx *c, int stage, float *d_lo, float *d_hi)
{
    if (!c || stage < 0 || stage > 2)
        return BGK_EINVAL;
    if (!c->has_exchange || c->prec != BGK_FP32_SPLIT)
        return fail(c, BGK_EINVAL, "bgk_halo_pack: no exchange faces");
    const size_t row = (size_t)c->NP * kWarp * sizeof(float);  // one element of one tile
    const int ef = c->ne[1] * c->ne[2];
    for (int side = 0; side < 2; side++) {
        float *dst = side ? d_hi : d_lo;
        if (!dst)
            continue;
        const int ex = side ? c->ne[0] - 1 : 0;
        for (int q = 0; q < (int)c->chunks.size(); q++) {
            // rows (tile, face element) of the chunk's stage source: element ex + ne_x r of tile vt, at a
            // uniform pitch of ne_x elements
            const float *src = stage_source(c, q, stage) + (int64_t)ex * c->NP * kWarp;
            float *d = dst + (int64_t)c->chunks[q].vt0 * ef * c->NP * kWarp;
            CK(cudaMemcpy2DAsync(d, row, src, row * c->ne[0], row, (size_t)c->chunks[q].nvt * ef,
                                 cudaMemcpyDeviceToDevice, c->stream));
        }
    }
    return BGK_OK;
}

int bgk_stage(bgk_ctx *c, double dt, int stage)
{
    if (!c || stage < 0 || stage > 2 || !(dt > 0.0) || !std::isfinite(dt))
        return BGK_EINVAL;
    if (c->prec != BGK_FP32_SPLIT)
        return fail(c, BGK_EINVAL, "bgk_stage is built for the FP32-split form");
    if (c->ftab && !c->met)
        return fail(c, BGK_EINVAL, "unstructured connectivity needs bgk_set_geometry before stepping");
    if (c->sticky)
        return read_status(c);
    return enqueue_stage(c, dt, stage, c->stream);
}

int bgk_step(bgk_ctx *c, double dt, int nsteps)
{
    if (!c || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt))
        return BGK_EINVAL;
    if (c->ftab && !c->met)  // a connectivity table means nothing without the elements' node coordinates
        return fail(c, BGK_EINVAL, "unstructured connectivity needs bgk_set_geometry before stepping");
    if (c->has_exchange)  // the halos must be refreshed between the stages
        return fail(c, BGK_EINVAL, "a context with exchange faces steps by bgk_stage, with a halo exchange before "
                                   "every stage");
    if (c->sticky)
        return read_status(c);
    if (nsteps == 0)
        return BGK_OK;
    if (c->timing) {
        for (int n = 0; n < nsteps; n++) {
            int rc = enqueue_step(c, dt, c->stream);
            if (rc)
                return rc;
        }
        return BGK_OK;
    }
    if (!c->gexec || c->gdt != dt) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaStream_t cap;
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_fail(c, e, "cudaStreamBeginCapture");
        }
        int rc = enqueue_step(c, dt, cap);
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (rc)
            return rc;
        CK(e);
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        c->gdt = dt;
    }
    for (int n = 0; n < nsteps; n++)
        CK(cudaGraphLaunch(c->gexec, c->stream));
    return BGK_OK;
}

int bgk_moments(bgk_ctx *c, double *Q)
{
    if (!c || !Q)
        return BGK_EINVAL;
    CK(cudaMemcpyAsync(Q, c->Q, c->npts * 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return read_status(c);
}

int bgk_moments_device(bgk_ctx *c, double *d_Q)
{
    if (!c || !d_Q)
        return BGK_EINVAL;
    CK(cudaMemcpyAsync(d_Q, c->Q, c->npts * 5 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return BGK_OK;
}

int bgk_equilibrium(bgk_ctx *c, double *prim_out)
{
    if (!c || !prim_out)
        return BGK_EINVAL;
    CK(cudaMemcpyAsync(prim_out, c->prim, c->npts * 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    const int rc = read_status(c);
    // the Newton kernel keeps lnC = ln(rho' (2 pi theta')^(-m/2)) as its warm start: rho' from it
    for (int64_t i = 0; i < c->npts; i++) {
        double *pp = prim_out + i * 5;
        pp[0] = pp[4] > 0.0 ? exp(pp[0]) * pow(2.0 * kPi * pp[4], 0.5 * c->vdim) : 0.0;
    }
    return rc;
}

int bgk_synchronize(bgk_ctx *c)
{
    if (!c)
        return BGK_EINVAL;
    return read_status(c);
}

double bgk_dt(const bgk_ctx *c, double cfl)
{
    if (!c)
        return -1.0;
    double smax = 0.0;
    for (int64_t k = 0; k < c->nvel; k++) {
        const int kk[3] = {(int)(k % c->nv[0]), (int)((k / c->nv[0]) % c->nv[1]), (int)(k / (c->nv[0] * c->nv[1]))};
        double s = 0.0;
        for (int d = 0; d < c->dim; d++)
            s += fabs(c->vlo[d] + kk[d] * c->dv[d]) / c->h[d];
        smax = std::max(smax, s);
    }
    if (c->met)  // curvilinear: the metric's transport speed in reference units (the affine value above)
        smax = c->curv_smax;
    double tmin = c->tau;
    if (c->opts.mu_ref > 0.0) {  // the smallest collision time of the current state
        std::vector<double> Q(c->npts * 5);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
            cudaMemcpy(Q.data(), c->Q, Q.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return -1.0;
        tmin = INFINITY;
        for (int64_t i = 0; i < c->npts; i++) {
            const double *q = &Q[i * 5];
            const double rho = q[0],
                         th = (2.0 / c->vdim) * (q[4] / rho - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / (rho * rho));
            tmin = std::min(tmin, c->opts.mu_ref * pow(th, c->opts.mu_omega) / (rho * th));
        }
    }
    return std::min(cfl / smax, tmin);
}


// ------------------------------------------------------------------------------------------------
// Curvilinear hexahedra. Every element maps the reference cube by the degree-p interpolant of its
// solution-node coordinates. Metric terms (Kopriva's conservative curl form, so the discrete metric
// identities hold and a constant state is kept): Ja^i_n = -(curl_r (X_l grad_r X_m))_i for (n, m, l)
// cyclic, with every product taken at the nodes and differentiated with the FR derivative matrix.
// Face normals: Ja^d interpolated to the face from both elements and averaged (single-valued, so the
// upwind flux is conservative); a non-periodic boundary face keeps the element's own.
// ------------------------------------------------------------------------------------------------
namespace {

// d/dr_j of a nodal field u[NP] (x fastest) with the FP64 derivative matrix
void dref(const bgk_ctx *c, const double *u, int j, double *out)
{
    const int n = c->N1, stride = j == 0 ? 1 : (j == 1 ? n : n * n);
    for (int i = 0; i < c->NP; i++) {
        const int ij = (i / stride) % n, base = i - ij * stride;
        double a = 0.0;
        for (int k = 0; k < n; k++)
            a += c->ops64.D[ij][k] * u[base + k * stride];
        out[i] = a;
    }
}

}  // namespace

int bgk_set_connectivity(bgk_ctx *c, const int *nbr, const int *nface, const int *orient)
{
    if (!c || !nbr || !nface || !orient)
        return BGK_EINVAL;
    if (c->has_exchange)
        return fail(c, BGK_EINVAL, "exchange faces are built for the affine structured mesh");
    if (c->dim != 3)
        return fail(c, BGK_EINVAL, "unstructured connectivity is built for hexahedra (dim = 3)");
    const int E = c->E, N1 = c->N1, NQ = N1 * N1;
    for (int64_t q = 0; q < (int64_t)E * 6; q++) {
        if (nbr[q] >= E || nbr[q] < -6 || nface[q] < 0 || nface[q] > 5 || orient[q] < 0 || orient[q] > 7)
            return fail(c, BGK_EINVAL, "connectivity table entry out of range at " + std::to_string(q));
        if (nbr[q] < 0 && c->bc[-1 - nbr[q]] != BGK_BC_DIRICHLET && c->bc[-1 - nbr[q]] != BGK_BC_DIFFUSE_WALL)
            return fail(c, BGK_EINVAL, "a boundary face must take the data of a Dirichlet or diffuse-wall face");
    }
    std::vector<int4> tab((size_t)E * 6);
    std::vector<unsigned char> base((size_t)E * 6 * NQ);
    c->wlist_h.clear();
    c->wall_idx.assign((size_t)E * 6, -1);
    for (int e = 0; e < E; e++)
        for (int f = 0; f < 6; f++) {
            const int q = e * 6 + f, dn = nface[q] / 2, o = orient[q];
            const int stride = dn == 0 ? 1 : (dn == 1 ? N1 : NQ);
            int wi = -1;
            if (nbr[q] < 0 && c->bc[-1 - nbr[q]] == BGK_BC_DIFFUSE_WALL) {
                wi = (int)c->wlist_h.size();
                c->wlist_h.push_back(make_int4(e, f, -1 - nbr[q], 0));
            }
            c->wall_idx[q] = wi;
            tab[q] = make_int4(nbr[q], stride, nface[q] % 2, wi);
            // face point (a, b) of our face -> the neighbour's (a', b') along its other axes (increasing)
            const int s1 = dn == 0 ? N1 : 1, s2 = dn == 2 ? N1 : NQ;
            for (int ln = 0; ln < NQ; ln++) {
                const int a = ln % N1, b = ln / N1;
                int an = (o & 1) ? b : a, bn = (o & 1) ? a : b;
                if (o & 2)
                    an = N1 - 1 - an;
                if (o & 4)
                    bn = N1 - 1 - bn;
                base[(size_t)q * NQ + ln] = (unsigned char)(an * s1 + bn * s2);
            }
        }
    if (!c->ftab) {
        CK(dalloc(c, &c->ftab, tab.size()));
        CK(dalloc(c, &c->fbase, base.size()));
    }
    CK(cudaMemcpy(c->ftab, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->fbase, base.data(), base.size(), cudaMemcpyHostToDevice));
    if (!c->wlist_h.empty()) {  // the wall-face list, its normals (set with the geometry) and densities
        const size_t nw = c->wlist_h.size();
        if (c->wlist) {
            cudaFree(c->wlist);
            cudaFree(c->wnu);
            cudaFree(c->rhowu32);
            cudaFree(c->rhowu64);
            c->wlist = nullptr;
            c->wnu = nullptr;
            c->rhowu32 = nullptr;
            c->rhowu64 = nullptr;
        }
        CK(dalloc(c, &c->wlist, nw));
        CK(dalloc(c, &c->wnu, nw * NQ * 4));
        CK(cudaMemset(c->wnu, 0, nw * NQ * 4 * sizeof(double)));
        if (c->prec == BGK_FP64)
            CK(dalloc(c, &c->rhowu64, nw * NQ));
        else
            CK(dalloc(c, &c->rhowu32, nw * NQ));
        CK(cudaMemcpy(c->wlist, c->wlist_h.data(), nw * sizeof(int4), cudaMemcpyHostToDevice));
    }
    c->cnbr.assign(nbr, nbr + (size_t)E * 6);
    c->cface.assign(nface, nface + (size_t)E * 6);
    c->corient.assign(orient, orient + (size_t)E * 6);
    if (!c->geom.empty()) {  // face normals follow the new neighbours
        const std::vector<double> x = c->geom;
        return bgk_set_geometry(c, x.data());
    }
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BGK_OK;
}

int bgk_set_geometry(bgk_ctx *c, const double *x)
{
    if (!c || !x)
        return BGK_EINVAL;
    if (c->has_exchange)
        return fail(c, BGK_EINVAL, "exchange faces are built for the affine structured mesh");
    if (c->dim != 3)
        return fail(c, BGK_EINVAL, "curvilinear geometry is built for hexahedra (dim = 3)");
    const int NP = c->NP, N1 = c->N1, NQ = N1 * N1, E = c->E;
    std::vector<double> Ja((size_t)c->npts * 9), J(c->npts);
    std::vector<double> X(NP), dX(9 * (size_t)NP), V(NP), dV(9 * (size_t)NP);
    int64_t bad = 0;
    for (int e = 0; e < E; e++) {
        const double *xe = x + (int64_t)e * NP * 3;
        for (int n = 0; n < 3; n++) {  // dX[n][j] = dX_n / dr_j
            for (int i = 0; i < NP; i++)
                X[i] = xe[3 * i + n];
            for (int j = 0; j < 3; j++)
                dref(c, X.data(), j, &dX[(size_t)(3 * n + j) * NP]);
        }
        double *Je = &J[(size_t)e * NP], *Jae = &Ja[(size_t)e * NP * 9];
        for (int i = 0; i < NP; i++) {
            double M[3][3];
            for (int n = 0; n < 3; n++)
                for (int j = 0; j < 3; j++)
                    M[n][j] = dX[(size_t)(3 * n + j) * NP + i];
            Je[i] = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                    M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            bad += !(Je[i] > 0.0);
        }
        for (int n = 0; n < 3; n++) {
            const int m = (n + 1) % 3, l = (n + 2) % 3;
            for (int j = 0; j < 3; j++) {  // V_j = X_l dX_m/dr_j; dV[j][k] = d V_j / d r_k
                for (int i = 0; i < NP; i++)
                    V[i] = xe[3 * i + l] * dX[(size_t)(3 * m + j) * NP + i];
                for (int k = 0; k < 3; k++)
                    dref(c, V.data(), k, &dV[(size_t)(3 * j + k) * NP]);
            }
            for (int i = 0; i < NP; i++) {
                auto g = [&](int j, int k) { return dV[(size_t)(3 * j + k) * NP + i]; };
                Jae[(size_t)i * 9 + 0 * 3 + n] = -(g(2, 1) - g(1, 2));
                Jae[(size_t)i * 9 + 1 * 3 + n] = -(g(0, 2) - g(2, 0));
                Jae[(size_t)i * 9 + 2 * 3 + n] = -(g(1, 0) - g(0, 1));
            }
        }
    }
    if (bad)
        return fail(c, BGK_EINVAL, "curvilinear geometry: J <= 0 at " + std::to_string(bad) + " nodes");
    // face normals [E][3][2][NQ] and the per-element sum of W J
    auto own_face = [&](int e, int d, int side, int ln, double *Nv) {
        const int a = ln % N1, bq = ln / N1;  // face point: the two other coordinates in increasing axis order
        int ic[3];
        Nv[0] = Nv[1] = Nv[2] = 0.0;
        for (int j = 0; j < N1; j++) {
            if (d == 0) { ic[0] = j; ic[1] = a; ic[2] = bq; }
            else if (d == 1) { ic[0] = a; ic[1] = j; ic[2] = bq; }
            else { ic[0] = a; ic[1] = bq; ic[2] = j; }
            const int node = ic[0] + N1 * (ic[1] + N1 * ic[2]);
            const double lj = side ? c->ops64.lp[j] : c->ops64.lm[j];
            for (int n = 0; n < 3; n++)
                Nv[n] += lj * Ja[((size_t)e * NP + node) * 9 + d * 3 + n];
        }
    };
    std::vector<float4> met((size_t)E * NP * 3), fn((size_t)E * 6 * NQ);
    std::vector<double> wn(c->has_wall ? (size_t)6 * c->nfmax * NQ * 4 : 0, 0.0);  // curved wall normals
    std::vector<double> fn64_src((size_t)E * 6 * NQ * 3);                           // face normals in FP64
    std::vector<double> wnu(c->wlist_h.size() * NQ * 4, 0.0);                        // unstructured wall normals
    std::vector<float> iwj(E);
    for (int e = 0; e < E; e++) {
        const int ec[3] = {e % c->ne[0], (e / c->ne[0]) % c->ne[1], e / (c->ne[0] * c->ne[1])};
        double wj = 0.0;
        for (int i = 0; i < NP; i++) {
            const double W = c->ops64.wq[i % N1] * c->ops64.wq[(i / N1) % N1] * c->ops64.wq[i / NQ];
            const double Jv = J[(size_t)e * NP + i];
            const double *a = &Ja[((size_t)e * NP + i) * 9];
            wj += W * Jv;
            for (int d = 0; d < 3; d++)
                met[((size_t)e * NP + i) * 3 + d] = make_float4((float)a[d * 3], (float)a[d * 3 + 1], (float)a[d * 3 + 2],
                                                               (float)(d == 1 ? W * Jv : 1.0 / Jv));
        }
        iwj[e] = (float)(1.0 / wj);
        for (int d = 0; d < 3; d++)
            for (int side = 0; side < 2; side++) {
                int nc[3] = {ec[0], ec[1], ec[2]};
                nc[d] += side ? 1 : -1;
                const bool outside = nc[d] < 0 || nc[d] >= c->ne[d];
                bool shared = !outside || c->bc[2 * d + side] == BGK_BC_PERIODIC;
                nc[d] = (nc[d] + c->ne[d]) % c->ne[d];
                int en = nc[0] + c->ne[0] * (nc[1] + c->ne[1] * nc[2]);
                int dn = d, sn = 1 - side, orient = 0;
                if (!c->cnbr.empty()) {  // unstructured: the table's neighbour, shared face and orientation
                    en = c->cnbr[(size_t)e * 6 + 2 * d + side];
                    shared = en >= 0;
                    dn = c->cface[(size_t)e * 6 + 2 * d + side] / 2;
                    sn = c->cface[(size_t)e * 6 + 2 * d + side] % 2;
                    orient = c->corient[(size_t)e * 6 + 2 * d + side];
                }
                for (int ln = 0; ln < NQ; ln++) {
                    double Nv[3], Nn[3];
                    own_face(e, d, side, ln, Nv);
                    if (shared) {
                        // the neighbour's face point of ours, its Ja^{d'} there, and the sign that turns its
                        // +r_{d'} into our +r_d (equal directions when the shared faces have opposite sides)
                        int a = ln % N1, bq = ln / N1;
                        int an = (orient & 1) ? bq : a, bn = (orient & 1) ? a : bq;
                        if (orient & 2)
                            an = N1 - 1 - an;
                        if (orient & 4)
                            bn = N1 - 1 - bn;
                        own_face(en, dn, sn, an + N1 * bn, Nn);
                        const double sg = sn != side ? 1.0 : -1.0;
                        for (int n = 0; n < 3; n++)
                            Nv[n] = 0.5 * (Nv[n] + sg * Nn[n]);
                    }
                    fn[(((size_t)e * 3 + d) * 2 + side) * NQ + ln] = make_float4((float)Nv[0], (float)Nv[1], (float)Nv[2], 0.f);
                    for (int n = 0; n < 3; n++)
                        fn64_src[((((size_t)e * 3 + d) * 2 + side) * NQ + ln) * 3 + n] = Nv[n];
                    const int wi = c->wall_idx.empty() ? -1 : c->wall_idx[(size_t)e * 6 + 2 * d + side];
                    if (wi >= 0) {  // a wall face of the unstructured mesh: its outward unit normal
                        const double nn = sqrt(Nv[0] * Nv[0] + Nv[1] * Nv[1] + Nv[2] * Nv[2]), sg = side ? 1.0 : -1.0;
                        for (int n = 0; n < 3; n++)
                            wnu[((size_t)wi * NQ + ln) * 4 + n] = sg * Nv[n] / nn;
                    }
                    if (c->cnbr.empty() && !shared && c->bc[2 * d + side] == BGK_BC_DIFFUSE_WALL) {
                        // outward unit normal of the wall face point, at the wall kernel's face element index
                        const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
                        const int fe = ec[o1] + c->ne[o1] * ec[o2];
                        const double nn = sqrt(Nv[0] * Nv[0] + Nv[1] * Nv[1] + Nv[2] * Nv[2]), sg = side ? 1.0 : -1.0;
                        double *o = &wn[(((size_t)(2 * d + side) * c->nfmax + fe) * NQ + ln) * 4];
                        for (int n = 0; n < 3; n++)
                            o[n] = sg * Nv[n] / nn;
                    }
                }
            }
    }
    // stable-step speed: the maximum over a node's velocities of the convex sum_d |Ja^d . xi| is at a
    // corner of the velocity box
    double smax = 0.0;
    for (int64_t i = 0; i < c->npts; i++)
        for (int corner = 0; corner < 8; corner++) {
            double v[3];
            for (int d = 0; d < 3; d++)
                v[d] = c->vlo[d] + ((corner >> d) & 1 ? (c->nv[d] - 1) * c->dv[d] : 0.0);
            double sum = 0.0;
            for (int d = 0; d < 3; d++) {
                const double *a = &Ja[(size_t)i * 9 + d * 3];
                sum += fabs(a[0] * v[0] + a[1] * v[1] + a[2] * v[2]);
            }
            smax = std::max(smax, sum / (2.0 * J[i]));
        }
    if (!c->met) {
        CK(dalloc(c, &c->met, met.size()));
        CK(dalloc(c, &c->fnm, fn.size()));
        CK(dalloc(c, &c->iwj, iwj.size()));
    }
    CK(cudaMemcpy(c->met, met.data(), met.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->fnm, fn.data(), fn.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->iwj, iwj.data(), iwj.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (c->has_wall && c->cnbr.empty()) {
        if (!c->wn64)
            CK(dalloc(c, &c->wn64, wn.size()));
        CK(cudaMemcpy(c->wn64, wn.data(), wn.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (!wnu.empty())
        CK(cudaMemcpy(c->wnu, wnu.data(), wnu.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (c->prec == BGK_FP64) {  // the all-FP64 form reads the metric, 1/J and the face normals in FP64
        std::vector<double> ij(c->npts), fn64((size_t)E * 6 * NQ * 3);
        for (int64_t i = 0; i < c->npts; i++)
            ij[i] = 1.0 / J[i];
        for (size_t q = 0; q < fn.size(); q++)
            for (int n = 0; n < 3; n++)
                fn64[q * 3 + n] = fn64_src[q * 3 + n];
        if (!c->ja64) {
            CK(dalloc(c, &c->ja64, Ja.size()));
            CK(dalloc(c, &c->ijac64, ij.size()));
            CK(dalloc(c, &c->fnm64, fn64.size()));
        }
        CK(cudaMemcpy(c->ja64, Ja.data(), Ja.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->ijac64, ij.data(), ij.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->fnm64, fn64.data(), fn64.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    c->geom.assign(x, x + c->npts * 3);
    c->curv_smax = smax;
    if (c->gexec) {  // the captured launches carry the old arguments
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BGK_OK;
}

// Tile-shape autotuner: tiles per task G, per (mesh, degree, velocity grid), cached for the process.
static std::vector<std::pair<std::string, int>> g_tuned;

// Task lengths the autotuners try for chunks of at most maxc tiles: the powers of two from kMinTuneG to
// 64, and the lengths that split the longest chunk into k equal tasks (no short last task per element).
static std::vector<int> task_length_candidates(int maxc)
{
    std::vector<int> cands;
    for (int G = kMinTuneG; G <= 64 && G <= std::max(kMinTuneG, maxc); G *= 2)
        cands.push_back(G);
    for (int k : {1, 2, 3, 4, 6, 8, 12, 16}) {
        const int G = (maxc + k - 1) / k;
        if (G >= kMinTuneG && G <= 64)
            cands.push_back(G);
    }
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    return cands;
}

static void set_task_length(bgk_ctx *c, int G)
{
    c->G = G;
    c->ngroups = 0;
    for (auto &ch : c->chunks) {
        ch.group0 = c->ngroups;
        ch.ngroups = (ch.nvt + G - 1) / G;
        c->ngroups += ch.ngroups;
    }
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
}

int bgk_autotune(bgk_ctx *c, int *g_out)
{
    if (!c)
        return BGK_EINVAL;
    if (c->prec == BGK_FP64) {  // the plain form has no task shape
        if (g_out)
            *g_out = 0;
        return BGK_OK;
    }
    char key[256];
    snprintf(key, sizeof key, "%d/%d/%d,%d,%d/%d,%d,%d/%zu/%d", c->dim, c->p, c->nv[0], c->nv[1], c->nv[2], c->ne[0],
             c->ne[1], c->ne[2], c->chunks.size(),
             (int)(c->has_wall || c->has_force || c->bc[0] || c->bc[2] || c->bc[4]) + 2 * (c->met != nullptr) +
                 4 * (c->ftab != nullptr));
    for (auto &kv : g_tuned)
        if (kv.first == key) {
            set_task_length(c, kv.second);
            if (g_out)
                *g_out = c->G;
            return BGK_OK;
        }
    int maxc = 0;
    for (auto &ch : c->chunks)
        maxc = std::max(maxc, ch.nvt);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestG = c->G;
    const int C = (int)c->chunks.size();
    for (int G : task_length_candidates(maxc)) {
        set_task_length(c, G);
        float tot = 0.f;
        for (int rep = 0; rep < 3; rep++) {
            CK(cudaEventRecord(e0, c->stream));
            // stage 2 of every chunk: reads the first pool slots and f^n, writes the second slots
            for (int q = 0; q < C; q++) {
                const Chunk &ch = c->chunks[q];
                StageArgs A = stage_args(c, ch);
                A.src = c->pool + (int64_t)q * c->chunk_floats;
                A.fn = chunk_ptr(c, c->fA, ch.vt0);
                A.dst = c->pool + (int64_t)(q == 0 ? C : q - 1) * c->chunk_floats;
                stage_coeffs(A, 1, 0.1 * c->tau, c->tau);
                if (q == 0 && C > 1)
                    A.dst = c->pool + (int64_t)C * c->chunk_floats;
                CK(launch_stage(A, c->p, 0, ch.oct, c->stream));
            }
            CK(cudaEventRecord(e1, c->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0)
                tot += ms;
        }
        if (tot < best) {
            best = tot;
            bestG = G;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_task_length(c, bestG);
    g_tuned.emplace_back(key, bestG);
    if (g_out)
        *g_out = bestG;
    return BGK_OK;
}

int bgk_set_timing(bgk_ctx *c, int on)
{
    if (!c)
        return BGK_EINVAL;
    c->timing = on != 0;
    c->nev = 0;
    return BGK_OK;
}

int bgk_timing(bgk_ctx *c, double *stage_ms, int64_t *stage_launches, double *newton_ms, int64_t *newton_launches,
               double *stage_alg_bytes)
{
    if (!c)
        return BGK_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    double sm = 0, nm = 0, by = 0;
    int64_t sl = 0, nl = 0;
    for (size_t q = 0; q < c->nev; q++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->evs[q].a, c->evs[q].b));
        if (c->evs[q].kind == 0) {
            sm += ms;
            sl++;
            by += c->evs[q].bytes;
        } else {
            nm += ms;
            nl++;
        }
    }
    if (stage_ms)
        *stage_ms = sm;
    if (stage_launches)
        *stage_launches = sl;
    if (newton_ms)
        *newton_ms = nm;
    if (newton_launches)
        *newton_launches = nl;
    if (stage_alg_bytes)
        *stage_alg_bytes = sl ? by / sl : 0.0;
    return BGK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------
// Batches of independent line-element problems: per RK stage one persistent stage launch per degree
// present and one Newton launch over all members, the whole step captured in one CUDA graph.

struct bgk_batch {
    int n = 0;
    std::vector<bgk_ctx *> probs;
    StageArgs *d_args = nullptr;    // [3][n] stage arguments of every member
    NewtonArgs *d_nargs = nullptr;  // [n]
    int2 *d_task_member = nullptr;  // [total_tasks] (member, its task index) of every stage task
    int task_cap = 0;               // capacity of d_task_member
    int *d_pt_start = nullptr;      // [n + 1] point prefix sums
    int *d_counter = nullptr;       // [kMaxN1 + 1][4] per degree: work counter, first task, end (persistent launches)
    int *err = nullptr;             // status word shared by the members' Newton solves
    int total_tasks = 0, total_pts = 0;
    int ctas[kMaxN1 + 1] = {0};     // CTAs of each degree's launch, 0 where the batch has no member of that degree
    std::vector<double> dt;         // time step of every member in the device arguments
    std::vector<int> G;             // task length of every member in the device arguments
    double alg_bytes[3] = {0, 0, 0};
    cudaStream_t stream = nullptr, own = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string last;
    int sticky = 0;
    bool timing = false;
    std::vector<bgk_ctx::Ev> evs;
    size_t nev = 0;
};

namespace {

int bfail(bgk_batch *b, int code, const std::string &msg)
{
    b->last = msg;
    return code;
}

#define BK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return bfail(b, BGK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Build and upload the members' stage and Newton arguments for time steps dt (one chunk per member:
// stage 1 A -> slot 0, stage 2 slot 0 (+ A) -> slot 1, stage 3 slot 1 (+ A) -> A in place).
int batch_upload(bgk_batch *b, const double *dt)
{
    const int n = b->n;
    std::vector<StageArgs> sa(3 * (size_t)n);
    std::vector<NewtonArgs> na(n);
    std::vector<int> ts(n + 1, 0), ps(n + 1, 0);
    for (int s = 0; s < 3; s++)
        b->alg_bytes[s] = 0.0;
    for (int q = 0; q < n; q++) {
        bgk_ctx *c = b->probs[q];
        const Chunk &ch = c->chunks[0];
        float *Aq = c->fA, *s1 = c->pool, *s2 = c->pool + c->chunk_floats;
        int64_t real = 0;
        for (int v = 0; v < c->nslots; v++)
            real += c->slotk[v] >= 0;
        for (int st = 0; st < 3; st++) {
            StageArgs A = stage_args(c, ch);
            A.src = st == 0 ? Aq : (st == 1 ? s1 : s2);
            A.fn = st == 0 ? nullptr : Aq;
            A.dst = st == 0 ? s1 : (st == 1 ? s2 : Aq);
            stage_coeffs(A, st, dt[q], c->tau);
            sa[(size_t)st * n + q] = A;
            b->alg_bytes[st] += (double)real * c->npts * sizeof(float) * (st == 0 ? 2 : 3);
        }
        NewtonArgs N = newton_args(c, 0);
        N.err = b->err;
        na[q] = N;
        const int64_t t = ts[q] + (int64_t)stage1d_tasks(sa[q]);
        const int64_t pt = ps[q] + c->npts;
        if (t > INT32_MAX / 2 || pt > INT32_MAX / 2)
            return bfail(b, BGK_EINVAL, "batch too large");
        ts[q + 1] = (int)t;
        ps[q + 1] = (int)pt;
        b->dt[q] = dt[q];
        b->G[q] = c->G;
    }
    b->total_tasks = ts[n];
    b->total_pts = ps[n];
    // the task table degree by degree: one persistent launch per degree takes its range
    std::vector<int2> tm;
    tm.reserve((size_t)ts[n]);
    std::vector<int> block(4 * (kMaxN1 + 1), 0);
    for (int n1 = 0; n1 <= kMaxN1; n1++) {
        block[4 * n1 + 1] = (int)tm.size();
        for (int q = 0; q < n; q++)
            if (b->probs[q]->N1 == n1)
                for (int k = 0; k < ts[q + 1] - ts[q]; k++)
                    tm.push_back(make_int2(q, k));
        block[4 * n1 + 2] = (int)tm.size();
    }
    if (ts[n] > b->task_cap) {  // a larger table: the captured step graph holds the old one's address
        BK(cudaStreamSynchronize(b->stream));
        if (b->d_task_member)
            BK(cudaFree(b->d_task_member));
        b->d_task_member = nullptr;
        b->task_cap = 0;
        BK(cudaMalloc((void **)&b->d_task_member, (size_t)ts[n] * sizeof(int2)));
        b->task_cap = ts[n];
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
    }
    BK(cudaMemcpyAsync(b->d_args, sa.data(), sa.size() * sizeof(StageArgs), cudaMemcpyHostToDevice, b->stream));
    BK(cudaMemcpyAsync(b->d_nargs, na.data(), na.size() * sizeof(NewtonArgs), cudaMemcpyHostToDevice, b->stream));
    BK(cudaMemcpyAsync(b->d_task_member, tm.data(), tm.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    BK(cudaMemcpyAsync(b->d_counter, block.data(), block.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BK(cudaMemcpyAsync(b->d_pt_start, ps.data(), ps.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
    return BGK_OK;
}

void bev_begin(bgk_batch *b, int kind, double bytes)
{
    if (!b->timing)
        return;
    if (b->nev == b->evs.size()) {
        bgk_ctx::Ev ev{};
        cudaEventCreate(&ev.a);
        cudaEventCreate(&ev.b);
        b->evs.push_back(ev);
    }
    b->evs[b->nev].kind = kind;
    b->evs[b->nev].bytes = bytes;
    cudaEventRecord(b->evs[b->nev].a, b->stream);
}

void bev_end(bgk_batch *b)
{
    if (!b->timing)
        return;
    cudaEventRecord(b->evs[b->nev].b, b->stream);
    b->nev++;
}

// One SSP-RK3 step of every member: per stage one persistent stage launch per degree and one Newton
// launch.
int batch_enqueue(bgk_batch *b, cudaStream_t s)
{
    for (int st = 0; st < 3; st++) {
        bev_begin(b, 0, b->alg_bytes[st]);
        for (int n1 = 0; n1 <= kMaxN1; n1++)
            if (b->ctas[n1])
                BK(launch_stage1d_batch(n1, b->d_args + (size_t)st * b->n, b->d_task_member, b->d_counter + 4 * n1,
                                        b->ctas[n1], s));
        bev_end(b);
        bev_begin(b, 1, 0.0);
        BK(launch_newton_batch(b->d_nargs, b->d_pt_start, b->n, b->total_pts, s));
        bev_end(b);
    }
    return BGK_OK;
}

int batch_status(bgk_batch *b)
{
    int e = 0;
    BK(cudaStreamSynchronize(b->stream));
    BK(cudaMemcpy(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e)
        for (bgk_ctx *c : b->probs)
            c->sticky |= e;  // the members' states are no longer valid either
    b->sticky |= e;
    if (b->sticky & kErrDomain)
        return bfail(b, BGK_EDOMAIN, "non-physical state (rho <= 0, theta <= 0 or NaN) met on the device");
    if (b->sticky & kErrNewton)
        return bfail(b, BGK_ENEWTON, "conservative-Maxwellian Newton solve did not converge at some point");
    return BGK_OK;
}

}  // namespace

extern "C" {

const char *bgk_batch_last_error(const bgk_batch *b) { return b ? b->last.c_str() : "null batch"; }

void bgk_batch_destroy(bgk_batch *b)
{
    if (!b)
        return;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    for (auto &ev : b->evs) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    if (b->ev)
        cudaEventDestroy(b->ev);
    void *bufs[] = {b->d_args, b->d_nargs, b->d_task_member, b->d_pt_start, b->d_counter, b->err};
    for (void *p : bufs)
        if (p)
            cudaFree(p);
    if (b->own)
        cudaStreamDestroy(b->own);
    delete b;
}

int bgk_batch_create(int n, bgk_ctx *const *probs, bgk_batch **out)
{
    if (!out)
        return BGK_EINVAL;
    *out = nullptr;
    if (n < 1 || !probs)
        return BGK_EINVAL;
    bgk_batch *b = new bgk_batch();
    auto bail = [&](int code, const std::string &msg) {
        fprintf(stderr, "bgk_batch_create: %s\n", msg.c_str());
        bgk_batch_destroy(b);
        return code;
    };
    std::vector<const bgk_ctx *> seen;
    for (int q = 0; q < n; q++) {
        bgk_ctx *c = probs[q];
        if (!c)
            return bail(BGK_EINVAL, "null member");
        if (c->prec != BGK_FP32_SPLIT || c->dim != 1 || c->p > 3)
            return bail(BGK_EINVAL, "members must be FP32-split line problems (dim = 1) with p <= 3");
        if (c->chunks.size() != 1)
            return bail(BGK_EINVAL, "members must be created with opts.chunks = 1");
        if (c->sticky)
            return bail(BGK_EINVAL, "a member holds a device error");
        seen.push_back(c);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return bail(BGK_EINVAL, "a context appears twice");
    b->n = n;
    b->probs.assign(probs, probs + n);
    b->dt.assign(n, -1.0);
    b->G.assign(n, 0);
    cudaError_t e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->d_args, 3 * (size_t)n * sizeof(StageArgs));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->d_nargs, (size_t)n * sizeof(NewtonArgs));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->d_pt_start, (size_t)(n + 1) * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->d_counter, 4 * (kMaxN1 + 1) * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(b->err, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();  // the memset on the legacy stream, before any non-blocking stream's work
    // the line operators of every degree present, for the constant table of the persistent launches
    bool done[kMaxN1 + 1] = {false};
    for (int q = 0; q < n && e == cudaSuccess; q++) {
        const bgk_ctx *c = probs[q];
        if (!done[c->N1])
            e = set_batch_ops(c->N1, c->ops);
        done[c->N1] = true;
    }
    if (e != cudaSuccess)
        return bail(e == cudaErrorMemoryAllocation ? BGK_ENOMEM : BGK_ECUDA, cudaGetErrorString(e));
    b->stream = b->own;
    for (int n1 = 0; n1 <= kMaxN1; n1++)  // one persistent launch per degree present
        b->ctas[n1] = done[n1] ? stage1d_batch_ctas(n1) : 0;
    *out = b;
    return BGK_OK;
}

int bgk_batch_set_stream(bgk_batch *b, void *stream)
{
    if (!b)
        return BGK_EINVAL;
    b->stream = stream ? (cudaStream_t)stream : b->own;
    return BGK_OK;
}

int bgk_batch_step(bgk_batch *b, const double *dt, int nsteps)
{
    if (!b || !dt || nsteps < 0)
        return BGK_EINVAL;
    for (int q = 0; q < b->n; q++)
        if (!(dt[q] > 0.0) || !std::isfinite(dt[q]))
            return bfail(b, BGK_EINVAL, "every time step must be positive and finite");
    if (b->sticky)
        return batch_status(b);
    for (bgk_ctx *c : b->probs)
        if (c->sticky)
            return bfail(b, BGK_EINVAL, "a member holds a device error");
    if (nsteps == 0)
        return BGK_OK;
    // the members' pending work (state set-up) comes first
    for (bgk_ctx *c : b->probs) {
        BK(cudaEventRecord(b->ev, c->stream));
        BK(cudaStreamWaitEvent(b->stream, b->ev, 0));
    }
    bool stale = false;
    for (int q = 0; q < b->n; q++)
        stale = stale || b->dt[q] != dt[q] || b->G[q] != b->probs[q]->G;
    if (stale) {
        int rc = batch_upload(b, dt);
        if (rc)
            return rc;
    }
    if (b->timing) {
        for (int k = 0; k < nsteps; k++) {
            int rc = batch_enqueue(b, b->stream);
            if (rc)
                return rc;
        }
    } else {
        if (!b->gexec) {  // the graph reads the device argument tables, so new time steps need no capture
            cudaStream_t cap;
            BK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaStreamDestroy(cap);
                BK(e);
            }
            int rc = batch_enqueue(b, cap);
            e = cudaStreamEndCapture(cap, &g);
            cudaStreamDestroy(cap);
            if (rc)
                return rc;
            BK(e);
            e = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            BK(e);
        }
        for (int k = 0; k < nsteps; k++)
            BK(cudaGraphLaunch(b->gexec, b->stream));
    }
    // the members' later work (moments, their own steps) follows the batch
    BK(cudaEventRecord(b->ev, b->stream));
    for (bgk_ctx *c : b->probs)
        BK(cudaStreamWaitEvent(c->stream, b->ev, 0));
    return BGK_OK;
}

int bgk_batch_synchronize(bgk_batch *b)
{
    if (!b)
        return BGK_EINVAL;
    return batch_status(b);
}

int bgk_batch_autotune(bgk_batch *b)
{
    if (!b)
        return BGK_EINVAL;
    std::vector<double> dt(b->dt);
    for (int q = 0; q < b->n; q++)
        if (!(dt[q] > 0.0))
            dt[q] = 0.1 * b->probs[q]->tau;  // any step: the timed stage's values are discarded
    // classes of members with the same (degree, velocity grid)
    std::vector<int> cls(b->n, -1);
    std::vector<int> rep;
    for (int q = 0; q < b->n; q++) {
        const bgk_ctx *c = b->probs[q];
        for (size_t k = 0; k < rep.size() && cls[q] < 0; k++) {
            const bgk_ctx *r = b->probs[rep[k]];
            if (r->p == c->p && r->nv[0] == c->nv[0] && r->nv[1] == c->nv[1] && r->nv[2] == c->nv[2])
                cls[q] = (int)k;
        }
        if (cls[q] < 0) {
            cls[q] = (int)rep.size();
            rep.push_back(q);
        }
    }
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    auto timed = [&](float &ms_out) -> int {
        int rc = batch_upload(b, dt.data());
        if (rc)
            return rc;
        float tot = 0.f;
        for (int r = 0; r < 3; r++) {
            // stage 2: reads slot 0 and f^n, writes slot 1 (f^n, the moments and equilibrium untouched)
            BK(cudaEventRecord(e0, b->stream));
            for (int n1 = 0; n1 <= kMaxN1; n1++)
                if (b->ctas[n1])
                    BK(launch_stage1d_batch(n1, b->d_args + b->n, b->d_task_member, b->d_counter + 4 * n1, b->ctas[n1],
                                            b->stream));
            BK(cudaEventRecord(e1, b->stream));
            BK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BK(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0)
                tot += ms;
        }
        ms_out = tot;
        return BGK_OK;
    };
    for (bgk_ctx *c : b->probs) {
        BK(cudaEventRecord(b->ev, c->stream));
        BK(cudaStreamWaitEvent(b->stream, b->ev, 0));
    }
    for (size_t k = 0; k < rep.size(); k++) {
        float best = 1e30f;
        int bestG = b->probs[rep[k]]->G;
        int maxc = 0;  // the class's longest chunk (members with the same degree and velocity grid)
        for (const Chunk &ch : b->probs[rep[k]]->chunks)
            maxc = std::max(maxc, ch.nvt);
        for (int G : task_length_candidates(maxc)) {
            for (int q = 0; q < b->n; q++)
                if (cls[q] == (int)k)
                    set_task_length(b->probs[q], G);
            float ms = 0.f;
            int rc = timed(ms);
            if (rc)
                return rc;
            if (ms < best) {
                best = ms;
                bestG = G;
            }
        }
        for (int q = 0; q < b->n; q++)
            if (cls[q] == (int)k)
                set_task_length(b->probs[q], bestG);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::fill(b->G.begin(), b->G.end(), 0);  // re-upload with the chosen lengths on the next step
    return BGK_OK;
}

int bgk_batch_info(const bgk_batch *b, int64_t *npoints, int64_t *ndof, int64_t *tasks)
{
    if (!b)
        return BGK_EINVAL;
    int64_t np = 0, nd = 0, nt = 0;
    for (const bgk_ctx *c : b->probs) {
        np += c->npts;
        nd += c->npts * c->nvel;
        nt += stage1d_tasks(stage_args(const_cast<bgk_ctx *>(c), c->chunks[0]));
    }
    if (npoints)
        *npoints = np;
    if (ndof)
        *ndof = nd;
    if (tasks)
        *tasks = nt;
    return BGK_OK;
}

int bgk_batch_set_timing(bgk_batch *b, int on)
{
    if (!b)
        return BGK_EINVAL;
    b->timing = on != 0;
    b->nev = 0;
    return BGK_OK;
}

int bgk_batch_timing(bgk_batch *b, double *stage_ms, int64_t *stage_launches, double *newton_ms,
                     int64_t *newton_launches, double *stage_alg_bytes)
{
    if (!b)
        return BGK_EINVAL;
    BK(cudaStreamSynchronize(b->stream));
    double sm = 0, nm = 0, by = 0;
    int64_t sl = 0, nl = 0;
    for (size_t q = 0; q < b->nev; q++) {
        float ms = 0.f;
        BK(cudaEventElapsedTime(&ms, b->evs[q].a, b->evs[q].b));
        if (b->evs[q].kind == 0) {
            sm += ms;
            sl++;
            by += b->evs[q].bytes;
        } else {
            nm += ms;
            nl++;
        }
    }
    if (stage_ms)
        *stage_ms = sm;
    if (stage_launches)
        *stage_launches = sl;
    if (newton_ms)
        *newton_ms = nm;
    if (newton_launches)
        *newton_launches = nl;
    if (stage_alg_bytes)
        *stage_alg_bytes = sl ? by / sl : 0.0;
    return BGK_OK;
}

}  // extern "C"
