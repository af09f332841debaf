/*
 * bgk_oracle.c -- FP64 CPU oracle for one explicit SSP-RK3 step of the Boltzmann-BGK equation
 * (Dzanic & Martinelli, Sec. 2). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it to check and time the CUDA library; the library never
 * calls it. Everything is plain FP64 loops in the order the paper states the method, with no
 * blocking, fusion or reordering. OpenMP only splits the outer loop over elements or points.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous on each):
 *   - The Maxwellian normalisation uses the velocity dimension m (Eq. 4 writes d/2): m = 3, or m = 2
 *     when the third velocity axis has a single node (the two-dimensional velocity space of the
 *     paper's planar cases, Sec. 2, m >= d).
 *   - Monatomic gas, P = rho*theta and E = rho|U|^2/2 + (m/2) rho theta (Eq. 4); for m = 2 the third
 *     momentum component is identically zero and the Newton unknown U'z is left out.
 *   - Velocity grid nodes include both endpoints; trapezoid weights; tensor product (Eq. 12).
 *   - Correction functions: left/right Radau polynomials (Huynh's g_DG), which recover nodal DG.
 *   - Interface flux points are the tensor Gauss-Legendre points of each face.
 *   - Upwind tie u_n = 0 gives zero flux either way (Eq. 9).
 *   - Conservative Maxwellian: Newton on (rho', U', theta') from the continuous state of Q,
 *     scaled max-norm residual (mass / rho, momentum / (rho sqrt(theta)), energy / E).
 *   - Boundaries (the paper gives none for this path): Dirichlet ghost = sampled continuous
 *     Maxwellian of the prescribed state; diffuse wall ghost = rho_w * M(T_w, U_w) with rho_w
 *     chosen per face point for zero net discrete mass flux.
 *   - Body force: source g * (beta . psi) with (sum_k w g psi psi^T) beta = (0, rho F, rho U.F),
 *     whose discrete moments are exactly those of -F . grad_xi f.
 *   - Curvilinear hexahedra (optional, oracle_set_geometry): each element maps the reference cube by the
 *     degree-p interpolant of its solution-node coordinates; the advection is the FR residual of the
 *     reference-space flux (Ja^i . xi) f divided by J, with the metric terms Ja^i in Kopriva's
 *     conservative curl form (which satisfies the discrete metric identities, so a constant state is
 *     preserved) and a single-valued face normal (the mean of the two elements' interpolated Ja^i at
 *     the face) in the upwind flux (Eq. 9 with u_n = Ja^i . xi). The limiter's element mean is then
 *     J-weighted.
 */
#include "bgk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define MAXN 16

struct orc_ctx {
    int dim, p, n1, np;     /* n1 = p + 1 nodes per direction, np = n1^dim nodes per element */
    int ne[3];
    double lo[3], hi[3], h[3];
    int64_t nelem, npts;
    int bc[6];
    double bcs[30];
    int nv[3];
    int vdim;               /* velocity dimension m: 3, or 2 when nv[2] == 1 (no u_z) */
    int64_t nvel;
    double *xi;             /* [nvel][3] */
    double *w;              /* [nvel] */
    double tau;
    int collide;
    double force[3];
    int has_force;
    double xg[MAXN], wg[MAXN], D[MAXN * MAXN], lm[MAXN], lp[MAXN], dgl[MAXN], dgr[MAXN];
    double *f;              /* [npts][nvel] */
    double *ghost;          /* [6][nvel]: Dirichlet ghost Maxwellian, or unit-density wall Maxwellian */
    double *halo[6];        /* exchange faces: the neighbouring subdomain's element layer [nface][np][nvel] */
    double *sf1, *sf2;      /* stage sources of oracle_stage (allocated on first use) */
    double newton_tol;
    int newton_max;
    int continuous;         /* 1: g is the sampled continuous Maxwellian of Q (no Newton; ablation) */
    double mu_ref, mu_omega; /* mu_ref > 0: tau = mu / P per point, mu = mu_ref theta^omega (Sec. 2, Eq. 5) */
    int limiter;            /* 1: Zhang-Shu positivity limiter on every stage output */
    /* curvilinear geometry (NULL: the affine mesh of lo/hi) */
    double *gx;             /* [npts][3] node coordinates */
    double *Ja;             /* [npts][3][3] metric terms Ja^i_n (i: reference direction, n: component) */
    double *Jd;             /* [npts] Jacobian determinant J */
    double *fn;             /* [nelem][3][2][n1^2][3] common contravariant face normals (direction, side) */
    /* unstructured connectivity (NULL: the structured element grid); per element and local face 2d+side */
    int *cn;                /* neighbour element, or -1 - g at a boundary face with the ghost of face g */
    int *cf;                /* the neighbour's local face 2d'+s' */
    int *co;                /* orientation of the neighbour's face points (see oracle_set_connectivity) */
};

/* ------------------------------------------------------------------------------------------ */
/* Reference-element operators (Sec. 2.1, Eqs. 7-8)                                            */
/* ------------------------------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) and its derivative by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre(int n, double x, double *P, double *dP)
{
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (n == 0) {
        *P = 1.0;
        *dP = 0.0;
        return;
    }
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        double d2 = d0 + (2.0 * k + 1.0) * p1;
        p0 = p1;
        p1 = p2;
        d0 = d1;
        d1 = d2;
    }
    *P = p1;
    *dP = d1;
}

int oracle_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || n > MAXN || !x || !w)
        return -1;
    for (int i = 0; i < n; i++) {
        /* roots of P_n by Newton from the usual cosine guess, then w = 2 / ((1 - x^2) P_n'(x)^2) */
        double r = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double P, dP;
            legendre(n, r, &P, &dP);
            double dr = P / dP;
            r -= dr;
            if (fabs(dr) < 1e-16)
                break;
        }
        double P, dP;
        legendre(n, r, &P, &dP);
        x[n - 1 - i] = r;
        w[n - 1 - i] = 2.0 / ((1.0 - r * r) * dP * dP);
    }
    return 0;
}

/* Lagrange basis polynomial l_j of the nodes x[0..n-1], evaluated at y. */
static double lagrange(int n, const double *x, int j, double y)
{
    double v = 1.0;
    for (int k = 0; k < n; k++)
        if (k != j)
            v *= (y - x[k]) / (x[j] - x[k]);
    return v;
}

/* Derivative l_j'(y) by the product rule. */
static double lagrange_deriv(int n, const double *x, int j, double y)
{
    double s = 0.0;
    for (int m = 0; m < n; m++) {
        if (m == j)
            continue;
        double t = 1.0 / (x[j] - x[m]);
        for (int k = 0; k < n; k++)
            if (k != j && k != m)
                t *= (y - x[k]) / (x[j] - x[k]);
        s += t;
    }
    return s;
}

int oracle_fr_operators(int p, double *D, double *lm, double *lp, double *dgl, double *dgr)
{
    int n = p + 1;
    double x[MAXN], w[MAXN];
    if (p < 0 || n > MAXN)
        return -1;
    oracle_gauss_legendre(n, x, w);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            D[i * n + j] = lagrange_deriv(n, x, j, x[i]);
    for (int j = 0; j < n; j++) {
        lm[j] = lagrange(n, x, j, -1.0);
        lp[j] = lagrange(n, x, j, 1.0);
    }
    /* g_L = (-1)^p / 2 (P_p - P_{p+1}) and g_R = (P_p + P_{p+1}) / 2: g_L(-1) = 1, g_L(1) = 0 and
     * mirror for g_R (Huynh's DG-recovering correction functions). */
    double sgn = (p % 2 == 0) ? 1.0 : -1.0;
    for (int i = 0; i < n; i++) {
        double Pp, dPp, Pq, dPq;
        legendre(p, x[i], &Pp, &dPp);
        legendre(p + 1, x[i], &Pq, &dPq);
        dgl[i] = 0.5 * sgn * (dPp - dPq);
        dgr[i] = 0.5 * (dPp + dPq);
    }
    return 0;
}

int oracle_velocity_grid(const int *nv, const double *vlo, const double *vhi, double *xi, double *w)
{
    double x1[3][256], w1[3][256];
    for (int d = 0; d < 3; d++) {
        if (d == 2 && nv[2] == 1) {  /* m = 2: the u_z axis is absent (one node at 0, unit weight) */
            x1[2][0] = 0.0;
            w1[2][0] = 1.0;
            continue;
        }
        if (nv[d] < 2 || nv[d] > 256 || !(vhi[d] > vlo[d]))
            return -1;
        double dx = (vhi[d] - vlo[d]) / (nv[d] - 1);
        for (int k = 0; k < nv[d]; k++) {
            x1[d][k] = vlo[d] + k * dx;
            w1[d][k] = (k == 0 || k == nv[d] - 1) ? 0.5 * dx : dx;
        }
    }
    int64_t k = 0;
    for (int kz = 0; kz < nv[2]; kz++)
        for (int ky = 0; ky < nv[1]; ky++)
            for (int kx = 0; kx < nv[0]; kx++, k++) {
                xi[3 * k + 0] = x1[0][kx];
                xi[3 * k + 1] = x1[1][ky];
                xi[3 * k + 2] = x1[2][kz];
                w[k] = w1[0][kx] * w1[1][ky] * w1[2][kz];
            }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Maxwellian and moments (Sec. 2, Eqs. 2 and 4; Sec. 2.1, Eq. 12)                            */
/* ------------------------------------------------------------------------------------------ */

/* Continuous Maxwellian at velocity v for (rho, U, theta) in velocity dimension m (Eq. 4); for
 * m = 2 the third components of U and v take no part. */
static double maxwellian(int m, double rho, const double *U, double theta, const double *v)
{
    double r2 = 0.0;
    for (int d = 0; d < m; d++)
        r2 += (v[d] - U[d]) * (v[d] - U[d]);
    return rho / pow(2.0 * ORC_PI * theta, 0.5 * m) * exp(-r2 / (2.0 * theta));
}

/* theta of the moments Q in velocity dimension m: E = rho |U|^2 / 2 + (m / 2) rho theta. */
static double theta_of(int m, const double *Q)
{
    const double rho = Q[0];
    return (2.0 / m) * (Q[4] / rho - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]) / (rho * rho));
}

static void psi_of(const double *v, double *psi)
{
    psi[0] = 1.0;
    psi[1] = v[0];
    psi[2] = v[1];
    psi[3] = v[2];
    psi[4] = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

/* Q = sum_k w_k psi(xi_k) f_k for one point. */
static void moments_point(const orc_ctx *c, const double *fp, double *Q)
{
    for (int m = 0; m < 5; m++)
        Q[m] = 0.0;
    for (int64_t k = 0; k < c->nvel; k++) {
        double psi[5];
        psi_of(c->xi + 3 * k, psi);
        for (int m = 0; m < 5; m++)
            Q[m] += c->w[k] * psi[m] * fp[k];
    }
}

int oracle_moments_of(const orc_ctx *c, const double *f, double *Q)
{
    if (!c || !f || !Q)
        return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->npts; i++)
        moments_point(c, f + i * c->nvel, Q + 5 * i);
    return 0;
}

int oracle_moments(const orc_ctx *c, double *Q) { return oracle_moments_of(c, c->f, Q); }

int oracle_sample_maxwellian(const orc_ctx *c, const double *prim, double *g)
{
    if (!c || !prim || !g || !(prim[0] > 0) || !(prim[4] > 0))
        return -1;
    for (int64_t k = 0; k < c->nvel; k++)
        g[k] = maxwellian(c->vdim, prim[0], prim + 1, prim[4], c->xi + 3 * k);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Discretely-conservative Maxwellian (Sec. 2.1, text after Eq. 13)                            */
/* ------------------------------------------------------------------------------------------ */

/* Solve A x = b (n x n, row-major, copied) by Gaussian elimination with partial pivoting. */
static int solve_dense(int n, const double *A_in, const double *b_in, double *x)
{
    double A[25], b[5];
    memcpy(A, A_in, sizeof(double) * n * n);
    memcpy(b, b_in, sizeof(double) * n);
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col]))
                piv = r;
        if (A[piv * n + col] == 0.0 || !isfinite(A[piv * n + col]))
            return -1;
        if (piv != col) {
            for (int k = 0; k < n; k++) {
                double t = A[col * n + k];
                A[col * n + k] = A[piv * n + k];
                A[piv * n + k] = t;
            }
            double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < n; r++) {
            double m = A[r * n + col] / A[col * n + col];
            for (int k = col; k < n; k++)
                A[r * n + k] -= m * A[col * n + k];
            b[r] -= m * b[col];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++)
            s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
    return 0;
}

/* Solve the n x n system restricted to the unknowns of velocity dimension m (m = 2 leaves out the
 * third momentum component, whose row and column vanish); x of a left-out unknown is 0. */
static int solve_active(int m, const double *A, const double *b, double *x)
{
    if (m == 3)
        return solve_dense(5, A, b, x);
    static const int act[4] = {0, 1, 2, 4};
    double As[16], bs[4], xs[4];
    for (int r = 0; r < 4; r++) {
        bs[r] = b[act[r]];
        for (int q = 0; q < 4; q++)
            As[r * 4 + q] = A[act[r] * 5 + act[q]];
    }
    if (solve_dense(4, As, bs, xs) != 0)
        return -1;
    for (int r = 0; r < 5; r++)
        x[r] = 0.0;
    for (int r = 0; r < 4; r++)
        x[act[r]] = xs[r];
    return 0;
}

/* Residual G(P) = sum_k w_k psi_k g_k(P) - Q and, when J is non-NULL, its Jacobian with respect to
 * P = (rho', U'x, U'y, U'z, theta'), written out from the closed-form derivatives of the Maxwellian:
 * dg/drho' = g / rho', dg/dU'_d = g (xi_d - U'_d) / theta', dg/dtheta' = g (|xi - U'|^2 / (2 theta'^2)
 * - m / (2 theta')). */
static void newton_eval(const orc_ctx *c, const double *P, const double *Q, double *G, double *J)
{
    for (int m = 0; m < 5; m++)
        G[m] = -Q[m];
    if (J)
        for (int m = 0; m < 25; m++)
            J[m] = 0.0;
    for (int64_t k = 0; k < c->nvel; k++) {
        const double *v = c->xi + 3 * k;
        double g = maxwellian(c->vdim, P[0], P + 1, P[4], v);
        double psi[5];
        psi_of(v, psi);
        for (int m = 0; m < 5; m++)
            G[m] += c->w[k] * psi[m] * g;
        if (J) {
            double r2 = 0.0, dg[5] = {0, 0, 0, 0, 0};
            for (int d = 0; d < c->vdim; d++)
                r2 += (v[d] - P[1 + d]) * (v[d] - P[1 + d]);
            dg[0] = g / P[0];
            for (int d = 0; d < c->vdim; d++)
                dg[1 + d] = g * (v[d] - P[1 + d]) / P[4];
            dg[4] = g * (r2 / (2.0 * P[4] * P[4]) - 0.5 * c->vdim / P[4]);
            for (int m = 0; m < 5; m++)
                for (int n = 0; n < 5; n++)
                    J[m * 5 + n] += c->w[k] * psi[m] * dg[n];
        }
    }
}

static double scaled_norm(const double *G, const double *s)
{
    double r = 0.0;
    for (int m = 0; m < 5; m++) {
        double a = fabs(G[m]) / s[m];
        if (!(a <= r))
            r = a; /* also propagates NaN */
    }
    return r;
}

/* Newton for one point. Returns 0 when converged, -1 otherwise. */
static int newton_point(const orc_ctx *c, const double *Q, double *P, int *iters, double *resid)
{
    double rho = Q[0];
    double U[3] = {0, 0, 0}, theta = -1.0;
    if (rho > 0) {
        for (int d = 0; d < 3; d++)
            U[d] = Q[1 + d] / rho;
        theta = theta_of(c->vdim, Q);
    }
    P[0] = rho;
    P[1] = U[0];
    P[2] = U[1];
    P[3] = U[2];
    P[4] = theta;
    if (iters)
        *iters = 0;
    if (resid)
        *resid = INFINITY;
    if (!(rho > 0) || !(theta > 0) || !isfinite(rho) || !isfinite(theta))
        return -1;
    if (c->continuous)  /* the state of Q itself: the equilibrium that Sec. 2.1 shows is not conservative */
        return 0;
    double s[5] = {rho, rho * sqrt(theta), rho * sqrt(theta), rho * sqrt(theta), fabs(Q[4])};
    double G[5], J[25];
    newton_eval(c, P, Q, G, J);
    double res = scaled_norm(G, s);
    int it = 0;
    while (!(res <= c->newton_tol) && it < c->newton_max) {
        double rhs[5], dP[5];
        for (int m = 0; m < 5; m++)
            rhs[m] = -G[m];
        if (solve_active(c->vdim, J, rhs, dP) != 0)
            break;
        it++;
        /* full Newton step, halved only while it leaves the admissible set or raises the residual */
        double lam = 1.0, Pt[5], Gt[5], Jt[25], rest = INFINITY;
        int accepted = 0;
        for (int h = 0; h < 40; h++, lam *= 0.5) {
            for (int m = 0; m < 5; m++)
                Pt[m] = P[m] + lam * dP[m];
            if (!(Pt[0] > 0) || !(Pt[4] > 0))
                continue;
            newton_eval(c, Pt, Q, Gt, Jt);
            rest = scaled_norm(Gt, s);
            if (rest < res) {
                accepted = 1;
                break;
            }
        }
        if (!accepted)
            break;
        memcpy(P, Pt, sizeof Pt);
        memcpy(G, Gt, sizeof Gt);
        memcpy(J, Jt, sizeof Jt);
        res = rest;
    }
    if (iters)
        *iters = it;
    if (resid)
        *resid = res;
    /* a stalled line search at the round-off floor still counts as converged */
    return (res <= c->newton_tol || res <= 1e-11) ? 0 : -1;
}

int oracle_conservative_maxwellian(const orc_ctx *c, int64_t n, const double *Q, double *prim_out,
                                   int *iters, double *resid)
{
    if (!c || !Q || !prim_out || n < 0)
        return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (int64_t i = 0; i < n; i++) {
        int it;
        double r;
        if (newton_point(c, Q + 5 * i, prim_out + 5 * i, &it, &r) != 0)
            bad++;
        if (iters)
            iters[i] = it;
        if (resid)
            resid[i] = r;
    }
    return bad;
}

/* ------------------------------------------------------------------------------------------ */
/* Mesh and problem                                                                            */
/* ------------------------------------------------------------------------------------------ */

static int64_t ipow(int b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; i++)
        r *= b;
    return r;
}

/* Elements on a face of direction d (the product of the other two directions' counts) and the index
 * of element ec among them: the other two coordinates, lower direction fastest. */
static int64_t face_count(const orc_ctx *c, int d)
{
    return d == 0 ? (int64_t)c->ne[1] * c->ne[2] : (d == 1 ? (int64_t)c->ne[0] * c->ne[2] : (int64_t)c->ne[0] * c->ne[1]);
}
static int64_t face_index(const orc_ctx *c, const int *ec, int d)
{
    return d == 0 ? ec[1] + (int64_t)c->ne[1] * ec[2] : (d == 1 ? ec[0] + (int64_t)c->ne[0] * ec[2] : ec[0] + (int64_t)c->ne[0] * ec[1]);
}

orc_ctx *oracle_create(int dim, const int *nelem, const double *lo, const double *hi, const int *bc,
                       const double *bc_state, int p, const int *nv, const double *vlo,
                       const double *vhi, double tau, const double *force)
{
    if (dim < 1 || dim > 3 || p < 0 || p + 1 > MAXN || !nelem || !lo || !hi || !nv || !vlo || !vhi)
        return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c)
        return NULL;
    c->dim = dim;
    c->p = p;
    c->n1 = p + 1;
    c->np = (int)ipow(c->n1, dim);
    c->nelem = 1;
    for (int d = 0; d < 3; d++) {
        c->ne[d] = (d < dim) ? nelem[d] : 1;
        c->lo[d] = (d < dim) ? lo[d] : 0.0;
        c->hi[d] = (d < dim) ? hi[d] : 1.0;
        if (c->ne[d] < 1 || !(c->hi[d] > c->lo[d])) {
            free(c);
            return NULL;
        }
        c->h[d] = (c->hi[d] - c->lo[d]) / c->ne[d];
        c->nelem *= c->ne[d];
    }
    c->npts = c->nelem * c->np;
    for (int i = 0; i < 6; i++)
        c->bc[i] = bc ? bc[i] : ORC_PERIODIC;
    for (int i = 0; i < 30; i++)
        c->bcs[i] = bc_state ? bc_state[i] : 0.0;
    for (int d = 0; d < 3; d++)
        c->nv[d] = nv[d];
    c->vdim = nv[2] == 1 ? 2 : 3;
    if (c->vdim < dim) {  /* the velocity space spans at least the physical space (m >= d) */
        free(c);
        return NULL;
    }
    c->nvel = (int64_t)nv[0] * nv[1] * nv[2];
    c->xi = (double *)malloc(sizeof(double) * 3 * c->nvel);
    c->w = (double *)malloc(sizeof(double) * c->nvel);
    c->f = (double *)calloc((size_t)(c->npts * c->nvel), sizeof(double));
    c->ghost = (double *)calloc((size_t)(6 * c->nvel), sizeof(double));
    if (!c->xi || !c->w || !c->f || !c->ghost || oracle_velocity_grid(nv, vlo, vhi, c->xi, c->w) != 0) {
        oracle_destroy(c);
        return NULL;
    }
    c->tau = tau;
    c->collide = (tau > 0.0 && isfinite(tau));
    for (int d = 0; d < 3; d++)
        c->force[d] = force ? force[d] : 0.0;
    c->has_force = force && (force[0] != 0.0 || force[1] != 0.0 || force[2] != 0.0);
    oracle_fr_operators(p, c->D, c->lm, c->lp, c->dgl, c->dgr);
    oracle_gauss_legendre(c->n1, c->xg, c->wg);
    c->newton_tol = 1e-13;
    c->newton_max = 50;
    /* ghost Maxwellians of non-periodic faces */
    for (int fc = 0; fc < 6; fc++) {
        if (fc / 2 >= dim)
            continue;
        const double *s = c->bcs + 5 * fc;
        if (c->bc[fc] == ORC_DIRICHLET || c->bc[fc] == ORC_WALL) {
            double rho = (c->bc[fc] == ORC_DIRICHLET) ? s[0] : 1.0;
            if (!(rho > 0) || !(s[4] > 0)) {
                oracle_destroy(c);
                return NULL;
            }
            for (int64_t k = 0; k < c->nvel; k++)
                c->ghost[fc * c->nvel + k] = maxwellian(c->vdim, rho, s + 1, s[4], c->xi + 3 * k);
        } else if (c->bc[fc] == ORC_EXCHANGE) {
            c->halo[fc] = (double *)calloc((size_t)(face_count(c, fc / 2) * c->np * c->nvel), sizeof(double));
            if (!c->halo[fc]) {
                oracle_destroy(c);
                return NULL;
            }
        } else if (c->bc[fc] != ORC_PERIODIC) {
            oracle_destroy(c);
            return NULL;
        }
    }
    return c;
}

void oracle_destroy(orc_ctx *c)
{
    if (!c)
        return;
    free(c->xi);
    free(c->w);
    free(c->f);
    free(c->ghost);
    free(c->gx);
    free(c->Ja);
    free(c->Jd);
    free(c->fn);
    free(c->cn);
    free(c->cf);
    free(c->co);
    for (int fc = 0; fc < 6; fc++)
        free(c->halo[fc]);
    free(c->sf1);
    free(c->sf2);
    free(c);
}

int64_t oracle_npoints(const orc_ctx *c) { return c ? c->npts : -1; }
int64_t oracle_nvel(const orc_ctx *c) { return c ? c->nvel : -1; }

void oracle_set_newton(orc_ctx *c, double tol, int max_it)
{
    c->newton_tol = tol;
    c->newton_max = max_it;
}

void oracle_set_maxwellian(orc_ctx *c, int continuous) { c->continuous = continuous != 0; }

void oracle_set_limiter(orc_ctx *c, int on) { c->limiter = on != 0; }

void oracle_set_viscosity(orc_ctx *c, double mu_ref, double omega)
{
    c->mu_ref = mu_ref;
    c->mu_omega = omega;
}

/* Zhang-Shu positivity limiter (Sec. 2.1, Eqs. 10-11), per element and velocity: with the element mean
 * fbar = sum_i W_i f_i / sum_i W_i (tensor Gauss-Legendre weights W) and fmin = min_i f_i, every node value
 * becomes fbar + beta (f_i - fbar), beta = min(|fbar / (fbar - fmin)|, 1), when some f_i < 0. On
 * curvilinear elements the mean is over the physical element (weights W_i J_i). */
int oracle_limit(const orc_ctx *c, double *f)
{
    const int n1 = c->n1, np = c->np;
    double W[MAXN * MAXN * MAXN], Wsum = 0.0;
    for (int i = 0; i < np; i++) {
        W[i] = c->wg[i % n1];
        if (c->dim >= 2)
            W[i] *= c->wg[(i / n1) % n1];
        if (c->dim >= 3)
            W[i] *= c->wg[i / (n1 * n1)];
        Wsum += W[i];
    }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < c->nelem; e++)
        for (int64_t k = 0; k < c->nvel; k++) {
            double fbar = 0.0, fmin = INFINITY, wsum = Wsum;
            if (c->Jd) { /* curvilinear: the mean over the physical element, weights W J */
                wsum = 0.0;
                for (int i = 0; i < np; i++)
                    wsum += W[i] * c->Jd[e * np + i];
            }
            for (int i = 0; i < np; i++) {
                const double v = f[(e * np + i) * c->nvel + k];
                fbar += (c->Jd ? W[i] * c->Jd[e * np + i] : W[i]) * v;
                if (v < fmin)
                    fmin = v;
            }
            fbar /= wsum;
            if (!(fmin < 0.0))
                continue;
            double beta = fabs(fbar / (fbar - fmin));
            if (beta > 1.0)
                beta = 1.0;
            for (int i = 0; i < np; i++) {
                double *v = &f[(e * np + i) * c->nvel + k];
                *v = fbar + beta * (*v - fbar);
            }
        }
    return 0;
}

/* element coordinates (ex, ey, ez) <-> index, x fastest */
static void elem_coords(const orc_ctx *c, int64_t e, int *ec)
{
    ec[0] = (int)(e % c->ne[0]);
    ec[1] = (int)((e / c->ne[0]) % c->ne[1]);
    ec[2] = (int)(e / ((int64_t)c->ne[0] * c->ne[1]));
}

static int64_t elem_index(const orc_ctx *c, const int *ec)
{
    return ec[0] + (int64_t)c->ne[0] * (ec[1] + (int64_t)c->ne[1] * ec[2]);
}

/* node (ix, iy, iz) -> index within an element, x fastest (unused directions 0) */
static int node_index(const orc_ctx *c, const int *ic)
{
    int i = 0;
    for (int d = c->dim - 1; d >= 0; d--)
        i = i * c->n1 + ic[d];
    return i;
}

int oracle_points(const orc_ctx *c, double *x)
{
    if (!c || !x)
        return -1;
    if (c->gx) {
        memcpy(x, c->gx, sizeof(double) * 3 * c->npts);
        return 0;
    }
    for (int64_t e = 0; e < c->nelem; e++) {
        int ec[3];
        elem_coords(c, e, ec);
        for (int i = 0; i < c->np; i++) {
            int ic[3] = {0, 0, 0}, t = i;
            for (int d = 0; d < c->dim; d++) {
                ic[d] = t % c->n1;
                t /= c->n1;
            }
            double *xp = x + 3 * (e * c->np + i);
            for (int d = 0; d < 3; d++)
                xp[d] = (d < c->dim) ? c->lo[d] + (ec[d] + 0.5 * (c->xg[ic[d]] + 1.0)) * c->h[d] : 0.0;
        }
    }
    return 0;
}

int oracle_set_state(orc_ctx *c, const double *prim)
{
    if (!c || !prim)
        return -1;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < c->npts; i++) {
        const double *s = prim + 5 * i;
        if (!(s[0] > 0) || !(s[4] > 0)) {
            bad++;
            continue;
        }
        for (int64_t k = 0; k < c->nvel; k++)
            c->f[i * c->nvel + k] = maxwellian(c->vdim, s[0], s + 1, s[4], c->xi + 3 * k);
    }
    return bad ? -2 : 0;
}

int oracle_set_f(orc_ctx *c, const double *f)
{
    if (!c || !f)
        return -1;
    memcpy(c->f, f, sizeof(double) * (size_t)(c->npts * c->nvel));
    return 0;
}

int oracle_get_f(const orc_ctx *c, double *f)
{
    if (!c || !f)
        return -1;
    memcpy(f, c->f, sizeof(double) * (size_t)(c->npts * c->nvel));
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Curvilinear hexahedra: metric terms and face normals                                        */
/* ------------------------------------------------------------------------------------------ */

/* Derivative along reference direction j of a nodal field u of one element, at every node. */
static void ref_deriv(const orc_ctx *c, const double *u, int j, double *du)
{
    for (int i = 0; i < c->np; i++) {
        int ic[3] = {i % c->n1, (i / c->n1) % c->n1, i / (c->n1 * c->n1)};
        double s = 0.0;
        for (int k = 0; k < c->n1; k++) {
            int kc[3] = {ic[0], ic[1], ic[2]};
            kc[j] = k;
            s += c->D[ic[j] * c->n1 + k] * u[node_index(c, kc)];
        }
        du[i] = s;
    }
}

/* Metric terms of one element from its node coordinates X[np][3]: Kopriva's conservative curl form
 * Ja^i_n = -(curl_r V)_i with V_j = X_l dX_m/dr_j, (n, m, l) cyclic, every product interpolated at
 * the nodes and differentiated with D; J = det(dX_n/dr_j). */
static void element_metric(const orc_ctx *c, const double *X, double *Ja, double *J)
{
    const int np = c->np;
    double *Xc = (double *)malloc(sizeof(double) * np * 4), *dX = (double *)malloc(sizeof(double) * 9 * np);
    double *V = Xc + np, *dV = (double *)malloc(sizeof(double) * 9 * np);
    for (int n = 0; n < 3; n++) {
        for (int i = 0; i < np; i++)
            Xc[i] = X[3 * i + n];
        for (int j = 0; j < 3; j++)
            ref_deriv(c, Xc, j, dX + (n * 3 + j) * np); /* dX[n][j] = dX_n / dr_j */
    }
    for (int n = 0; n < 3; n++) {
        const int m = (n + 1) % 3, l = (n + 2) % 3;
        /* V_j = X_l dX_m/dr_j and its derivatives dV[j][k] = d V_j / d r_k */
        for (int j = 0; j < 3; j++) {
            for (int i = 0; i < np; i++)
                V[i] = X[3 * i + l] * dX[(m * 3 + j) * np + i];
            for (int k = 0; k < 3; k++)
                ref_deriv(c, V, k, dV + (j * 3 + k) * np);
        }
        for (int i = 0; i < np; i++) {
            /* curl components: (dV3/dr2 - dV2/dr3, dV1/dr3 - dV3/dr1, dV2/dr1 - dV1/dr2) */
            const double cu[3] = {dV[(2 * 3 + 1) * np + i] - dV[(1 * 3 + 2) * np + i],
                                  dV[(0 * 3 + 2) * np + i] - dV[(2 * 3 + 0) * np + i],
                                  dV[(1 * 3 + 0) * np + i] - dV[(0 * 3 + 1) * np + i]};
            for (int r = 0; r < 3; r++)
                Ja[(i * 3 + r) * 3 + n] = -cu[r];
        }
    }
    for (int i = 0; i < np; i++) {
        double M[3][3];
        for (int n = 0; n < 3; n++)
            for (int j = 0; j < 3; j++)
                M[n][j] = dX[(n * 3 + j) * np + i];
        J[i] = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    }
    free(Xc);
    free(dX);
    free(dV);
}

/* Own element's Ja^d interpolated to face point ln of its face (d, side). */
static void face_metric(const orc_ctx *c, int64_t e, int d, int side, int ln, double *N)
{
    int ic[3] = {0, 0, 0}, t = ln;
    for (int q = 0; q < 3; q++) {
        if (q == d)
            continue;
        ic[q] = t % c->n1;
        t /= c->n1;
    }
    const double *l = side ? c->lp : c->lm;
    N[0] = N[1] = N[2] = 0.0;
    for (int j = 0; j < c->n1; j++) {
        ic[d] = j;
        const double *a = c->Ja + ((e * c->np + node_index(c, ic)) * 3 + d) * 3;
        for (int n = 0; n < 3; n++)
            N[n] += l[j] * a[n];
    }
}

static void face_normals(orc_ctx *c);
static int64_t table_neighbour(const orc_ctx *c, int64_t e, int d, int side, const int *ic, int64_t *nodes, int *sp);

static int has_exchange(const orc_ctx *c)
{
    for (int fc = 0; fc < 6; fc++)
        if (c->bc[fc] == ORC_EXCHANGE)
            return 1;
    return 0;
}

int oracle_set_geometry(orc_ctx *c, const double *x)
{
    if (c && has_exchange(c)) /* exchange faces are on the structured affine mesh only */
        return -1;
    if (!c || !x || c->dim != 3)
        return -1;
    const int nf = c->n1 * c->n1;
    c->gx = (double *)realloc(c->gx, sizeof(double) * 3 * c->npts);
    c->Ja = (double *)realloc(c->Ja, sizeof(double) * 9 * c->npts);
    c->Jd = (double *)realloc(c->Jd, sizeof(double) * c->npts);
    c->fn = (double *)realloc(c->fn, sizeof(double) * (size_t)(c->nelem * 3 * 2 * nf * 3));
    if (!c->gx || !c->Ja || !c->Jd || !c->fn)
        return -1;
    memcpy(c->gx, x, sizeof(double) * 3 * c->npts);
    int bad = 0;
    for (int64_t e = 0; e < c->nelem; e++) {
        element_metric(c, x + 3 * e * c->np, c->Ja + 9 * e * c->np, c->Jd + e * c->np);
        for (int i = 0; i < c->np; i++)
            if (!(c->Jd[e * c->np + i] > 0.0))
                bad++;
    }
    face_normals(c);
    return bad ? -2 : 0;
}

/* Single-valued face normals: the mean of both elements' interpolated Ja^d on interior and periodic
 * faces (with the neighbour's own axis, face point and sign under unstructured connectivity), the
 * element's own on a boundary face. */
static void face_normals(orc_ctx *c)
{
    const int nf = c->n1 * c->n1;
    for (int64_t e = 0; e < c->nelem; e++) {
        int ec[3];
        elem_coords(c, e, ec);
        if (c->cn) {
            for (int d = 0; d < 3; d++)
                for (int side = 0; side < 2; side++)
                    for (int ln = 0; ln < nf; ln++) {
                        int ic[3] = {0, 0, 0}, t = ln;
                        for (int q = 0; q < 3; q++) {
                            if (q == d)
                                continue;
                            ic[q] = t % c->n1;
                            t /= c->n1;
                        }
                        double N[3], Nn[3];
                        face_metric(c, e, d, side, ln, N);
                        int64_t nodes[MAXN];
                        int sp;
                        const int64_t en = table_neighbour(c, e, d, side, ic, nodes, &sp);
                        if (en >= 0) {
                            /* the neighbour's Ja^{d'} interpolated to the shared face point; its +r_{d'}
                             * points the same way as our +r_d when the faces have opposite sides */
                            const int dn = c->cf[e * 6 + 2 * d + side] / 2;
                            const double *l = sp ? c->lp : c->lm, sg = (sp != side) ? 1.0 : -1.0;
                            Nn[0] = Nn[1] = Nn[2] = 0.0;
                            for (int j = 0; j < c->n1; j++)
                                for (int n = 0; n < 3; n++)
                                    Nn[n] += l[j] * c->Ja[(nodes[j] * 3 + dn) * 3 + n];
                            for (int n = 0; n < 3; n++)
                                N[n] = 0.5 * (N[n] + sg * Nn[n]);
                        }
                        memcpy(c->fn + ((((e * 3 + d) * 2 + side) * nf + ln) * 3), N, sizeof N);
                    }
            continue;
        }
        for (int d = 0; d < 3; d++)
            for (int side = 0; side < 2; side++) {
                int nc[3] = {ec[0], ec[1], ec[2]};
                nc[d] += side ? 1 : -1;
                const int outside = nc[d] < 0 || nc[d] >= c->ne[d];
                const int periodic = c->bc[2 * d + side] == ORC_PERIODIC;
                nc[d] = (nc[d] + c->ne[d]) % c->ne[d];
                const int64_t en = elem_index(c, nc);
                for (int ln = 0; ln < nf; ln++) {
                    double N[3], Nn[3];
                    face_metric(c, e, d, side, ln, N);
                    if (!outside || periodic) {
                        face_metric(c, en, d, 1 - side, ln, Nn);
                        for (int n = 0; n < 3; n++)
                            N[n] = 0.5 * (N[n] + Nn[n]);
                    }
                    memcpy(c->fn + ((((e * 3 + d) * 2 + side) * nf + ln) * 3), N, sizeof N);
                }
            }
    }
}

int oracle_set_connectivity(orc_ctx *c, const int *nbr, const int *nface, const int *orient)
{
    if (c && has_exchange(c))
        return -1;
    if (!c || !nbr || !nface || !orient || c->dim != 3)
        return -1;
    for (int64_t q = 0; q < c->nelem * 6; q++) {
        if (nbr[q] >= c->nelem || nbr[q] < -6 || nface[q] < 0 || nface[q] > 5 || orient[q] < 0 || orient[q] > 7)
            return -1;
        if (nbr[q] < 0 && c->bc[-1 - nbr[q]] != ORC_DIRICHLET && c->bc[-1 - nbr[q]] != ORC_WALL)
            return -1;
    }
    const size_t n = sizeof(int) * (size_t)(c->nelem * 6);
    c->cn = (int *)realloc(c->cn, n);
    c->cf = (int *)realloc(c->cf, n);
    c->co = (int *)realloc(c->co, n);
    if (!c->cn || !c->cf || !c->co)
        return -1;
    memcpy(c->cn, nbr, n);
    memcpy(c->cf, nface, n);
    memcpy(c->co, orient, n);
    if (c->Ja)
        face_normals(c);
    return 0;
}

int oracle_metric(const orc_ctx *c, double *Ja, double *J)
{
    if (!c || !c->Ja)
        return -1;
    if (Ja)
        memcpy(Ja, c->Ja, sizeof(double) * 9 * c->npts);
    if (J)
        memcpy(J, c->Jd, sizeof(double) * c->npts);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* FR advection residual with the upwind flux (Sec. 2.1, Eqs. 7-9)                             */
/* ------------------------------------------------------------------------------------------ */

/* Exterior value seen from the face (direction d, side) of the element at ec, for the face point
 * whose node coordinates along the other directions are ic (ic[d] ignored), velocity k.
 * Periodic / interior faces: the neighbour's trace interpolated to the shared face.
 * Dirichlet: the ghost Maxwellian. Wall: rho_w * unit-density wall Maxwellian, rho_w from zero net
 * discrete mass flux through this face point (computed by the caller and passed as rho_w). */
/* Face point of face (d, side) given by the node coordinates ic (ic[d] ignored) as (a, b): the coordinates
 * along the two other axes in increasing order. */
static void face_ab(int d, const int *ic, int *a, int *b)
{
    *a = ic[d == 0 ? 1 : 0];
    *b = ic[d == 2 ? 1 : 2];
}

/* Unstructured connectivity: the neighbour across local face (d, side) of element e and, for the face
 * point ic, the neighbour's nodes along its own normal axis d' (nodes[0..n1-1], from its low end) and
 * the side s' of its shared face. Returns the neighbour element, or -1 - g at a boundary face. */
static int64_t table_neighbour(const orc_ctx *c, int64_t e, int d, int side, const int *ic, int64_t *nodes, int *sp)
{
    const int fc = 2 * d + side;
    const int en = c->cn[e * 6 + fc];
    if (en < 0)
        return en;
    const int fcn = c->cf[e * 6 + fc], o = c->co[e * 6 + fc];
    const int dn = fcn / 2;
    int a, b;
    face_ab(d, ic, &a, &b);
    int an = (o & 1) ? b : a, bn = (o & 1) ? a : b;
    if (o & 2)
        an = c->n1 - 1 - an;
    if (o & 4)
        bn = c->n1 - 1 - bn;
    int jc[3];
    jc[dn == 0 ? 1 : 0] = an;
    jc[dn == 2 ? 1 : 2] = bn;
    for (int j = 0; j < c->n1; j++) {
        jc[dn] = j;
        nodes[j] = (int64_t)en * c->np + node_index(c, jc);
    }
    *sp = fcn & 1;
    return en;
}

static double exterior_value(const orc_ctx *c, const double *f, const int *ec, int d, int side,
                             const int *ic, int64_t k, double rho_w)
{
    if (c->cn) { /* unstructured: the neighbour's trace at its shared face, or the boundary ghost */
        int64_t nodes[MAXN];
        int sp;
        const int64_t en = table_neighbour(c, elem_index(c, ec), d, side, ic, nodes, &sp);
        if (en < 0) /* a boundary face: the ghost of its class, times the wall density on a wall */
            return (c->bc[-1 - en] == ORC_WALL ? rho_w : 1.0) * c->ghost[(-1 - en) * c->nvel + k];
        const double *l = sp ? c->lp : c->lm;
        double t = 0.0;
        for (int j = 0; j < c->n1; j++)
            t += l[j] * f[nodes[j] * c->nvel + k];
        return t;
    }
    int nc[3] = {ec[0], ec[1], ec[2]};
    nc[d] += side ? 1 : -1;
    int fc = 2 * d + side;
    if (nc[d] < 0 || nc[d] >= c->ne[d]) {
        if (c->bc[fc] == ORC_DIRICHLET)
            return c->ghost[fc * c->nvel + k];
        if (c->bc[fc] == ORC_WALL)
            return rho_w * c->ghost[fc * c->nvel + k];
        if (c->bc[fc] == ORC_EXCHANGE) {
            /* the neighbouring subdomain's element across the face, from its halo layer: its trace at
             * the shared face, as for a neighbour inside the mesh */
            const double *l = side ? c->lm : c->lp;
            const double *hl = c->halo[fc] + face_index(c, ec, d) * c->np * c->nvel;
            double t = 0.0;
            int jc[3] = {ic[0], ic[1], ic[2]};
            for (int j = 0; j < c->n1; j++) {
                jc[d] = j;
                t += l[j] * hl[(int64_t)node_index(c, jc) * c->nvel + k];
            }
            return t;
        }
        nc[d] = (nc[d] + c->ne[d]) % c->ne[d];
    }
    int64_t en = elem_index(c, nc);
    /* the neighbour's trace at its face opposite to ours: its +1 end if we look left, -1 if right */
    const double *l = side ? c->lm : c->lp;
    double t = 0.0;
    int jc[3] = {ic[0], ic[1], ic[2]};
    for (int j = 0; j < c->n1; j++) {
        jc[d] = j;
        t += l[j] * f[(en * c->np + node_index(c, jc)) * c->nvel + k];
    }
    return t;
}

/* Interior trace of the element at the face (d, side), face point ic, velocity k. */
static double interior_trace(const orc_ctx *c, const double *f, int64_t e, int d, int side,
                             const int *ic, int64_t k)
{
    const double *l = side ? c->lp : c->lm;
    double t = 0.0;
    int jc[3] = {ic[0], ic[1], ic[2]};
    for (int j = 0; j < c->n1; j++) {
        jc[d] = j;
        t += l[j] * f[(e * c->np + node_index(c, jc)) * c->nvel + k];
    }
    return t;
}

/* Wall density at a face point: sum over outgoing velocities of w |xi_n| f_trace divided by the
 * sum over incoming velocities of w |xi_n| M_w (unit density). Outgoing = leaving the domain. */
static double wall_density(const orc_ctx *c, const double *f, int64_t e, int d, int side, const int *ic)
{
    int fc = 2 * d + side;
    double out = 0.0, in = 0.0;
    for (int64_t k = 0; k < c->nvel; k++) {
        double un = side ? c->xi[3 * k + d] : -c->xi[3 * k + d]; /* xi . n_out */
        if (un > 0)
            out += c->w[k] * un * interior_trace(c, f, e, d, side, ic, k);
        else if (un < 0)
            in += c->w[k] * (-un) * c->ghost[fc * c->nvel + k];
    }
    return out / in;
}

/* Diffuse-wall density at a face point of a curved wall: as wall_density, with the outward unit normal
 * n = +-N / |N| of the face normal N at the point (N points towards +r_d, outward on the high face);
 * fc: the wall's boundary data (its structured face). */
static double wall_density_curved(const orc_ctx *c, const double *f, int64_t e, int d, int side, const int *ic,
                                  const double *N, int fc)
{
    const double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]), sg = side ? 1.0 : -1.0;
    const double n[3] = {sg * N[0] / nn, sg * N[1] / nn, sg * N[2] / nn};
    double out = 0.0, in = 0.0;
    for (int64_t k = 0; k < c->nvel; k++) {
        const double *v = c->xi + 3 * k;
        const double un = n[0] * v[0] + n[1] * v[1] + n[2] * v[2]; /* xi . n_out */
        if (un > 0)
            out += c->w[k] * un * interior_trace(c, f, e, d, side, ic, k);
        else if (un < 0)
            in += c->w[k] * (-un) * c->ghost[fc * c->nvel + k];
    }
    return out / in;
}

/* The residual on curvilinear hexahedra: along every reference line of direction d, the nodal fluxes
 * F_j = (Ja^d . xi) f_j, their derivative D F, and the FR correction with the upwind common flux of the
 * face normal N (Eq. 9 with u_n = N . xi, positive in +r_d); R = -(sum_d dF_d) / J. */
static int residual_curved(const orc_ctx *c, const double *f, double *R)
{
    const int n1 = c->n1, nf = n1 * n1;
    memset(R, 0, sizeof(double) * (size_t)(c->npts * c->nvel));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < c->nelem; e++) {
        int ec[3];
        elem_coords(c, e, ec);
        for (int d = 0; d < 3; d++)
            for (int ln = 0; ln < nf; ln++) {
                int ic[3] = {0, 0, 0}, t = ln;
                for (int q = 0; q < 3; q++) {
                    if (q == d)
                        continue;
                    ic[q] = t % n1;
                    t /= n1;
                }
                int64_t pts[MAXN];
                for (int j = 0; j < n1; j++) {
                    int jc[3] = {ic[0], ic[1], ic[2]};
                    jc[d] = j;
                    pts[j] = e * c->np + node_index(c, jc);
                }
                const double *NL = c->fn + (((e * 3 + d) * 2 + 0) * nf + ln) * 3;
                const double *NR = c->fn + (((e * 3 + d) * 2 + 1) * nf + ln) * 3;
                /* wall densities of the line's two faces, if they are walls */
                double rw[2] = {0.0, 0.0};
                for (int side = 0; side < 2; side++) {
                    int wall, g = 2 * d + side;
                    if (c->cn) { /* a boundary face whose ghost class is a wall */
                        const int en = c->cn[e * 6 + 2 * d + side];
                        g = -1 - en;
                        wall = en < 0 && c->bc[g] == ORC_WALL;
                    } else {
                        const int edge = side ? (ec[d] == c->ne[d] - 1) : (ec[d] == 0);
                        wall = edge && c->bc[g] == ORC_WALL;
                    }
                    if (wall)
                        rw[side] = wall_density_curved(c, f, e, d, side, ic, side ? NR : NL, g);
                }
                for (int64_t k = 0; k < c->nvel; k++) {
                    const double *v = c->xi + 3 * k;
                    double fl[MAXN], F[MAXN], fL = 0.0, fR = 0.0, FL = 0.0, FR = 0.0;
                    for (int j = 0; j < n1; j++) {
                        const double *a = c->Ja + (pts[j] * 3 + d) * 3;
                        fl[j] = f[pts[j] * c->nvel + k];
                        F[j] = (a[0] * v[0] + a[1] * v[1] + a[2] * v[2]) * fl[j];
                        fL += c->lm[j] * fl[j];
                        fR += c->lp[j] * fl[j];
                        FL += c->lm[j] * F[j];
                        FR += c->lp[j] * F[j];
                    }
                    const double uL = NL[0] * v[0] + NL[1] * v[1] + NL[2] * v[2];
                    const double uR = NR[0] * v[0] + NR[1] * v[1] + NR[2] * v[2];
                    const double FIL = uL > 0 ? uL * exterior_value(c, f, ec, d, 0, ic, k, rw[0]) : uL * fL;
                    const double FIR = uR > 0 ? uR * fR : uR * exterior_value(c, f, ec, d, 1, ic, k, rw[1]);
                    for (int i = 0; i < n1; i++) {
                        double dF = 0.0;
                        for (int j = 0; j < n1; j++)
                            dF += c->D[i * n1 + j] * F[j];
                        dF += (FIL - FL) * c->dgl[i] + (FIR - FR) * c->dgr[i];
                        R[pts[i] * c->nvel + k] -= dF / c->Jd[pts[i]];
                    }
                }
            }
    }
    return 0;
}

int oracle_residual(const orc_ctx *c, const double *f, double *R)
{
    if (!c || !f || !R)
        return -1;
    if (c->Ja)
        return residual_curved(c, f, R);
    if (c->cn) /* unstructured connectivity needs the node coordinates */
        return -1;
    const int n1 = c->n1;
    memset(R, 0, sizeof(double) * (size_t)(c->npts * c->nvel));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < c->nelem; e++) {
        int ec[3];
        elem_coords(c, e, ec);
        for (int d = 0; d < c->dim; d++) {
            int nlines = (int)ipow(n1, c->dim - 1);
            for (int ln = 0; ln < nlines; ln++) {
                /* node coordinates of this line along the directions other than d */
                int ic[3] = {0, 0, 0}, t = ln;
                for (int q = 0; q < c->dim; q++) {
                    if (q == d)
                        continue;
                    ic[q] = t % n1;
                    t /= n1;
                }
                int64_t pts[MAXN];
                for (int j = 0; j < n1; j++) {
                    int jc[3] = {ic[0], ic[1], ic[2]};
                    jc[d] = j;
                    pts[j] = e * c->np + node_index(c, jc);
                }
                /* wall densities of the two faces of this line, if they are walls */
                double rw[2] = {0.0, 0.0};
                for (int side = 0; side < 2; side++) {
                    int edge = side ? (ec[d] == c->ne[d] - 1) : (ec[d] == 0);
                    if (edge && c->bc[2 * d + side] == ORC_WALL)
                        rw[side] = wall_density(c, f, e, d, side, ic);
                }
                for (int64_t k = 0; k < c->nvel; k++) {
                    double a = c->xi[3 * k + d];
                    double fl[MAXN];
                    for (int j = 0; j < n1; j++)
                        fl[j] = f[pts[j] * c->nvel + k];
                    double fL = 0.0, fR = 0.0;
                    for (int j = 0; j < n1; j++) {
                        fL += c->lm[j] * fl[j];
                        fR += c->lp[j] * fl[j];
                    }
                    /* upwind common fluxes (Eq. 9) expressed as fluxes in +x_d */
                    double FL, FR;
                    if (a > 0) {
                        FL = a * exterior_value(c, f, ec, d, 0, ic, k, rw[0]);
                        FR = a * fR;
                    } else {
                        FL = a * fL;
                        FR = a * exterior_value(c, f, ec, d, 1, ic, k, rw[1]);
                    }
                    for (int i = 0; i < n1; i++) {
                        double dF = 0.0;
                        for (int j = 0; j < n1; j++)
                            dF += c->D[i * n1 + j] * a * fl[j];
                        dF += (FL - a * fL) * c->dgl[i] + (FR - a * fR) * c->dgr[i];
                        R[pts[i] * c->nvel + k] -= (2.0 / c->h[d]) * dF;
                    }
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* BGK relaxation and SSP-RK3 (Sec. 2, Eq. 3; Sec. 2.2)                                        */
/* ------------------------------------------------------------------------------------------ */

int oracle_rhs(const orc_ctx *c, const double *f, double *L)
{
    if (oracle_residual(c, f, L) != 0)
        return -1;
    if (!c->collide && !c->has_force)
        return 0;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
    for (int64_t i = 0; i < c->npts; i++) {
        const double *fp = f + i * c->nvel;
        double *Lp = L + i * c->nvel;
        double Q[5], P[5];
        moments_point(c, fp, Q);
        if (newton_point(c, Q, P, NULL, NULL) != 0) {
            bad++;
            continue;
        }
        double beta[5] = {0, 0, 0, 0, 0};
        if (c->has_force) {
            /* (sum_k w g psi psi^T) beta = (0, rho F, rho U . F) */
            double A[25] = {0}, b[5];
            for (int64_t k = 0; k < c->nvel; k++) {
                double g = maxwellian(c->vdim, P[0], P + 1, P[4], c->xi + 3 * k), psi[5];
                psi_of(c->xi + 3 * k, psi);
                for (int m = 0; m < 5; m++)
                    for (int n = 0; n < 5; n++)
                        A[m * 5 + n] += c->w[k] * g * psi[m] * psi[n];
            }
            double rho = Q[0];
            b[0] = 0.0;
            for (int d = 0; d < 3; d++)
                b[1 + d] = rho * c->force[d];
            b[4] = Q[1] * c->force[0] + Q[2] * c->force[1] + Q[3] * c->force[2];
            if (solve_active(c->vdim, A, b, beta) != 0) {
                bad++;
                continue;
            }
        }
        /* collision time: the constant tau, or mu(theta) / P of this point's state (P = rho theta) */
        double tau = c->tau;
        if (c->mu_ref > 0.0) {
            const double rho = Q[0];
            const double th = theta_of(c->vdim, Q);
            tau = c->mu_ref * pow(th, c->mu_omega) / (rho * th);
        }
        for (int64_t k = 0; k < c->nvel; k++) {
            double g = maxwellian(c->vdim, P[0], P + 1, P[4], c->xi + 3 * k);
            if (c->collide)
                Lp[k] += (g - fp[k]) / tau;
            if (c->has_force) {
                double psi[5], s = 0.0;
                psi_of(c->xi + 3 * k, psi);
                for (int m = 0; m < 5; m++)
                    s += beta[m] * psi[m];
                Lp[k] += g * s;
            }
        }
    }
    return bad ? -bad : 0;
}

int oracle_step(orc_ctx *c, double dt, int nsteps)
{
    if (!c || nsteps < 0 || !(dt > 0))
        return -1;
    size_t n = (size_t)(c->npts * c->nvel);
    double *f1 = (double *)malloc(sizeof(double) * n);
    double *f2 = (double *)malloc(sizeof(double) * n);
    double *L = (double *)malloc(sizeof(double) * n);
    if (!f1 || !f2 || !L) {
        free(f1);
        free(f2);
        free(L);
        return -1;
    }
    int fails = 0;
    double *f = c->f;
    for (int s = 0; s < nsteps; s++) {
        /* Shu-Osher SSP-RK3 */
        fails += -oracle_rhs(c, f, L);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; q++)
            f1[q] = f[q] + dt * L[q];
        if (c->limiter)
            oracle_limit(c, f1);
        fails += -oracle_rhs(c, f1, L);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; q++)
            f2[q] = 0.75 * f[q] + 0.25 * (f1[q] + dt * L[q]);
        if (c->limiter)
            oracle_limit(c, f2);
        fails += -oracle_rhs(c, f2, L);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; q++)
            f[q] = (1.0 / 3.0) * f[q] + (2.0 / 3.0) * (f2[q] + dt * L[q]);
        if (c->limiter)
            oracle_limit(c, f);
    }
    free(f1);
    free(f2);
    free(L);
    return fails ? -fails : 0;
}

/* One Shu-Osher stage of the SSP-RK3 step of oracle_step, with the same arithmetic: stage 0 forms
 * f1 = f + dt L(f), stage 1 f2 = 3/4 f + 1/4 (f1 + dt L(f1)), stage 2 f = 1/3 f + 2/3 (f2 + dt L(f2)),
 * the limiter after each when it is on. Three calls in order equal one oracle_step; between them the
 * caller may refresh exchange halos from the other subdomains' stage sources (oracle_pack_halo). */
int oracle_stage(orc_ctx *c, double dt, int stage)
{
    if (!c || stage < 0 || stage > 2)
        return -1;
    size_t n = (size_t)(c->npts * c->nvel);
    if (!c->sf1)
        c->sf1 = (double *)malloc(sizeof(double) * n);
    if (!c->sf2)
        c->sf2 = (double *)malloc(sizeof(double) * n);
    double *L = (double *)malloc(sizeof(double) * n);
    if (!c->sf1 || !c->sf2 || !L) {
        free(L);
        return -1;
    }
    double *f = c->f, *f1 = c->sf1, *f2 = c->sf2;
    int fails = 0;
    if (stage == 0) {
        fails += -oracle_rhs(c, f, L);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; q++)
            f1[q] = f[q] + dt * L[q];
        if (c->limiter)
            oracle_limit(c, f1);
    } else if (stage == 1) {
        fails += -oracle_rhs(c, f1, L);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; q++)
            f2[q] = 0.75 * f[q] + 0.25 * (f1[q] + dt * L[q]);
        if (c->limiter)
            oracle_limit(c, f2);
    } else {
        fails += -oracle_rhs(c, f2, L);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; q++)
            f[q] = (1.0 / 3.0) * f[q] + (2.0 / 3.0) * (f2[q] + dt * L[q]);
        if (c->limiter)
            oracle_limit(c, f);
    }
    free(L);
    return fails ? -fails : 0;
}

/* The element layer next to face fc (2 d + side) of the source of stage `stage` (0: f, 1: f1, 2: f2):
 * out[face_index][node][velocity], the data a neighbouring subdomain takes as the halo of its opposite
 * face. */
int oracle_pack_halo(const orc_ctx *c, int fc, int stage, double *out)
{
    if (!c || fc < 0 || fc >= 2 * c->dim || stage < 0 || stage > 2 || !out || (stage > 0 && !(stage == 1 ? c->sf1 : c->sf2)))
        return -1;
    const double *src = stage == 0 ? c->f : (stage == 1 ? c->sf1 : c->sf2);
    const int d = fc / 2, side = fc % 2;
    for (int64_t e = 0; e < c->nelem; e++) {
        int ec[3];
        elem_coords(c, e, ec);
        if (ec[d] != (side ? c->ne[d] - 1 : 0))
            continue;
        memcpy(out + face_index(c, ec, d) * c->np * c->nvel, src + e * c->np * c->nvel,
               sizeof(double) * (size_t)(c->np * c->nvel));
    }
    return 0;
}

/* The halo of exchange face fc: in[face_index][node][velocity] (copied). */
int oracle_set_halo(orc_ctx *c, int fc, const double *in)
{
    if (!c || fc < 0 || fc >= 6 || !c->halo[fc] || !in)
        return -1;
    memcpy(c->halo[fc], in, sizeof(double) * (size_t)(face_count(c, fc / 2) * c->np * c->nvel));
    return 0;
}

double oracle_dt(const orc_ctx *c, double cfl)
{
    double smax = 0.0;
    for (int64_t k = 0; k < c->nvel; k++) {
        double s = 0.0;
        for (int d = 0; d < c->dim; d++)
            s += fabs(c->xi[3 * k + d]) / c->h[d];
        if (s > smax)
            smax = s;
    }
    if (c->Ja) { /* curvilinear: max over nodes of sum_d |Ja^d . xi| / (2 J) (the affine value above) */
        smax = 0.0;
        for (int64_t i = 0; i < c->npts; i++)
            for (int64_t k = 0; k < c->nvel; k++) {
                const double *v = c->xi + 3 * k;
                double s = 0.0;
                for (int d = 0; d < 3; d++) {
                    const double *a = c->Ja + (i * 3 + d) * 3;
                    s += fabs(a[0] * v[0] + a[1] * v[1] + a[2] * v[2]);
                }
                s /= 2.0 * c->Jd[i];
                if (s > smax)
                    smax = s;
            }
    }
    double dt = cfl / smax;
    if (c->collide && c->tau < dt)
        dt = c->tau;
    return dt;
}
