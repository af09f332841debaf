/*
 * bgk_oracle.h -- FP64 CPU oracle for the Boltzmann-BGK hot path of Dzanic & Martinelli,
 * "Towards full molecular gas dynamics simulations of complex flows via the Boltzmann equation".
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, plain reference that the CUDA library is checked
 * against. Only the test suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (paper section / equation):
 *   - Gauss-Legendre solution points, Lagrange derivative matrix, end interpolants and the
 *     DG-recovering (Radau) correction-function derivatives of flux reconstruction (Sec. 2.1, Eqs. 7-8).
 *   - The upwind common interface flux (Sec. 2.1, Eq. 9) and the FR advection residual of every
 *     velocity node on a structured affine line/hex mesh (Sec. 2.1, Eqs. 6-9).
 *   - The uniform velocity grid with trapezoid weights (Sec. 2.1 "Velocity discretization", Eq. 12),
 *     the moments Q = M[f psi] (Sec. 2, Eq. 2; Eq. 12).
 *   - The discretely-conservative Maxwellian: a Maxwellian at a perturbed state (rho', U', theta')
 *     found by Newton's method with a closed-form Jacobian so that its discrete moments equal Q
 *     (Sec. 2.1, the text after Eq. 13).
 *   - The BGK relaxation (g - f)/tau (Sec. 2, Eq. 3) and explicit SSP-RK3 time stepping (Sec. 2.2).
 *   - The Zhang-Shu positivity limiter of every stage output (Sec. 2.1, Eqs. 10-11), a power-law
 *     viscosity giving tau per point (Sec. 2, Eq. 5), and the ablation's continuous Maxwellian of Q
 *     (Sec. 2.1, Eq. 13) in place of the conservative one.
 *   - Boundaries: Dirichlet Maxwellian ghosts, diffuse walls whose density per face point gives zero
 *     net discrete mass flux, and the body-force source projected on the equilibrium.
 *   - Meshes: line, quadrilateral and hexahedral elements (dim = 1, 2, 3); curvilinear hexahedra from
 *     node coordinates (metric terms in Kopriva's conservative curl form, upwinding on the shared face
 *     normal); unstructured hexahedral connectivity (neighbour, shared-face and orientation tables).
 *   - The two-dimensional velocity space (m = 2, a velocity grid with one node on its third axis).
 * Every part is pinned by the CPU tests against what the paper and the mathematics fix (closed forms,
 * invariants, an independent second formulation, brute force on small inputs); the Sod and Mach-5
 * shock structures have no closed form, so beyond agreement with the oracle their physics is parity
 * unpinned.
 *
 * Conventions: all arrays are FP64 and caller-owned. Point order = element-major (element index
 * x-fastest), then node index x-fastest. Velocity order k = kx + nx*(ky + ny*kz). f is [n_x][N_v].
 * Functions return 0 on success and a negative value on bad arguments or failure.
 */
#ifndef BGK_ORACLE_H
#define BGK_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds, one per (direction, side) */
#define ORC_PERIODIC 0
#define ORC_DIRICHLET 1
#define ORC_WALL 2
/* a face shared with a neighbouring subdomain of a partitioned mesh: its exterior values come from a
 * halo, the neighbour's element layer next to the shared face (oracle_set_halo) */
#define ORC_EXCHANGE 3

typedef struct orc_ctx orc_ctx;

/* Gauss-Legendre nodes x[n] and weights w[n] on [-1, 1]. */
int oracle_gauss_legendre(int n, double *x, double *w);

/* FR reference operators for degree p (n = p + 1 nodes):
 *   D[i*n + j] = l_j'(x_i), lm[j] = l_j(-1), lp[j] = l_j(+1),
 *   dgl[i] = g_L'(x_i), dgr[i] = g_R'(x_i) for the left/right Radau correction functions
 *   (Huynh's g_DG, which makes FR identical to nodal DG). */
int oracle_fr_operators(int p, double *D, double *lm, double *lp, double *dgl, double *dgr);

/* Uniform velocity grid, endpoints included, tensor trapezoid weights.
 * nv[3] nodes per axis on [vlo, vhi]; xi is [N_v][3], w is [N_v]. nv[2] = 1 selects the
 * two-dimensional velocity space (m = 2): the third components are 0, the weights are the 2-D ones
 * and vlo[2], vhi[2] are not read. */
int oracle_velocity_grid(const int *nv, const double *vlo, const double *vhi, double *xi, double *w);

/* Create a problem. dim in {1,2,3}; nelem[dim], lo[dim], hi[dim] describe an affine structured mesh.
 * bc[2*d + side] is ORC_PERIODIC / ORC_DIRICHLET / ORC_WALL / ORC_EXCHANGE; bc_state[(2*d+side)*5 + c] holds
 * (rho, u, v, w, T) of a Dirichlet state or (unused, u_w, v_w, w_w, T_w) of a wall.
 * tau <= 0 or tau = +inf switches the collision term off (pure advection).
 * force[3] is a constant body force per unit mass (may be NULL). Returns NULL on error.
 * Velocity dimension m = 3, or m = 2 when nv[2] = 1 (then dim <= 2; E = rho|U|^2/2 + rho theta, the
 * third momentum component is identically 0 and the third velocity component of every state, of
 * bc_state and of force is not used). */
orc_ctx *oracle_create(int dim, const int *nelem, const double *lo, const double *hi,
                       const int *bc, const double *bc_state, int p,
                       const int *nv, const double *vlo, const double *vhi,
                       double tau, const double *force);
void oracle_destroy(orc_ctx *c);

/* Partitioned meshes (spatial domain decomposition; the upwind common flux of Sec. 2.1, Eq. 9, is the
 * only coupling between elements, so a subdomain needs, per RK stage, only its neighbours' element
 * layers next to the shared faces). oracle_stage runs one Shu-Osher stage (0, 1, 2) of the step of
 * oracle_step with the same arithmetic; oracle_pack_halo writes the element layer next to face fc of
 * the source of a stage, out[face element][node][velocity] (face elements: the two other coordinates,
 * the lower direction fastest); oracle_set_halo sets the halo of an ORC_EXCHANGE face (same layout).
 * Exchange faces need the structured affine mesh (no oracle_set_geometry / oracle_set_connectivity). */
int oracle_stage(orc_ctx *c, double dt, int stage);
int oracle_pack_halo(const orc_ctx *c, int fc, int stage, double *out);
int oracle_set_halo(orc_ctx *c, int fc, const double *in);
int64_t oracle_npoints(const orc_ctx *c);
int64_t oracle_nvel(const orc_ctx *c);

/* Node coordinates, [n_x][3] (unused components 0). */
int oracle_points(const orc_ctx *c, double *x);

/* Set f to the sampled continuous Maxwellian of prim [n_x][5] = (rho, u, v, w, T). */
int oracle_set_state(orc_ctx *c, const double *prim);
int oracle_set_f(orc_ctx *c, const double *f);
int oracle_get_f(const orc_ctx *c, double *f);

/* Moments Q [n_x][5] = (rho, rho u, rho v, rho w, E) of the current f (Eq. 2 with Eq. 12). */
int oracle_moments(const orc_ctx *c, double *Q);

/* Moments of an arbitrary f [n_x][N_v]. */
int oracle_moments_of(const orc_ctx *c, const double *f, double *Q);

/* Advection residual R = -xi . grad f of an arbitrary f (FR, upwind flux, boundary ghosts). */
int oracle_residual(const orc_ctx *c, const double *f, double *R);

/* Discretely-conservative Maxwellian for n moment vectors Q[n][5] on this problem's velocity grid.
 * prim_out[n][5] = (rho', U'x, U'y, U'z, theta'); iters[n] and resid[n] (scaled max-norm) may be NULL.
 * Returns the number of points that did not converge (0 on success), negative on bad input. */
int oracle_conservative_maxwellian(const orc_ctx *c, int64_t n, const double *Q, double *prim_out,
                                   int *iters, double *resid);

/* Sample the Maxwellian of prim (rho, U, theta) on the velocity grid: g[N_v]. */
int oracle_sample_maxwellian(const orc_ctx *c, const double *prim, double *g);

/* The right-hand side L(f) = R_adv(f) + (g[f] - f)/tau (+ body-force source) of an arbitrary f. */
int oracle_rhs(const orc_ctx *c, const double *f, double *L);

/* Advance the stored f by nsteps SSP-RK3 steps of size dt. Returns 0, or the negative count of
 * Newton failures met. */
int oracle_step(orc_ctx *c, double dt, int nsteps);

/* Largest stable explicit step: min(cfl / max_k sum_d |xi_kd| / h_d, tau). */
double oracle_dt(const orc_ctx *c, double cfl);

/* Newton tolerance and iteration cap used by the conservative Maxwellian (defaults 1e-13, 50). */
void oracle_set_newton(orc_ctx *c, double tol, int max_it);

/* Equilibrium of the BGK source: 0 (default) the discretely-conservative Maxwellian (Sec. 2.1, text
 * after Eq. 13); 1 the sampled continuous Maxwellian of the moments Q, which Sec. 2.1 (Eq. 13) shows is
 * not conservative on the discrete grid (the ablation of the method). */
void oracle_set_maxwellian(orc_ctx *c, int continuous);

/* Zhang-Shu positivity limiter (Sec. 2.1, Eqs. 10-11) on every RK stage output: off by default. */
void oracle_set_limiter(orc_ctx *c, int on);

/* Variable collision time (Sec. 2, Eq. 5): with mu_ref > 0 every point relaxes with tau = mu / P,
 * mu = mu_ref theta^omega (a power law, reference temperature 1) and P = rho theta of the point's
 * moments; mu_ref <= 0 restores the constant tau given at creation (which must stay > 0). */
void oracle_set_viscosity(orc_ctx *c, double mu_ref, double omega);

/* Curvilinear hexahedra (dim = 3; on a diffuse wall the wall density of every face point is set by
 * zero net mass flux through the curved face's own normal there):
 * x[n_x][3] are the physical coordinates of every
 * solution node (point order as above); each element is the degree-p interpolant of its nodes. The
 * metric terms Ja^i_n (Kopriva's conservative curl form) and J are computed here, the advection
 * becomes the reference-space FR residual of (Ja^i . xi) f over J, with face normals averaged between
 * the two elements of a face, the limiter's mean is J-weighted and oracle_dt uses the metric.
 * Returns 0, -2 if some node has J <= 0, -1 on bad input. */
int oracle_set_geometry(orc_ctx *c, const double *x);

/* Unstructured connectivity (dim = 3): per element e and local face
 * f = 2d + side (d the reference axis, side 0 = the r_d = -1 face), [nelem][6] arrays:
 *   nbr[e][f]    the neighbour element, or -1 - g at a boundary face that takes the boundary data of
 *                the structured face g (whose bc must be ORC_DIRICHLET or ORC_WALL);
 *   nface[e][f]  the neighbour's local face 2d' + s' that is shared;
 *   orient[e][f] how face points match: with (a, b) the node coordinates of a face point along the two
 *                other axes in increasing order, the neighbour's (a', b') is (b, a) if bit 0 is set,
 *                else (a, b), then a' -> p - a' if bit 1, b' -> p - b' if bit 2.
 * Replaces the structured element grid for the advection (which then needs oracle_set_geometry: the
 * node coordinates carry every element's position and orientation). Returns 0 or -1. */
int oracle_set_connectivity(orc_ctx *c, const int *nbr, const int *nface, const int *orient);

/* Metric terms Ja[n_x][3][3] (reference direction i, component n) and J[n_x] of the geometry set by
 * oracle_set_geometry (either pointer may be NULL); -1 without a geometry. */
int oracle_metric(const orc_ctx *c, double *Ja, double *J);

/* Apply the limiter to f[n_x][N_v] in place (element mean with the tensor Gauss-Legendre weights). */
int oracle_limit(const orc_ctx *c, double *f);

#ifdef __cplusplus
}
#endif
#endif
