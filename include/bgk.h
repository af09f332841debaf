/*
 * bgk.h -- C ABI of libbgk: one explicit SSP-RK3 step of the Boltzmann-BGK equation on a discrete
 * velocity grid, on one NVIDIA GB300 (sm_103a), after Dzanic & Martinelli, "Towards full molecular
 * gas dynamics simulations of complex flows via the Boltzmann equation" (arXiv 2308.06196).
 *
 * The method (paper Sec. 2 and 2.1):
 *   d f_k/dt + xi_k . grad f_k = (g_k - f_k) / tau                                   (Eqs. 1, 3)
 * for every node xi_k of a uniform Cartesian velocity grid with trapezoid weights w_k (Eq. 12).
 * Transport is one linear advection per velocity, discretised by flux reconstruction with
 * Gauss-Legendre solution points, DG-recovering correction functions and the upwind interface flux
 * (Eqs. 7-9). The moments Q = sum_k w_k psi_k f_k, psi = (1, xi, |xi|^2/2) (Eq. 2 with Eq. 12) feed
 * a per-point Newton solve for the discretely-conservative Maxwellian g (a Maxwellian at a
 * perturbed state whose discrete moments equal Q; Sec. 2.1, text after Eq. 13). Time stepping is
 * explicit (Sec. 2.2): Shu-Osher SSP-RK3.
 *
 * Precision forms: BGK_FP32_SPLIT stores and advects f in FP32, sums moments in FP32 per 32
 * velocities and combines them exactly in double-float, and solves the Newton problem in FP64
 * (FP32 iterations plus an FP64 residual refinement). BGK_FP64 keeps f, moments and Newton in FP64.
 *
 * Conventions
 *   - Every function returns BGK_OK (0) or a negative BGK_E* code; bgk_last_error() describes the
 *     last failure of a context. Device-side failures (Newton did not converge, non-physical state)
 *     are sticky: they are reported by bgk_synchronize(), bgk_moments() and later calls until the
 *     context is destroyed.
 *   - Host arrays are FP64, caller-owned and only read or written during the call.
 *   - Device pointers (the *_device variants) are caller-owned device memory on the context's
 *     device; the call enqueues work on the context's stream and returns without synchronising.
 *   - Point order: element-major with the element index x-fastest, then the node index x-fastest
 *     (nodes are the tensor Gauss-Legendre points of the element). n_x = elements * (p+1)^dim.
 *   - Velocity order: k = kx + n[0] * (ky + n[1] * kz); N_v = n[0] * n[1] * n[2].
 *   - All device memory of a context is allocated by bgk_create and owned by the library.
 */
#ifndef BGK_H
#define BGK_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define BGK_OK 0
#define BGK_EINVAL -1   /* bad argument or unsupported configuration */
#define BGK_ENOMEM -2   /* device memory too small for this configuration (checked before any launch) */
#define BGK_ECUDA -3    /* a CUDA runtime call failed */
#define BGK_ENEWTON -4  /* the conservative-Maxwellian Newton solve did not converge at some point */
#define BGK_EDOMAIN -5  /* non-physical state met: rho <= 0, theta <= 0 or NaN */
#define BGK_ETIMEOUT -6 /* a bounded device wait gave up (reserved; no kernel waits at present) */

#define BGK_BC_PERIODIC 0
#define BGK_BC_DIRICHLET 1     /* ghost = sampled continuous Maxwellian of bc_state (rho,u,v,w,T) */
#define BGK_BC_DIFFUSE_WALL 2  /* ghost = rho_w * M(T_w, U_w), rho_w per face point for zero net discrete
                                  mass flux, recomputed every stage (hexahedral meshes, dim = 3) */
#define BGK_BC_EXCHANGE 3      /* an x face shared with a neighbouring subdomain of a partitioned mesh: the
                                  exterior values come from a halo (bgk_set_halo); affine hexahedra in the
                                  FP32-split form; such a context steps by bgk_stage */

#define BGK_FP32_SPLIT 0
#define BGK_FP64 1

typedef struct bgk_ctx bgk_ctx;

/* Structured affine mesh of line (dim = 1), quadrilateral (dim = 2) or hexahedral (dim = 3) elements on [lo, hi].
 * Only the first dim entries of nelem/lo/hi/bc/bc_state are read. The velocity space is 3-D unless the
 * velocity grid has n[2] = 1 (see bgk_vgrid). */
typedef struct {
    int dim;
    int nelem[3];
    double lo[3], hi[3];
    int bc[3][2];              /* [direction][side 0 = lo, 1 = hi] */
    double bc_state[3][2][5];  /* Dirichlet: rho,u,v,w,T.  Wall: (unused),u_w,v_w,w_w,T_w */
} bgk_mesh;

/* Uniform velocity grid, n[d] >= 2 nodes on [lo[d], hi[d]] per axis, endpoints included, tensor
 * trapezoid weights (Sec. 2.1, Eq. 12); at least one axis needs 3 or more nodes (on two nodes every
 * function of xi_d is affine in xi_d, so with two on every axis |xi|^2 is a combination of 1 and xi,
 * the energy moment depends on the others and the conservative Maxwellian is not unique: BGK_EINVAL).
 * n[2] = 1 selects the two-dimensional velocity space (velocity dimension
 * m = 2, Sec. 2 with m >= d, so dim <= 2): velocities (u_x, u_y), the Maxwellian normalised by
 * (2 pi theta)^(m/2) (Eq. 4), E = rho |U|^2 / 2 + (m/2) rho theta; lo[2] and hi[2] are not read, the
 * third momentum component of Q is identically 0 and the third velocity component of every state
 * (bgk_set_state, Dirichlet data) is not used. */
typedef struct {
    int n[3];
    double lo[3], hi[3];
} bgk_vgrid;

typedef struct {
    int precision;           /* BGK_FP32_SPLIT (default) or BGK_FP64 */
    double body_force[3];    /* constant force per unit mass (0 = none; dim = 3). Source g (beta . psi) with
                                (sum_k w g psi psi^T) beta = (0, rho F, rho U . F): its discrete moments are
                                exactly those of -F . grad_xi f */
    int newton_max_it;       /* FP32 Newton iterations per solve, <= 0: default (2 warm, 12 cold) */
    double newton_tol;       /* reserved (the FP64 refinement fixes the final accuracy) */
    int limiter;             /* 1: Zhang-Shu positivity limiter (Sec. 2.1, Eqs. 10-11) on every stage output,
                                per element and velocity: towards the Gauss-Legendre-weighted element mean
                                where a node value is negative. Keeps element means (so conservation). */
    int chunks;              /* velocity chunks per stage, 0 = automatic */
    int vtiles_per_task;     /* 32-velocity tiles per warp task, 0 = automatic */
    int maxwellian;          /* BGK_MAXWELLIAN_CONSERVATIVE (0, the method) or BGK_MAXWELLIAN_CONTINUOUS
                                (the ablation: g = the sampled continuous Maxwellian of the moments, whose
                                discrete moments differ from them, Sec. 2.1, Eq. 13) */
    double mu_ref;           /* > 0: variable collision time tau = mu / P per point (Sec. 2, Eq. 5) with the
                                power law mu = mu_ref theta^mu_omega (reference temperature 1) and P = rho
                                theta of the point's moments at every stage; the tau argument of bgk_create
                                is then unused. FP32-split form: one velocity spacing on all axes. */
    double mu_omega;
} bgk_opts;

#define BGK_MAXWELLIAN_CONSERVATIVE 0
#define BGK_MAXWELLIAN_CONTINUOUS 1

/* Create a problem on the current CUDA device: plans the velocity tiles, builds the FR operators
 * (Eqs. 7-8) in FP64 on the host and allocates every device buffer. p in [1, 3] for dim = 2, 3 and
 * [1, 5] for dim = 1; opts may be NULL. tau > 0 is the constant relaxation time (Eq. 3 with a fixed
 * tau). The state is zero until bgk_set_state/bgk_set_f. Returns BGK_ENOMEM, without allocating,
 * when the buffers would not fit in free device memory. */
int bgk_create(const bgk_mesh *mesh, int p, const bgk_vgrid *vgrid, double tau,
               const bgk_opts *opts, bgk_ctx **out);
void bgk_destroy(bgk_ctx *ctx);
const char *bgk_last_error(const bgk_ctx *ctx);

/* Use this CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream) for all
 * later work of the context. NULL selects the context's own non-blocking stream. */
int bgk_set_stream(bgk_ctx *ctx, void *stream);

/* Sizes: number of points n_x, velocities N_v, degrees of freedom n_x * N_v, bytes of device
 * memory held. Any pointer may be NULL. */
int bgk_info(const bgk_ctx *ctx, int64_t *npoints, int64_t *nvel, int64_t *ndof, int64_t *device_bytes);

/* Node coordinates x[n_x][3] (unused components 0), host. */
int bgk_points(const bgk_ctx *ctx, double *x);

/* Set f to the sampled continuous Maxwellian (Eq. 4, velocity dimension m) of the primitive state
 * prim[n_x][5] = (rho, u, v, w, T) (theta = T), then compute its moments and conservative
 * Maxwellian. Host array (synchronises) or device array (asynchronous) variant. A point with
 * rho <= 0, T <= 0 or NaN makes the context's status BGK_EDOMAIN (returned by the host variant, by
 * the device variant's next synchronising call). */
int bgk_set_state(bgk_ctx *ctx, const double *prim);
int bgk_set_state_device(bgk_ctx *ctx, const double *d_prim);

/* Copy the distribution function in or out as f[n_x][N_v] FP64 (host; synchronises). bgk_set_f then
 * computes the moments and conservative Maxwellian of the new f (a point of non-positive density:
 * BGK_EDOMAIN, sticky). */
int bgk_set_f(bgk_ctx *ctx, const double *f);
int bgk_get_f(bgk_ctx *ctx, double *f);

/* Enqueue nsteps SSP-RK3 steps of size dt. Each step is three stages; each stage advects every
 * velocity (Eqs. 7-9), applies the BGK relaxation towards the conservative Maxwellian of the
 * stage's input (Eq. 3) and combines the Shu-Osher stage, then recomputes the moments and the
 * conservative Maxwellian of its output. Asynchronous on the context stream. BGK_EINVAL for
 * nsteps < 0 or a dt that is not positive and finite, and for connectivity tables without node
 * coordinates; a sticky device status from earlier work is returned instead of enqueuing. */
int bgk_step(bgk_ctx *ctx, double dt, int nsteps);

/* Moments Q[n_x][5] = (rho, rho u, rho v, rho w, E) of the current f (Eq. 2 with Eq. 12).
 * Host variant synchronises and returns the sticky device status; device variant is asynchronous. */
int bgk_moments(bgk_ctx *ctx, double *Q);
int bgk_moments_device(bgk_ctx *ctx, double *d_Q);

/* Perturbed state (rho', U'x, U'y, U'z, theta') of the conservative Maxwellian of the current f,
 * per point, host (synchronises). Its discrete moments equal bgk_moments(). */
int bgk_equilibrium(bgk_ctx *ctx, double *prim_out);

/* Wait for the context's stream and return the sticky device status. */
int bgk_synchronize(bgk_ctx *ctx);

/* Explicit step size min(cfl / max_k sum_d |xi_kd| / h_d, tau); with a variable collision time, the
 * smallest tau of the current state (synchronises). */
double bgk_dt(const bgk_ctx *ctx, double cfl);

/* Tile-shape autotuner: times the stage kernel for several task lengths (32-velocity tiles per warp
 * task: 2, 4, ..., 64, and the lengths that split the longest velocity chunk into 1, 2, 3, 4, 6, 8,
 * 12 or 16 equal tasks) on this context's own buffers, keeps the fastest for this context and caches it
 * per (dim, degree, velocity grid, mesh, chunking) for the rest of the process. Does not change f,
 * the moments or the equilibrium; invalidates the captured graph. *g_out (may be NULL) receives the
 * chosen length (0 for the all-FP64 form, which has no task shape). */
int bgk_autotune(bgk_ctx *ctx, int *g_out);

/* Curvilinear hexahedra (the mapped elements of Sec. 2.1's FR on unstructured curved meshes; dim = 3,
 * both precision forms, every boundary kind). x is host memory, FP64, [n_x][3]: the physical coordinates of
 * every solution node in the point order of bgk_points (element-major, x-fastest; the mesh connectivity
 * and periodicity stay those of bgk_create). Each element maps the reference cube by the degree-p
 * interpolant of its nodes. The library computes in FP64 the metric terms Ja^i (Kopriva's conservative
 * curl form, so a constant state is kept to round-off), J, and the face normals (the mean of the two
 * elements' interpolated Ja^i on a shared face), and from then on advects the reference-space flux
 * (Ja^i . xi) f / J with per-lane upwinding at every face point (Eq. 9 with u_n = Ja^i . xi). The
 * limiter's element mean becomes J-weighted; on a diffuse wall every face point's density makes the
 * net discrete mass flux through its own outward unit normal vanish; bgk_points returns x; bgk_dt uses
 * the metric. The state is kept. Returns BGK_EINVAL for dim != 3 or a node with J <= 0. */
int bgk_set_geometry(bgk_ctx *ctx, const double *x);

/* Unstructured hexahedral connectivity (with bgk_set_geometry, whose node coordinates then carry every
 * element's position and local-axis orientation; dim = 3, both precision forms). Host
 * arrays [n_elements][6], indexed by element and local face f = 2d + side (reference axis d, side 0 the
 * r_d = -1 face):
 *   nbr[e][f]    the neighbour element, or -1 - g at a boundary face, which takes the boundary data of
 *                face g of bgk_create (bc[g / 2][g % 2] must be BGK_BC_DIRICHLET or BGK_BC_DIFFUSE_WALL;
 *                a wall face gets its own wall density per face point);
 *   nface[e][f]  the neighbour's local face 2d' + s' that is shared;
 *   orient[e][f] the face-point match: for the face point with node coordinates (a, b) along our two
 *                other axes (in increasing axis order) the neighbour's (a', b') is (b, a) if bit 0 is
 *                set, else (a, b); then a' -> p - a' if bit 1, b' -> p - b' if bit 2.
 * The element count stays that of bgk_create (its grid shape no longer matters for the advection).
 * Recomputes the face normals when a geometry is already set. Returns BGK_EINVAL on a bad table. */
int bgk_set_connectivity(bgk_ctx *ctx, const int *nbr, const int *nface, const int *orient);

/* Launch timing: when on, bgk_step launches its kernels directly (not through the CUDA graph) and
 * brackets every stage and Newton launch with CUDA events on the context stream. bgk_timing()
 * synchronises and returns the summed milliseconds and launch counts since timing was switched on,
 * and the algorithmic bytes one stage launch moves on average (the storage reads and writes of f
 * that the method must make: reads of f_s and f^n, writes of the stage output). */
int bgk_set_timing(bgk_ctx *ctx, int on);
int bgk_timing(bgk_ctx *ctx, double *stage_ms, int64_t *stage_launches, double *newton_ms,
               int64_t *newton_launches, double *stage_alg_bytes);

/* ---------------------------------------------------------------------------------------------
 * Spatial domain decomposition (a mesh cut into slabs along x). The upwind common flux (Sec. 2.1,
 * Eq. 9) is the only coupling between elements, so a slab needs, before every RK stage, only its
 * x-neighbours' element layers next to the shared faces. For a context with BGK_BC_EXCHANGE x faces:
 * bgk_halo_floats: the floats of one halo, nvt * ne_y * ne_z * (p+1)^3 * 32 (velocity tiles of 32
 *   slots, face elements y + ne_y z, nodes, slots: the library's tile layout of f);
 * bgk_halo_pack: enqueues, on the context stream, copies of the element layers next to the lo and hi x
 *   faces of the source of stage `stage` (0: f^n, 1 and 2: the previous stages' outputs) into the device
 *   buffers d_lo, d_hi (caller-owned, halo_floats each; either may be NULL), for the neighbours;
 * bgk_set_halo: the device buffer holding the neighbour's layer across face 0 (lo) or 1 (hi), read by
 *   the stage kernel from then on (caller-owned, kept valid while stages run; NULL: the context's own
 *   zero halo);
 * bgk_stage: enqueues stage `stage` of an SSP-RK3 step of size dt (the three stages in order make one
 *   bgk_step; asynchronous on the context stream). Any FP32-split context may step this way; one with
 *   exchange faces must (bgk_step refuses it), with the halos refreshed before every stage.
 * ------------------------------------------------------------------------------------------- */
int bgk_halo_floats(const bgk_ctx *ctx, int64_t *nfloats);
int bgk_halo_pack(bgk_ctx *ctx, int stage, float *d_lo, float *d_hi);
int bgk_set_halo(bgk_ctx *ctx, int face, const float *d_halo);
int bgk_stage(bgk_ctx *ctx, double dt, int stage);

/* Accuracy measurement between two forms of one discretisation (e.g. the FP32-split form against the
 * all-FP64 form of the same mesh, degree and velocity grid, Sec. 2.1 Eqs. 7-13): the largest
 * |f_a - f_b| and the largest |f_b| over every real degree of freedom of the current states, computed
 * on the device. Waits for b's stream, runs on a's stream and synchronises it. The two contexts must
 * have the same element count, degree and velocity plan (else BGK_EINVAL); either may be in either
 * precision. Allocates and frees 16 bytes of device memory per call. */
int bgk_f_distance(bgk_ctx *a, bgk_ctx *b, double *max_abs_diff, double *max_abs_b);

/* ---------------------------------------------------------------------------------------------
 * Batches of independent problems. The paper runs one problem at a time; the method's steps are
 * the same per member (Sec. 2.1-2.2), only scheduled together: each RK stage of every member runs
 * in one persistent stage launch per degree present (warps take (member, element run, tile run)
 * tasks from an atomic work counter, reset by a memset in the same stream) followed by one Newton
 * launch over all members' points, and one step of all members is captured in one CUDA graph.
 *
 * bgk_batch_create: members are n distinct contexts created on the current device with
 *   precision BGK_FP32_SPLIT, dim = 1, p <= 3 and opts.chunks = 1 (the three stage buffers of a
 *   member are then disjoint, so members and their tiles run concurrently). Their meshes, degrees,
 *   velocity grids, relaxation times and boundary kinds may all differ. The batch keeps pointers to
 *   the members (not owned): destroy the batch before any member. BGK_EINVAL for an unsuitable
 *   member or a repeated one. The batch has its own stream (bgk_batch_set_stream replaces it).
 * bgk_batch_step: enqueues nsteps steps of every member, member q with time step dt[q] (host array
 *   of n). Waits on the GPU for work already enqueued on the members' streams (e.g. bgk_set_state)
 *   and makes the members' streams wait for the batch, so bgk_moments / bgk_get_f of a member
 *   afterwards see the new state. Asynchronous; returns the sticky batch status.
 * bgk_batch_synchronize: waits for the batch stream and returns the status of all members' Newton
 *   solves (BGK_EDOMAIN / BGK_ENEWTON also become sticky in every member).
 * bgk_batch_autotune: the tile-shape autotuner of the batch: for every (degree, velocity grid) class
 *   of members in turn, times the persistent stage launch with the class's task length at the
 *   lengths bgk_autotune tries (the other classes fixed) and keeps the fastest. Changes no state.
 * bgk_batch_info: total points, degrees of freedom and stage tasks of the batch.
 * bgk_batch_set_timing / bgk_batch_timing: as bgk_set_timing / bgk_timing, for the batch launches.
 * ------------------------------------------------------------------------------------------- */
typedef struct bgk_batch bgk_batch;
int bgk_batch_create(int n, bgk_ctx *const *members, bgk_batch **out);
void bgk_batch_destroy(bgk_batch *batch);
const char *bgk_batch_last_error(const bgk_batch *batch);
int bgk_batch_set_stream(bgk_batch *batch, void *stream);
int bgk_batch_step(bgk_batch *batch, const double *dt, int nsteps);
int bgk_batch_synchronize(bgk_batch *batch);
int bgk_batch_autotune(bgk_batch *batch);
int bgk_batch_info(const bgk_batch *batch, int64_t *npoints, int64_t *ndof, int64_t *tasks);
int bgk_batch_set_timing(bgk_batch *batch, int on);
int bgk_batch_timing(bgk_batch *batch, double *stage_ms, int64_t *stage_launches, double *newton_ms,
                     int64_t *newton_launches, double *stage_alg_bytes);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free entry point. The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc (code running under another framework's device-memory pool or allocator hooks,
 * processes with a no-allocation policy after start-up, or ones whose device footprint is fixed
 * once sized), for whom bgk_create, which allocates its own buffers, is not an option.
 *
 * bgk_equilibrium_noalloc computes the moments Q and the discretely-conservative Maxwellian
 * (rho', U', theta') of every point of a distribution function that the caller already holds on
 * the device -- the same quantities that bgk_moments / bgk_equilibrium return for a context after
 * bgk_set_f -- and allocates nothing:
 *   d_f     device, FP32, [npts][N_v], velocity order k = kx + n[0] * (ky + n[1] * kz) (read only);
 *   vg      the uniform velocity grid (host struct, read during the call);
 *   d_Q     device, FP64, [npts][5] (rho, rho u, rho v, rho w, E), written;
 *   d_prim  device, FP64, [npts][5] (rho', U'x, U'y, U'z, theta'), written;
 *   stream  cudaStream_t to run on (NULL: the legacy default stream). The call waits for its own
 *           work on that stream and returns its status (BGK_OK, BGK_EDOMAIN, BGK_ENEWTON).
 * Scratch: one static device array of BGK_NOALLOC_SCRATCH_BYTES. A GPU holds it from the moment the
 * library's module is loaded on it until the process exits; under lazy module loading (the CUDA
 * default since 12.2) that is the first call of this entry point on that device, so the first call is
 * the sizing point: a caller whose device footprint must not grow after start-up makes one call during
 * start-up (or sets CUDA_MODULE_LOADING=EAGER). It must hold
 * 4 * (64 + npts * (5 * ceil(N_v / 2048) + 8)) bytes; larger requests return BGK_EINVAL with a message
 * on stderr, before any work is enqueued. The first call on a device also looks up that device's
 * address of the array (with the device current). The call is synchronous -- it waits for its work
 * and reads a status word back -- so it cannot be captured in a CUDA graph: on a capturing stream it
 * returns BGK_EINVAL (message on stderr) before enqueuing anything. Every call uses the same array,
 * which keeps the last call's contents: calls that overlap on the GPU (other streams, other host
 * threads) race on it, so serialise them. No cudaMalloc, cudaFree or allocating library routine is
 * called.
 * ------------------------------------------------------------------------------------------- */
#define BGK_NOALLOC_SCRATCH_BYTES (16ll << 20)
int bgk_equilibrium_noalloc(const float *d_f, int64_t npts, const bgk_vgrid *vg, double *d_Q, double *d_prim,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif
