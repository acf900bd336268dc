/*
 * pmt.h - C ABI of a GB300 (sm_103a) library for transferring fields between
 * particles and a periodic mesh, after D. Duque and P. Espanol, "Assignment
 * of fields from particles to mesh" (arXiv 1610.05258).
 *
 * Notation follows the paper: particles mu carry values A_mu and particle
 * functions psi_mu; mesh nodes i carry values Ab_i ("A bar") and mesh
 * functions psi_i; particle values interpolated back from the mesh are Abb_mu.
 *
 * Geometry.  The mesh is periodic: dim = 1 or 2, n nodes per side, box length
 * L, spacing h = L/n, nodes at x_i = i h (2D: node (i, j) has flat index
 * j*n + i).  Mesh functions are linear (1D) or bilinear (2D) finite elements
 * (Sec. 3.1 and 3.2).  Particle functions are linear finite elements too: hat
 * functions over the particles ordered around the circle in 1D, P1 functions
 * on the periodic Delaunay triangulation of the particles in 2D (Sec. 3.2,
 * App. A).  Positions may lie anywhere; a float coordinate x is mapped to the
 * torus coordinate X = floor(frac(fl32(x * fl32(1/L))) * 2^32), and every
 * geometric decision is taken exactly on X (physical position X L / 2^32).
 *
 * Memory.  Unless stated otherwise every pointer argument is a DEVICE pointer
 * owned by the caller, float32, and must stay valid until the work queued on
 * the context's stream has finished.  Particle arrays are structure-of-arrays:
 * px[np], py[np] (py is ignored and may be NULL when dim == 1) and particle
 * fields vals[F][np] (field f of particle k at vals[f*np + k]).  Mesh fields
 * are [F][n^dim].  Arguments marked "host" are host pointers; calls that write
 * a host result wait for the stream before returning.
 *
 * Ordering.  Results never depend on the order in which particles are given
 * beyond the symbolic tie-break of exactly cocircular particles, which uses
 * the particle index (lower index = stronger perturbation).
 *
 * Errors.  Every call returns a pm_status; nothing is thrown across the ABI.
 * Argument errors are detected on the host before any launch.  Errors found
 * on the device (non-finite positions, coincident particles, a triangulation
 * whose circumcircles span more than a quarter of the box, a solve that does
 * not converge) set a device status word that the next call that waits for
 * the stream returns; pm_sync() returns it explicitly.  pm_last_error() gives
 * a one-line description of the last failure.
 *
 * Concurrency.  A context owns all its workspace (sized at creation, so no
 * call allocates device memory) and its calls must not overlap: issue them on
 * one stream, or synchronise between them.
 */
#ifndef PMT_H
#define PMT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pm_status {
    PM_OK = 0,
    PM_EINVAL = 1,      /* bad argument (size, dimension, null pointer, F too large) */
    PM_ENOMEM = 2,      /* workspace allocation failed at creation                    */
    PM_ENOTCONV = 3,    /* mass solve reached max_iter above the requested tolerance  */
    PM_ETIMEOUT = 4,    /* a bounded device-side wait gave up                         */
    PM_EDEGENERATE = 5, /* non-finite or coincident positions, or a too sparse set    */
    PM_ECUDA = 6        /* a CUDA runtime call failed                                  */
} pm_status;

typedef struct pm_ctx pm_ctx;

/* Start of the mass solve. PM_WS_DIRECT: the exact inverse of the uniform
 * periodic mass matrix applied to b (M = M1 (x) M1, M1 = (h/6) circ(1,4,1),
 * whose inverse circulant has entries decaying as (sqrt 3 - 2)^|j|; applied as
 * separable convolutions truncated below 2e-10), after which conjugate
 * gradients only confirm the residual and set the mean mode exactly. */
enum { PM_WS_DELTA = 0, PM_WS_ZERO = 1, PM_WS_USER = 2, PM_WS_NET = 3, PM_WS_DIRECT = 4 };

/* Right-hand side of the mass assignment. PM_RHS_EXACT: b_j = int A psi_j
 * exactly (Eq. proj; conservative to rounding). PM_RHS_APPB: the quadrature
 * of App. B, read for this mesh as follows: on every mesh element A is
 * replaced by its quadratic (1D) or biquadratic (2D) interpolant through its
 * values at the element's nodes, edge midpoints and centre, and that
 * interpolant is integrated exactly against the hats. This amounts to b_i =
 * (h/3)^dim times the sum of A over the 3^dim points of the twice refined mesh
 * around node i. Not conservative (App. B); the solve reports cons_err. */
enum { PM_RHS_EXACT = 0, PM_RHS_APPB = 1 };

/* Solver of the mesh system M Ab = b (Sec. 2.4, Eq. phi_def). PM_SOLVER_CG:
 * conjugate gradients with FP64 inner products. PM_SOLVER_CHEBYSHEV:
 * Chebyshev iteration on the closed-form spectrum of the periodic mass
 * matrix ([h/3, h] in 1D, [h^2/9, h^2] bilinear, [h^2/4, h^2] P1), with no
 * inner products; the step count follows from ||b - M x0|| and the Chebyshev
 * bound, and the true residual is checked at the end. Both set the mean mode
 * exactly (conservative to rounding) and report the same pm_solve_info
 * (iters = Chebyshev steps). The particle-side full-mass solve always uses
 * conjugate gradients. */
enum { PM_SOLVER_CG = 0, PM_SOLVER_CHEBYSHEV = 1 };

typedef struct pm_net pm_net;

/* Options of the mass solve  M Ab = b  (Sec. 2.4, Eq. phi_def). */
typedef struct pm_solve_opts {
    int warm_start;  /* PM_WS_DELTA: start from the delta assignment (default);
                        PM_WS_ZERO: start from zero; PM_WS_USER: start from x0  */
    double rtol;     /* stop when ||b - M Ab||_2 <= rtol ||b||_2 (default 1e-6)  */
    int max_iter;    /* iteration cap (default 200)                              */
    const float *x0; /* device [F][n^dim], read when warm_start == PM_WS_USER     */
    pm_net *net;     /* PM_WS_NET: start from delta + alpha c, c the network's
                        correction and alpha the step that minimises the 2-norm
                        of the start's residual (alpha = 0 keeps the delta start);
                        only fields whose delta start is above 1e-4 in relative
                        residual get the network (the others keep delta), which
                        makes this start wait for the stream once */
    int rhs_mode;    /* PM_RHS_EXACT (default) or PM_RHS_APPB (pm_assign_mass)   */
    int solver;      /* PM_SOLVER_CG (default) or PM_SOLVER_CHEBYSHEV (mesh solve) */
} pm_solve_opts;

/* Per-field report of a mass solve (host memory, one entry per field). */
typedef struct pm_solve_info {
    int iters;             /* conjugate-gradient iterations taken                     */
    double init_rel_resid; /* ||b - M x0|| / ||b|| of the start vector (after its mean
                              is set exactly)                                          */
    double rel_resid;      /* true residual ||b - M Ab|| / ||b|| at exit, recomputed   */
    double sum_particles;  /* sum_mu v_mu A_mu  (Eq. cons, particle side)              */
    double sum_mesh;       /* sum_i v_i Ab_i with v_i = h^dim (Eq. cons, mesh side)     */
    double cons_err;       /* |sum_mesh - sum_particles| / sum_mu v_mu |A_mu|          */
    double energy_mesh;    /* int Ab^2 = Ab^T M Ab of the mesh fields (stability, Sec. 2.1
                              Eq. stab in integral form)                               */
    double energy_particles; /* int A^2 = A^T M_p A, (M_p)_{mu nu} = int psi_mu psi_nu, of
                              the particle fields (0 when the call has none)           */
} pm_solve_info;

/* Create a context for one periodic mesh (dim 1 or 2, n >= 4 nodes per side,
 * box length L > 0) able to take up to max_particles particles and max_fields
 * fields per call. stream is a cudaStream_t (NULL = legacy default stream).
 * Allocates all device workspace now. *out is set only on success. The mesh
 * functions are linear (1D) / bilinear (2D), as pm_ctx_create_mesh with
 * PM_MESH_Q1. */
pm_status pm_ctx_create(pm_ctx **out, int dim, int n, double L, long long max_particles, int max_fields,
                        void *stream);

/* Mesh functions psi_i of a 2D context (Sec. 3.2 uses linear FE functions on
 * a triangulation of the node grid). PM_MESH_Q1: bilinear on the square cells
 * (mass matrix (h^2/36)[1 4 1; 4 16 4; 1 4 1]). PM_MESH_P1: every cell split
 * by its diagonal from node (i, j) to (i+1, j+1), hats linear on the
 * triangles (mass matrix (h^2/12) times 6 at the node and 1 at its six
 * neighbours (i+-1, j), (i, j+-1), (i+1, j+1), (i-1, j-1)). G2P, FLIP, the
 * exact right-hand side, the mesh solve and the mesh -> particle integrals
 * follow the kind; delta does not depend on it. PM_RHS_APPB, PM_WS_DIRECT and
 * the network start exist for PM_MESH_Q1 only (PM_EINVAL otherwise). In 1D
 * both kinds are the linear hats. */
enum { PM_MESH_Q1 = 0, PM_MESH_P1 = 1 };
pm_status pm_ctx_create_mesh(pm_ctx **out, int dim, int n, double L, long long max_particles, int max_fields,
                             int mesh_kind, void *stream);
void pm_ctx_destroy(pm_ctx *ctx);
pm_status pm_ctx_set_stream(pm_ctx *ctx, void *stream);
/* Wait for the context's stream; return the device status word and clear it. */
pm_status pm_sync(pm_ctx *ctx);
const char *pm_last_error(const pm_ctx *ctx);
/* Bytes of device workspace the context holds. */
long long pm_ctx_workspace_bytes(const pm_ctx *ctx);

/* Mesh -> particle interpolation, Sec. 2.2 Eq. delta2 (Table 1, right
 * column for delta, FLIP and mass-delta):  out[f][k] = sum_i mesh[f][i] psi_i(r_k).
 * mesh [F][n^dim], px/py [np], out [F][np]. np may be 0. Asynchronous. */
pm_status pm_interpolate(pm_ctx *ctx, const float *mesh, int F, const float *px, const float *py, long long np,
                         float *out);

/* Delta interpolation (Eq. delta2, as pm_interpolate) at the particles of the
 * context's most recent sort, with the results in that sorted order: out
 * [F][np], slot s holding the value at caller particle perm[s] (the
 * permutation pm_sort returns: cell-major, then caller index). The same bits
 * as pm_interpolate gives for that particle. The particles are those of the
 * last call that sorted: pm_sort, pm_particle_volumes, pm_triangulate and
 * every assignment, right-hand side and mesh -> particle projection other
 * than pm_interpolate, on this context; their positions are not read again.
 * np must equal that call's particle count (PM_EINVAL otherwise, and when no
 * call has sorted yet). In sorted order a warp's particles share a few cells,
 * so their corner reads mostly hit in L1: use it where the caller's particles
 * stay put between the assignment and the interpolation and sorted results
 * serve (or are reordered once with the permutation). Asynchronous. No
 * counterpart in the paper: a data-layout variant of Eq. delta2. */
pm_status pm_interpolate_sorted(pm_ctx *ctx, const float *mesh, int F, long long np, float *out);

/* delta assignment, Sec. 2.2 Eq. delta:  mesh_out[f][i] = A_f(r_i) =
 * sum_mu vals[f][mu] psi_mu(r_i).  Needs np >= 2 (1D) / np >= 3 (2D).
 * Asynchronous. */
pm_status pm_assign_delta(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                          float *mesh_out);

/* FLIP assignment, Sec. 2.3 Eqs. PIC and FLIP_vol:
 *   v_i = sum_mu v_mu psi_i(r_mu),  Ab_i = sum_mu A_mu v_mu psi_i(r_mu) / v_i,
 * with particle volumes v_mu = int psi_mu (Eq. part_v). A node with v_i = 0
 * (no particle in its support, Sec. 2.3) gets Ab_i = 0.
 * node_volume_out [n^dim] (device, may be NULL) receives v_i; empty_nodes
 * (host, may be NULL) receives the number of nodes with v_i = 0 and makes the
 * call wait for the stream. */
pm_status pm_assign_flip(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                         float *mesh_out, float *node_volume_out, long long *empty_nodes);

/* PIC assignment, Sec. 2.3 Eq. PIC with the mesh volumes of Eq. mesh_v:
 *   Ab_i = sum_mu A_mu v_mu psi_i(r_mu) / v_i,  v_i = int psi_i = h^dim,
 * v_mu = int psi_mu (Eq. part_v). Conservative with the mesh volumes
 * (sum_i h^dim Ab_i = sum_mu v_mu A_mu); unlike FLIP it does not reproduce a
 * constant field where the particle volumes around a node do not add up to
 * h^dim. Layouts, ownership and errors as pm_assign_delta. Asynchronous. */
pm_status pm_assign_pic(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                        float *mesh_out);

/* Mass assignment ("mass-delta" particle -> mesh direction), Sec. 2.4
 * Eqs. proj and phi_def:  Ab = M^-1 b  with  m_ij = int psi_i psi_j  and
 * b_j = int A(r) psi_j(r) dr,  A the particle interpolant (Eq. part_interp).
 * b is integrated exactly (particle triangles clipped against mesh cells).
 * The solve is conjugate gradients on the matrix-free mass stencil, FP32
 * vectors with compensated sums, FP64 reductions; the mean mode of Ab is set
 * exactly from sum_j b_j first, so the result is conservative (Eq. cons) to
 * rounding whatever the iteration count. info (host, F entries, may be NULL)
 * makes the call wait for the stream; it also runs the stability
 * diagnostics (energy_mesh of the result, energy_particles of the input). */
pm_status pm_assign_mass(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                         float *mesh_out, const pm_solve_opts *opts, pm_solve_info *info);

/* pm_assign_mass with the particles and the result in HOST memory (same
 * method, same arithmetic, the same result bit for bit). px, py [np] and
 * vals [F][np] are read from host memory, mesh_out [F][n^dim] is written to
 * host memory. The positions are uploaded first, on the context's stream;
 * the values on a second stream of the context, while the sort and the
 * particle functions (which do not need them) run; the value gather waits for
 * them. Page-locked host buffers (cudaHostAlloc / cudaHostRegister) let the
 * uploads overlap the kernels; pageable ones work but copy synchronously.
 * The context holds device copies of the inputs and output at its maximum
 * sizes, allocated by its first host-buffer call (PM_ENOMEM if that fails);
 * later calls allocate nothing. Asynchronous like pm_assign_mass: mesh_out is
 * valid once the context's stream has completed (pm_sync), or on return when
 * info is given. The warm start PM_WS_USER (a device x0) is rejected with
 * PM_EINVAL; everything else as pm_assign_mass. No counterpart in the paper:
 * host-side data handling around Sec. 2.4. */
pm_status pm_assign_mass_host(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                              float *mesh_out, const pm_solve_opts *opts, pm_solve_info *info);

/* Lumped assignment (Table 1, "lumped" row; Sec. 2.4 remarks, Eq. lumped
 * with v_i = sum_j m_ij = h^dim):  mesh_out[f][i] = int A_f psi_i / h^dim,
 * the exact right-hand side of the mass assignment divided by the node
 * volume (no solve). Layouts, ownership and errors as pm_assign_mass. */
pm_status pm_assign_lumped(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                           float *mesh_out);

/* Mesh -> particle projections other than delta (Table 1, right column).
 * With the mesh interpolant Ab(r) = sum_i mesh[f][i] psi_i(r) and the particle
 * functions psi_mu (P1 on the periodic Delaunay triangulation in 2D, hats in
 * 1D), c_mu = int Ab psi_mu is integrated exactly (clipped triangle-cell
 * pieces by Green's theorem in 2D, Simpson on the merged breakpoints in 1D)
 * and
 *   pm_interpolate_lumped: out[f][mu] = c_mu / v_mu          (Eq. lumped)
 *   pm_interpolate_mass:   sum_nu m_{mu nu} out[f][nu] = c_mu (Eq. proj2, the
 *                          "full mass" projection), m_{mu nu} = int psi_mu
 *                          psi_nu applied matrix-free from the stars;
 *                          conjugate gradients with the Jacobi preconditioner
 *                          from the lumped start, FP64 reductions, to
 *                          ||c - M_p x|| <= rtol ||c|| (opts->rtol, max_iter;
 *                          warm_start ignored; opts may be NULL for 1e-6/200).
 * Both conserve the integral: sum_mu v_mu out_mu = int Ab (exactly for the
 * lumped one, to the residual for the full mass one). mesh [F][n^dim],
 * px/py [np] (np >= 3 in 2D, >= 2 in 1D), out [F][np] caller order, device
 * pointers. info (host, F entries, may be NULL): iters, start and final
 * relative residual, sum_mesh = int Ab, sum_particles = sum v_mu out_mu,
 * cons_err relative to sum |c_mu|, energy_mesh = int Ab^2 of the input mesh,
 * energy_particles = int Abb^2 of the result (full mass only: the
 * projection keeps energy_particles <= energy_mesh); passing it makes the
 * call wait. Errors as
 * pm_assign_mass (PM_ENOTCONV when the iteration cap is reached). */
pm_status pm_interpolate_lumped(pm_ctx *ctx, const float *mesh, int F, const float *px, const float *py, long long np,
                                float *out);
pm_status pm_interpolate_mass(pm_ctx *ctx, const float *mesh, int F, const float *px, const float *py, long long np,
                              float *out, const pm_solve_opts *opts, pm_solve_info *info);

/* Mass right-hand side alone: b_out[f][j] = int A_f(r) psi_j(r) dr (Sec. 2.4,
 * Eq. proj), exact. Asynchronous. */
pm_status pm_mass_rhs(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                      float *b_out);
/* The same with the quadrature chosen: rhs_mode PM_RHS_EXACT (as pm_mass_rhs)
 * or PM_RHS_APPB (App. B, see PM_RHS_APPB). PM_EINVAL on another mode. */
pm_status pm_mass_rhs_mode(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                           int rhs_mode, float *b_out);

/* Mesh mass matrix applied to mesh fields: y[f] = M x[f], m_ij = int psi_i psi_j
 * (Sec. 2.4). Asynchronous. */
pm_status pm_mass_apply(pm_ctx *ctx, const float *x, int F, float *y);

/* Solve M x[f] = b[f] (Sec. 2.4, Eq. phi_def) by conjugate gradients; the
 * start vector is zero or opts->x0 (PM_WS_DELTA is read as zero here).
 * info as in pm_assign_mass (sum_particles = sum_j b_j there; energy_mesh of
 * x, energy_particles 0). */
pm_status pm_mass_solve(pm_ctx *ctx, const float *b, int F, float *x, const pm_solve_opts *opts,
                        pm_solve_info *info);

/* Particle volumes v_mu = int psi_mu (Sec. 2.1, Eq. part_v), in the caller's
 * particle order. v_out [np]. Asynchronous. */
pm_status pm_particle_volumes(pm_ctx *ctx, const float *px, const float *py, long long np, float *v_out);

/* The periodic Delaunay triangulation of the particles (2D only, Sec. 3.2,
 * App. A): every triangle once, as caller particle indices (p, a, b) counter-
 * clockwise with p the vertex that comes first in the library's cell order,
 * and the image offsets (ax, ay, bx, by) in box lengths of a and b relative
 * to p. tri_out [max_tri][3], off_out [max_tri][4] (device, int32); *ntri
 * (host) receives the count (2 np on the torus). Waits for the stream. */
pm_status pm_triangulate(pm_ctx *ctx, const float *px, const float *py, long long np, int *tri_out, int *off_out,
                         long long max_tri, long long *ntri);

/* Counting sort of the particles by mesh cell (row-major cell, then caller
 * index; 1D: then torus coordinate): perm_out [np] receives caller indices in
 * sorted order, cell_start_out [n^dim + 1] the first sorted slot of every cell.
 * Asynchronous. */
pm_status pm_sort(pm_ctx *ctx, const float *px, const float *py, long long np, int *perm_out, int *cell_start_out);

/* ---------------------------------------------------------------------------
 * Particle advection: the driver step between mesh->particle and
 * particle->mesh in the paper's experiments (Sec. 3.1 dx/dt = u, Sec. 3.2
 * rigid rotation, Sec. 3.3 motion with the interpolated velocity). Positions
 * are updated in place and wrapped into [0, L). The shift and the rotation
 * compute the new position in FP64 from the float32 one, in the expression
 * order stated below with one rounding per operation, wrap it into [0, L) and
 * round it to float32 (a value that rounds to L becomes 0): the result is a
 * plain function of the inputs, reproducible bit for bit. Asynchronous.
 * ------------------------------------------------------------------------- */
/* x += dx (and y += dy in 2D), as x' = wrap(x + dx). */
pm_status pm_advect_shift(pm_ctx *ctx, float *px, float *py, long long np, double dx, double dy);
/* Rotate every particle about (cx, cy) by `angle` radians (2D only):
 * x' = cx + (c X - s Y), y' = cy + (s X + c Y) with X = x - cx, Y = y - cy,
 * c = cos(angle), s = sin(angle) from the host's libm. */
pm_status pm_advect_rotate(pm_ctx *ctx, float *px, float *py, long long np, double cx, double cy, double angle);
/* Explicit midpoint step  r += dt u(r + dt/2 vel)  with u interpolated from
 * the mesh velocity mesh_vel [dim][n^dim] (Eq. delta2) and vel [dim][np] the
 * particle velocity at the current position; vals [F][np] (may be NULL) are
 * multiplied by `factor` in the same pass. FP32 arithmetic (the midpoint is
 * a float32 position, as every particle position). */
pm_status pm_advect_rk2(pm_ctx *ctx, const float *mesh_vel, const float *vel, float *px, float *py, long long np,
                        double dt, float *vals, int F, double factor);

/* ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper: a small network predicts
 * the mass assignment of Sec. 2.4 from the delta assignment, Eq. delta, and
 * the residual of that start, r = b - M delta (b = int A psi_j, Eq. proj):
 * the exact correction is M^-1 r, a fixed operator that decays fast for
 * kappa(M) = 9 and that a local network can approximate; the start is
 * delta + max|A| / 64 * network output); conjugate gradients then finish the
 * solve to the requested residual, so the result keeps the solver's
 * guarantees whatever the network predicts).
 *
 * Network: 3x3 periodic convolutions 2 -> 32 -> 32 -> 32 -> 1, bias, ReLU
 * after the first three; BF16 activations, FP32 accumulation; the 32 -> 32
 * layers run on the tensor cores. Meshes must be 2D with n a multiple of 128.
 * Parameters: pm_net_num_params() floats, per layer W [Co][Ci][3][3] then
 * b [Co], tap (dy, dx) at [dy + 1][dx + 1] reading x[y + dy][x + dx].
 * ------------------------------------------------------------------------- */
int pm_net_num_params(void);
/* Allocate a network for up to max_batch images of up to max_n x max_n. */
pm_status pm_net_create(pm_net **out, int max_n, int max_batch, void *stream);
void pm_net_destroy(pm_net *net);
pm_status pm_net_set_stream(pm_net *net, void *stream);
/* Checkpoint: parameters, then the two Adam moments (3 * pm_net_num_params()
 * host floats) and the step count. */
pm_status pm_net_state(pm_net *net, float *host_out, long long *step);
/* Restore parameters (and the Adam moments if with_moments) and the step. */
pm_status pm_net_load(pm_net *net, const float *host_in, int with_moments, long long step);
/* out [B][n][n] = network(x [B][2][n][n]) (device). */
pm_status pm_net_forward(pm_net *net, const float *x, int B, int n, float *out);
/* One Adam step (learning rate lr) on 0.5 mean((network(x) - target)^2);
 * loss (host, may be NULL) receives the loss before the step and makes the
 * call wait. */
pm_status pm_net_train_step(pm_net *net, const float *x, const float *target, int B, int n, float lr, double *loss);
/* Gradient of the last training step (host, pm_net_num_params() floats). */
pm_status pm_net_grad(pm_net *net, float *host_out);
/* Network input of a mass assignment: delta assignment delta_out [F][n^2],
 * features feat_out [F][2][n^2] (delta / max|A_f| and
 * 64 (b_f - M delta_f) / (h^2 max|A_f|)) and, if scale_out (host, F floats)
 * is given, max|A_f| (waits). The network's target is
 * 64 (mass - delta) / max|A_f|. */
pm_status pm_net_features(pm_ctx *ctx, const float *px, const float *py, long long np, const float *vals, int F,
                          float *delta_out, float *feat_out, float *scale_out);

/* ---------------------------------------------------------------------------
 * Batches of independent instances (no counterpart in the paper: many
 * periodic problems of uneven mesh and particle sizes advanced together).
 *
 * All instances share one packed workspace and every phase of a step (pack,
 * sort, stars, right-hand side, start, per-instance solve on a thread-block
 * cluster) is one launch over all instances (about 18 kernels per step in
 * total), captured
 * once into a CUDA graph and replayed while the arguments stay the same.
 * ------------------------------------------------------------------------- */
typedef struct pm_batch pm_batch;
/* ninst 2D instances; instance k has an n[k] x n[k] mesh of box length L[k]
 * and up to max_np[k] particles (all host arrays; sum of max_np below 2^28).
 * Allocates the packed workspace now. stream is the caller's stream the
 * batch synchronises with. tune: 0 = choose, on the first call, by timing
 * one step for each setting (the solve's threads per CTA and CTAs per
 * instance, instances packed as given or largest first), cached per device
 * and size class for the process; 256, 512 or 1024 = that many threads, one
 * CTA per instance, instances as given. PM_EINVAL on any other value or an
 * invalid instance. */
pm_status pm_batch_create(pm_batch **out, int ninst, const int *n, const double *L, const long long *max_np,
                          int max_fields, int tune, void *stream);
void pm_batch_destroy(pm_batch *b);
const char *pm_batch_last_error(const pm_batch *b);
/* The solve's setting: threads per CTA, CTAs per instance (a thread-block
 * cluster of 1, 4 or 8 that reduces through distributed shared memory),
 * instances packed largest first (1) or as given (0), and the step time
 * measured when the autotuner chose it (0 if not tuned). Outputs may be NULL. */
pm_status pm_batch_tuning(const pm_batch *b, int *threads, int *cluster, int *largest_first, double *step_ms);
/* Fix the solve's setting (threads 256, 512 or 1024; cluster 1, 4 or 8;
 * packing order) instead of the autotuner's; PM_EINVAL otherwise. */
pm_status pm_batch_set_tuning(pm_batch *b, int threads, int cluster, int largest_first);
/* Start of the batch's solves: PM_WS_DIRECT (default: the exact inverse of
 * each instance's mass matrix), PM_WS_DELTA (the delta assignment) or
 * PM_WS_ZERO; PM_EINVAL otherwise. */
pm_status pm_batch_set_start(pm_batch *b, int warm_start);
/* Mass assignment of every instance (as pm_assign_mass from the batch's
 * start, PM_WS_DIRECT unless pm_batch_set_start chose another; the residual
 * is checked and conjugate gradients continue only while it is above rtol).
 * px, py, vals, mesh_out are HOST arrays of ninst DEVICE pointers (instance
 * k: px[k][np[k]], vals[k] [F][np[k]], mesh_out[k] [F][n[k]^2]); np is a host
 * array (3 <= np[k] <= max_np[k]). Without info the step is a graph replay
 * (asynchronous on the caller's stream). info (host, ninst*F entries,
 * instance-major, may be NULL) makes the call run the step with the
 * stability integrals and wait; errors of any instance are reported then. */
pm_status pm_batch_assign_mass(pm_batch *b, const float *const *px, const float *const *py, const long long *np,
                               const float *const *vals, int F, float *const *mesh_out, double rtol, int max_iter,
                               pm_solve_info *info);

/* ---------------------------------------------------------------------------
 * Allocation-free mass solve (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc when they need the solve: host
 * applications and plugin frameworks that own all device memory through their
 * own pool and forbid allocations by the libraries they load, and
 * latency-critical loops that cannot take the implicit device synchronisation
 * of cudaMalloc/cudaFree. Same result as pm_mass_solve() (conjugate gradients
 * on M x[f] = b[f], mean mode set exactly, true residual checked), but it
 * needs no context: its scratch is one file-scope device array of about
 * 16.2 MB that every GPU loading the library holds until exit. The caller
 * passes b [F][n^dim] and x [F][n^dim] (device); x is the start vector when
 * use_x0 != 0, else the solve starts from zero. Limit: F * n^dim <= 2^20
 * values (e.g. F = 1 at 1024^2, F = 4 at 512^2); larger sizes, dim not 1 or 2,
 * n < 4, L <= 0 or F outside 1..8 return PM_EINVAL before any GPU work. The
 * solve's grid is clamped to the 1024 blocks whose reduction partials the
 * array holds. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture. All
 * calls share the one array and each call leaves its contents behind, so calls
 * whose work overlaps on the GPU (different streams or threads without
 * ordering) race and give wrong results; serialise them. iters and rel_resid
 * (host, F entries each, may be NULL) make the call wait for the stream and
 * receive the iteration count and true relative residual per field; then
 * PM_ENOTCONV / PM_ETIMEOUT are reported too. With both NULL the call returns
 * as soon as the work is queued, and a solve that times out or does not
 * converge is NOT reported: the next call overwrites the status word. Errors
 * are status codes only (there is no context for pm_last_error()). No call
 * allocates memory. */
pm_status pm_mass_solve_noalloc(int dim, int n, double L, const float *b, int F, float *x, double rtol, int max_iter,
                                int use_x0, void *stream, int *iters, double *rel_resid);

/* ---------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper).
 * ------------------------------------------------------------------------- */
enum {
    PM_PH_SORT = 0,
    PM_PH_TRIANGULATE = 1, /* particle functions: Delaunay stars (2D) or 1D order, volumes */
    PM_PH_DELTA = 2,
    PM_PH_FLIP = 3,
    PM_PH_RHS = 4,
    PM_PH_SOLVE = 5,
    PM_PH_G2P = 6,
    PM_PH_ADVECT = 7,
    PM_PH_OTHER = 8,
    PM_PH_NET = 9,         /* learned warm start: network inference */
    PM_NPHASE = 10
};
/* When enabled, every phase's kernels are bracketed by CUDA events recorded
 * on the context's stream; pm_profile_read() waits for the stream and returns
 * the accumulated milliseconds and call counts per phase (arrays of
 * PM_NPHASE, either may be NULL), resetting them if `reset`. */
pm_status pm_profile(pm_ctx *ctx, int enable);
pm_status pm_profile_read(pm_ctx *ctx, double *ms, long long *calls, int reset);
/* Work counters of the 2D triangulation (Sec. 3.2 particle functions),
 * collected while pm_profile(ctx, 2) is in effect: that mode runs a counting
 * build of the triangulation kernel (same results, slower; not for timing).
 * counts[0..4] = candidates examined, candidates within the distance bound,
 * in-circle vertex tests, clips of the Voronoi cell, sum of the cell sizes
 * after each clip, summed over all particles and calls since the last reset,
 * each particle counted once, in the pass that completes its cell.
 * counts[5] = cells the main pass gave up to the retry passes (capacity 9),
 * counts[6] = cells the first retry pass gave up to the last (capacity 12),
 * counts[7] = in-circle vertex tests the float filter could not decide and
 * left to the exact 128-bit predicate.
 * Waits for the context's stream. Host array of `ncounts` entries (entries
 * past 7 are written as 0). PM_EINVAL on a NULL ctx or array. */
pm_status pm_work_read(pm_ctx *ctx, long long *counts, int ncounts, int reset);
const char *pm_phase_name(int phase);
/* Number of kernels this library has launched in the process so far. */
long long pm_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* PMT_H */
