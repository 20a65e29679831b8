/*
 * cgp.h - C ABI of the GB300 coarse-grid projection (CGP) Poisson library.
 *
 * The library implements the per-time-step hot path of the CGP method for
 * incompressible MHD (Kashefi, "A coarse-grid projection method for
 * accelerating incompressible MHD flow simulations", Sect. 2.2-2.3):
 *
 *   restrict u_f -> u_c (Eq. 19), form the Poisson right-hand side
 *   (Eq. 12 potential, Eq. 15 pressure), solve the P1 Laplacian by
 *   Jacobi-preconditioned CG, prolong the solution back (Eq. 20), and form
 *   grad(phi) and the Lorentz force j x B per fine triangle (Eqs. 4, 7, 13-14).
 *
 * Conventions shared by every call
 *   - Every function returns a cgp_status; nothing throws and no kernel traps.
 *     cgp_last_error() gives a human-readable message for the calling thread.
 *   - "device" pointers are CUDA device (or managed) pointers on the device
 *     that was current when the mesh was assembled; "host" pointers are plain
 *     host memory.  The caller owns every buffer it passes; the library owns
 *     the mesh data and solver scratch it allocates in cgp_assemble and frees
 *     in cgp_mesh_destroy.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream) unless stated otherwise.
 *   - Solver scratch lives in the mesh: two solves on the same mesh must not
 *     overlap on the GPU (use one stream per mesh, or one mesh per stream).
 *   - Vectors are contiguous FP64 arrays; index i of a coarse vector is
 *     coarse node i.
 *
 * Fine-mesh numbering (the nested 4-way splits of Sect. 2.3, Eq. 18; k = levels)
 *   - level l + 1 splits every triangle of level l (level 0 is the coarse
 *     mesh, level k the fine mesh): its nodes [0, n_l) are level l's nodes,
 *     node n_l + e is the midpoint of level-l edge e, edges sorted by
 *     (min vertex, max vertex);
 *   - triangle 4T + c of level l + 1 is child c of level-l triangle
 *     T = (a, b, c): (a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c),
 *     (m_ab, m_bc, m_ca); the fine children of coarse triangle T are the
 *     4^k consecutive triangles from 4^k T.
 *   The coarse nodes are the prefix of every level, so injection (Eq. 19) is
 *   the prefix q_f[0, n_c).
 */
#ifndef CGP_H
#define CGP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CGP_OK = 0,
  CGP_ERR_INVALID_ARG = 1,   /* bad handle, size, pointer or option */
  CGP_ERR_CUDA = 2,          /* a CUDA runtime call failed (message says which) */
  CGP_ERR_NOT_CONVERGED = 3, /* max_it reached; x holds the last iterate */
  CGP_ERR_BREAKDOWN = 4,     /* p.Kp <= 0: the matrix is not positive on the Krylov space */
  CGP_ERR_NONFINITE = 5,     /* NaN or Inf met in b, x0 or a reduction */
  CGP_ERR_TIMEOUT = 6,       /* a grid barrier of the persistent solver gave up */
  CGP_ERR_OOM = 7            /* device allocation failed */
} cgp_status;

typedef struct cgp_mesh_s* cgp_mesh;

typedef enum { CGP_RHS_POTENTIAL = 0, CGP_RHS_PRESSURE = 1 } cgp_rhs_kind;
typedef enum { CGP_FP64 = 0, CGP_MIXED = 1 } cgp_precision;

typedef struct {
  double tol;          /* stop when ||b - K x||_2 <= tol ||b||_2 (b after mean projection) */
  int max_it;          /* FP64: PCG iteration cap; MIXED: cap on the total inner iterations */
  int precision;       /* cgp_precision */
  double inner_tol;    /* MIXED: relative residual reduction of each FP32 inner solve */
  int use_x0;          /* 1: x holds the initial guess on entry; 0: start from zero */
  int max_sweeps;      /* MIXED: cap on refinement sweeps (<= 0 selects 50) */
} cgp_solve_opts;

typedef struct {
  int iterations;            /* PCG iterations (MIXED: inner iterations summed) */
  int outer_sweeps;          /* MIXED: refinement sweeps; FP64: restarts from the true residual (normally 0) */
  double rel_res_recursive;  /* FP64: recursive-residual norm / ||b||; MIXED: as rel_res_true */
  double rel_res_true;       /* ||b - K x|| / ||b|| of the returned x */
  int status;                /* cgp_status of the solve */
} cgp_solve_info;

/*
 * cgp_assemble - build a mesh pair and its Galerkin P1 operators (Sect. 2.3).
 *
 * xy_c   host, [n_c][2] coarse node coordinates (FP64, interleaved x, y).
 * tri_c  host, [t_c][3] coarse triangles, counter-clockwise, 0-based.
 * levels coarsening levels k between the fine and the coarse mesh (Eq. 18):
 *        1, 2 or 3 nested uniform 4-way splits (t_f = 4^k t_c).
 * out    receives the handle.
 *
 * Builds the fine mesh by the numbering above, the CSR pattern of the coarse
 * node graph (columns ascending), and on the GPU: K_ij = int grad psi_i .
 * grad psi_j, Gx_ij = int psi_j d_x psi_i, Gy_ij = int psi_j d_y psi_i,
 * D^-1 = 1/K_ii (FP64 and FP32 copies) and the fine node coordinates.
 * Blocks until the device data is ready.  Inputs are copied; the caller may
 * free them afterwards.  Errors: INVALID_ARG for sizes <= 0, indices out of
 * range, clockwise or degenerate triangles, levels outside [1, 3], or a fine
 * mesh beyond 32-bit indexing; OOM; CUDA.
 */
int cgp_assemble(const double* xy_c, int n_c, const int* tri_c, int t_c, int levels,
                 cgp_mesh* out);

/* Sizes of a mesh pair; any output pointer may be NULL.  n_e counts the coarse
 * edges, n_f and t_f the finest level, nnz K's pattern. */
int cgp_mesh_query(cgp_mesh m, int* n_c, int* t_c, int* n_e, int* n_f, int* t_f, int* nnz);

/* Coarsening levels k and the node count of every level, nodes host [k + 1]
 * (nodes[0] = n_c, nodes[k] = n_f); either pointer may be NULL. */
int cgp_mesh_levels(cgp_mesh m, int* levels, int* nodes);

/*
 * cgp_set_far_field - boundary condition of the solves on this mesh far from
 * the cylinder.  dirichlet = 0 (default): the natural condition everywhere
 * (d_n x = F . n, the reading of "the electric field vanishes far away" as
 * j . n = 0; K is singular and b, x0 and x are projected to mean zero).
 * dirichlet = 1: x = 0 on the outer boundary (the other reading of the same
 * sentence, Sect. 3), the natural condition on the other boundaries; the
 * outer-boundary rows and columns of K become the identity, b and x0 are
 * taken as zero there, nothing is projected.  The outer boundary is every
 * boundary curve (sides of one triangle, oriented as in their triangle) of
 * positive signed area; curves around holes are negative.  The first call
 * with 1 builds that system (synchronous; one allocation of about
 * 12 nnz + 13 n_c bytes, freed with the mesh).  Affects every later solve on
 * the mesh, batched ones included.  INVALID_ARG for other values or when the
 * mesh has no outer boundary.
 */
int cgp_set_far_field(cgp_mesh m, int dirichlet);

/* The outer-boundary nodes the Dirichlet variant holds at zero, ascending:
 * count (nullable) and nodes host [count] (nullable); INVALID_ARG before the
 * first cgp_set_far_field(m, 1). */
int cgp_far_field_nodes(cgp_mesh m, int* count, int* nodes);

/*
 * cgp_mesh_fine_geometry - host copies of the fine mesh (synchronous).
 * xy_f  host [n_f][2] or NULL;  tri_f host [t_f][3] or NULL;  edges host [n_e][2]
 * (the coarse edges) or NULL.
 */
int cgp_mesh_fine_geometry(cgp_mesh m, double* xy_f, int* tri_f, int* edges);

/*
 * cgp_mesh_matrices - host copies of the assembled coarse operators (synchronous).
 * rowptr [n_c+1], col [nnz], K/Gx/Gy [nnz], dinv [n_c]; any may be NULL.
 */
int cgp_mesh_matrices(cgp_mesh m, int* rowptr, int* col, double* K, double* Gx, double* Gy,
                      double* dinv);

/*
 * cgp_restrict - restriction by injection (Eq. 19) fused with the Poisson
 * right-hand side on the coarse mesh (Eq. 12 / Eq. 15 in weak form).
 *
 * kind        CGP_RHS_POTENTIAL: F = (u x B) in the x-y plane = (v B_z, -u B_z),
 *             the source of Delta phi = div(u x B) (Eqs. 5, 6, 12).
 *             CGP_RHS_PRESSURE: F = rho_over_dt * (u, v), the source of
 *             Delta p = (rho/dt) div(u~) (Eqs. 9, 15).
 * B           host [3], the magnetic field (only B_z enters F).
 * u_f, v_f    device [n_f] fine-node velocity components.
 * u_c, v_c    device [n_c] restricted velocity, or NULL to skip writing it.
 * b           device [n_c] output: b_i = sum_j Gx_ij F_x,j + Gy_ij F_y,j
 *             = int F . grad psi_i, the weak form of Delta x = div F with the
 *             natural condition d_n x = F . n.  b is not projected; the solver
 *             removes its mean.
 */
int cgp_restrict(cgp_mesh m, int kind, const double* B, double rho_over_dt,
                 const double* u_f, const double* v_f, double* u_c, double* v_c, double* b,
                 void* stream);

/*
 * cgp_poisson_solve - Jacobi-preconditioned CG on the singular Neumann system
 * K x = b (the coarse Poisson solve of CGP steps 2 and 6, Eqs. 12 and 15).
 *
 * b     device [n_c] right-hand side (not modified).
 * x     device [n_c]: the initial guess on entry when opts->use_x0, else
 *       ignored; the mean-zero solution on exit.
 * opts  host; NULL selects tol 1e-8, max_it 20000, FP64, x0 = 0.
 * info  host or NULL.  When non-NULL the call synchronises the stream once to
 *       read the solver state and returns the solve's status; when NULL the
 *       call is fully asynchronous and returns CGP_OK after the launch.
 *
 * b and x0 are projected to mean zero (the null space of K is the
 * constants), CG runs on the projected system, and the result is projected
 * again.  FP64 runs PCG in FP64, by default in the single-reduction form of
 * Chronopoulos and Gear (one grid barrier per iteration; the recurrences
 * for K p and the residual are checked against the true residual when the
 * recursive one converges, and CG restarts from the true residual if it
 * does not meet tol); tuning flag bit 1 selects the textbook iteration
 * (Saad, Alg. 9.1) with two barriers.  MIXED runs FP64 iterative refinement
 * (residual b - K x, correction sum and projection in FP64) around FP32 inner
 * PCG solves to inner_tol.  The whole solve is one persistent cooperative
 * kernel launch; its grid barriers give up after about two seconds without
 * progress and report CGP_ERR_TIMEOUT.  Not-converged is non-fatal: x holds
 * the last iterate.
 */
int cgp_poisson_solve(cgp_mesh m, const double* b, double* x, const cgp_solve_opts* opts,
                      cgp_solve_info* info, void* stream);

/*
 * cgp_poisson_solve_async - cgp_poisson_solve without any host synchronisation.
 *
 * Same arguments and semantics, except that the outcome is written by the
 * GPU into info_dev, a device pointer to one cgp_solve_info record (or NULL
 * to discard it): status CGP_ERR_TIMEOUT if a barrier gave up, else the
 * solve's status.  The call returns after the launch; host-side argument
 * errors are still returned immediately.  Suitable for back-to-back solves
 * and for stream capture.
 */
int cgp_poisson_solve_async(cgp_mesh m, const double* b, double* x, const cgp_solve_opts* opts,
                            cgp_solve_info* info_dev, void* stream);

/*
 * cgp_poisson_solve_noalloc - FP64 solve that allocates no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc when they solve (an application that hands all
 * device memory to its own pool or arena, a host framework whose allocator
 * must not be bypassed, a real-time loop where allocating, and the
 * synchronisation it can imply, is not allowed).  The caller passes the CSR
 * system K (rowptr [n+1], col [nnz], K [nnz], D^-1 [n], all device, e.g.
 * copied out with cgp_mesh_matrices) and b, x as in cgp_poisson_solve; the
 * solver's scratch is a static array inside the library, sized for
 * n <= CGP_STATIC_MAX_ROWS (65,536 rows, about 3.4 MB held on every GPU that
 * loads the library until the process exits).  Larger n is rejected with
 * CGP_ERR_INVALID_ARG.  Only opts->precision == CGP_FP64 is accepted.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  The address is kept together with the
 * identity of the device's CUDA context, so the first call after the caller
 * resets the device (cudaDeviceReset) looks it up again.  All calls share the
 * one array: calls that overlap on the GPU race on it, so serialise them (one
 * stream, one host thread at a time).
 * info behaves as in cgp_poisson_solve (NULL: asynchronous).
 */
#define CGP_STATIC_MAX_ROWS 65536
int cgp_poisson_solve_noalloc(int n, const int* rowptr, const int* col, const double* K,
                              const double* dinv, const double* b, double* x,
                              const cgp_solve_opts* opts, cgp_solve_info* info, void* stream);

/*
 * Batched solves: many independent systems in persistent launches.
 *
 * A batch fixes a list of distinct meshes (count >= 1; sizes may differ),
 * one right-hand side b[i] and one solution/initial-guess buffer x[i] per
 * mesh (device pointers, caller-owned, length n_c of that mesh; host arrays
 * of pointers, copied) and the solve options.  cgp_batch_solve runs every
 * system's Jacobi-PCG (FP64 or mixed precision, as in cgp_poisson_solve),
 * each system on its own group of blocks with its own barriers and
 * reductions, in one of two schedules:
 *   - waves (default): each system gets the blocks a solve of it alone would
 *     use (about 256 rows per block, at most blocks_per_sm x SMs), so that its
 *     rows fit in shared memory; systems are packed largest first into waves
 *     of at most blocks_per_sm x SMs blocks, and the waves run as consecutive
 *     cooperative launches, the wave of the smallest systems first: small
 *     systems share the GPU, large ones get all of it.  Tuning flag bits 5-6
 *     ask for 256 << k rows per block instead (k = 1..3; a system still gets
 *     at least the blocks that keep its chunk in shared memory), so that
 *     large systems share the GPU too;
 *   - packed (tuning flag bit 2): ONE cooperative launch holds every system,
 *     block groups sized in proportion to each system's work (nnz sqrt(n)).
 * Neither needs host work between launches, so a solve can be captured in a
 * CUDA graph and replayed.  The paper solves one system per time step
 * (Sect. 2.2); this serves many uneven independent systems at once (several
 * meshes, right-hand sides or Stuart numbers).
 *
 * cgp_batch_create    plans the launches (blocks per system, waves,
 *                     shared-memory residency, halo lists) and allocates the
 *                     batch's small device descriptors; synchronous.
 *                     INVALID_ARG if a mesh repeats (their scratch would be
 *                     shared) or a packed launch has more systems than
 *                     co-resident blocks.
 * cgp_batch_solve     the launches on `stream`, asynchronous.
 * cgp_batch_info      synchronises the device and reads each system's
 *                     outcome; seconds[i] (nullable) is the device time from
 *                     the launch's start to system i's finish.  Returns the
 *                     first non-OK status among the systems.
 * cgp_batch_set_tuning  re-plans with threads per block, lanes per CSR row,
 *                     blocks per SM (0 = as many as fit; waves: 0 or 1 =
 *                     one block per SM, never more than blocks of that size
 *                     fit on an SM) and flags (bit 0: rows in global
 *                     memory; bit 1: FP64 textbook iteration, as for
 *                     cgp_set_tuning; bit 2: one packed launch, not waves;
 *                     bit 3: tagged reductions (FP64 and mixed) and
 *                     bit 4: pipelined FP64 iteration, as for
 *                     cgp_set_tuning; bits 5-6: waves
 *                     with 256 << k rows per block).  INVALID_ARG for other
 *                     bits.
 * cgp_batch_autotune  times a set of launch shapes on the batch's own
 *                     systems (from x = 0) and keeps the fastest; writes the
 *                     best time in ms to best_ms (nullable).  Synchronous;
 *                     overwrites the x buffers.
 * cgp_batch_query     grid size, block, lanes, residency and blocks per
 *                     system (host [count], nullable).
 * cgp_poisson_solve_batched  one-shot create + solve (+ info when infos is
 *                     non-NULL) + destroy.
 */
typedef struct cgp_batch_s* cgp_batch;

int cgp_batch_create(const cgp_mesh* meshes, int count, const double* const* b, double* const* x,
                     const cgp_solve_opts* opts, cgp_batch* out);
int cgp_batch_solve(cgp_batch batch, void* stream);
int cgp_batch_info(cgp_batch batch, cgp_solve_info* infos, double* seconds);
int cgp_batch_set_tuning(cgp_batch batch, int block, int lanes, int blocks_per_sm, int flags);
int cgp_batch_autotune(cgp_batch batch, void* stream, double* best_ms);
int cgp_batch_query(cgp_batch batch, int* grid, int* block, int* lanes, int* resident, int* blocks);
int cgp_batch_destroy(cgp_batch batch);
int cgp_poisson_solve_batched(const cgp_mesh* meshes, int count, const double* const* b, double* const* x,
                              const cgp_solve_opts* opts, cgp_solve_info* infos, void* stream);

/*
 * Learned initial guess: a message-passing network on the coarse mesh's edges.
 *
 * The paper has no learned component; this addition to the method
 * predicts the PCG starting point of the potential solve (Eq. 12) from
 * the right-hand side b and the two previous solutions.  Per coarse node i,
 * f_i = [r/s_r, (phi1 - phi2)/s_d, b/s_b, x/15, y/15] with r = b - K phi1
 * (s = rms over nodes, each input scaled by its own size);
 * h0 = relu(We f + be); three layers of m_ij = relu(Wm [h_i; h_j; e_ij] + bm)
 * over the directed mesh edges i <- j (e_ij = (dx, dy, |d|) / mean edge
 * length), a_i = sum_j m_ij, h_i += relu(Wu [h_i; a_i] + bu); out = Wd h + bd;
 * x0 = phi1 + s_d * out (the solver projects x0 to mean zero).  Hidden width
 * 64; the dense layers run on the tensor cores in BF16 with FP32
 * accumulation; weights are kept in FP32 for Adam (lr given per step, betas
 * 0.9 / 0.999, eps 1e-8).  The training target is (phi(t) - phi1) / s_d
 * and the loss the mean squared error over all nodes of the batch.
 *
 * Parameters are one FP32 vector of cgp_gnn_param_count() values in this
 * order, row-major: We [64][5], be [64], then for l = 0, 1, 2: Wm_l [64][131],
 * bm_l [64], Wu_l [64][128], bu_l [64]; then Wd [64], bd [1].
 *
 * cgp_gnn_create   network for mesh m, training batches up to max_batch
 *                  samples; params host [param_count].  Allocates its device
 *                  memory; synchronous.
 * cgp_gnn_predict  x0 (device [n_c]) from b, phi1, phi2 (device [n_c]); async.
 *                  When every 16-node chunk gets its own block (n_c up to
 *                  16 x co-resident blocks) one cooperative launch runs the
 *                  whole forward, else the batched training forward does;
 *                  both take the same arithmetic steps in the same order,
 *                  so the same bits.  The cooperative launch's waits (one
 *                  grid barrier, then per-chunk flags of the neighbouring
 *                  chunks) give up after about two seconds and then leave
 *                  NaN in x0, which the solve reports as CGP_ERR_NONFINITE.
 *                  Calls on one network must not overlap on the GPU (they
 *                  share its activations and synchronisation words).
 * cgp_gnn_train_step  forward, loss, backward and one Adam step on `batch`
 *                  samples stacked sample-major (device [batch][n_c] each,
 *                  phi_t the solutions to learn); loss_dev (device float,
 *                  nullable) receives the batch loss; async.
 * cgp_gnn_gradients  forward + backward without the update; copies the
 *                  gradient (host [param_count]), the raw outputs (host
 *                  [batch][n_c]) and the loss (host) when non-NULL; synchronous.
 * cgp_gnn_get_params / cgp_gnn_set_params  host copies of the FP32 weights
 *                  (set also resets the Adam state); synchronous.
 */
typedef struct cgp_gnn_s* cgp_gnn;

int cgp_gnn_param_count(void);
int cgp_gnn_create(cgp_mesh m, int max_batch, const float* params, cgp_gnn* out);
int cgp_gnn_predict(cgp_gnn g, const double* b, const double* phi1, const double* phi2, double* x0, void* stream);
int cgp_gnn_train_step(cgp_gnn g, int batch, const double* b, const double* phi1, const double* phi2,
                       const double* phi_t, float lr, float* loss_dev, void* stream);
int cgp_gnn_gradients(cgp_gnn g, int batch, const double* b, const double* phi1, const double* phi2,
                      const double* phi_t, float* grads, float* out, float* loss, void* stream);
int cgp_gnn_get_params(cgp_gnn g, float* params);
int cgp_gnn_set_params(cgp_gnn g, const float* params);
int cgp_gnn_destroy(cgp_gnn g);

/*
 * cgp_prolong - prolongation by the P1 shape functions (Eq. 20), one level
 * at a time from the coarse to the fine mesh as the paper prescribes:
 * x_f[i] = x_c[i] for coarse nodes; then for l = 0 .. k-1,
 * x_f[n_l + e] = (x_f[a_e] + x_f[b_e]) / 2 at the midpoint of level-l edge e
 * (shape functions 1/2, 1/2, 0 there).  One launch per level.
 * x_c device [n_c]; x_f device [n_f].
 */
int cgp_prolong(cgp_mesh m, const double* x_c, double* x_f, void* stream);

/*
 * cgp_lorentz - gradient, current density and Lorentz force per fine triangle.
 *
 * For fine triangle t: g = grad phi_f (constant on P1), u_bar = vertex mean of
 * (u_f, v_f), j = sigma (-g + u_bar x B) (Ohm's law, Eqs. 4 and 7, with
 * g_z = u_z = 0), f = j x B (the source of Eqs. 2 and 8; with B = B_o k it is
 * the right-hand side of Eqs. 13-14).
 * phi_f, u_f, v_f  device [n_f].
 * B                host [3].
 * grad             device [2 * t_f], SoA: g_x for all triangles, then g_y.
 * force            device [2 * t_f], SoA: f_x then f_y; NULL computes only grad
 *                  (the pressure gradient of Eqs. 16-17).
 */
int cgp_lorentz(cgp_mesh m, const double* phi_f, const double* u_f, const double* v_f,
                const double* B, double sigma, double* grad, double* force, void* stream);

/*
 * cgp_velocity_correct - the velocity update of the pressure correction on the
 * fine mesh (Eqs. 16-17): u = u~ - (dt/rho) dp/dx, v = v~ - (dt/rho) dp/dy at
 * every fine node, with the P1 gradient of p_f (constant per fine triangle)
 * brought to the nodes by the lumped P1 mass: the area-weighted mean of the
 * gradients of the fine triangles around the node.
 * p_f, u_t, v_t, u, v  device [n_f]; u, v may alias u_t, v_t.
 * dt_over_rho          dt / rho.
 * The first call on a mesh builds the fine node -> triangle incidence
 * (synchronous, one allocation of about 24 t_f bytes, freed with the mesh).
 */
int cgp_velocity_correct(cgp_mesh m, const double* p_f, const double* u_t, const double* v_t,
                         double dt_over_rho, double* u, double* v, void* stream);

/*
 * cgp_spmv - y = K x with the coarse stiffness matrix (the product inside
 * every CG iteration).  precision CGP_FP64: x, y device double [n_c];
 * precision 1 (FP32): x, y device float [n_c] with the FP32 copy of K.
 */
int cgp_spmv(cgp_mesh m, int precision, const void* x, void* y, void* stream);

/*
 * cgp_mesh_set_ogrid - declare the coarse mesh an n_theta x n_r O-grid
 * (node (j, i) = j * n_theta + i, ring j = 0 .. n_r, angle i periodic, every
 * quad cut along its (i, j) - (i+1, j+1) diagonal) and build the seven-plane
 * stencil form of K: values at the fixed (angle, ring) offsets (0,0), (+-1,0),
 * (0,+-1), (+1,+1), (-1,-1), zeros where a neighbour does not exist, and no
 * column indices (9 s n bytes per product against CSR's 12 s n + 4 n; a
 * structured-stencil storage choice beside the paper's unstructured CSR).
 * Afterwards SpMV tuning flag bit 0 selects it for cgp_spmv, and solver
 * tuning flag bit 5 selects the O-grid tiles with the stencil product for
 * the persistent FP64 solver (cgp_set_tuning; cgp_autotune considers it).
 * Synchronous; one allocation of 84 n_c bytes (FP64 and FP32 planes), freed
 * with the mesh.  INVALID_ARG if n_theta * (n_r + 1) != n_c or if any row's
 * CSR pattern differs from the stencil.
 */
int cgp_mesh_set_ogrid(cgp_mesh m, int n_theta, int n_r);

/*
 * cgp_set_tuning / cgp_get_tuning - launch shape of a kernel family on this mesh.
 *
 * what    CGP_TUNE_SOLVE_FP64, CGP_TUNE_SOLVE_MIXED (the persistent solver),
 *         CGP_TUNE_SPMV_FP64, CGP_TUNE_SPMV_FP32 (cgp_spmv).
 * block   threads per block: a multiple of 32 in [64, 512] for the solver,
 *         [64, 256] for the SpMV; 0 = default.
 * lanes   threads cooperating on one CSR row: 1, 2, 4, 8 or 32 (32 is one
 *         warp per row); 0 = default.
 * blocks  solver: blocks of the persistent grid (clamped to what can be
 *         co-resident); SpMV: grid size; 0 = chosen from the size.
 * flags   solver: bit 0 keeps each block's rows in global memory instead of
 *         shared memory; bit 1 (FP64 only) runs the textbook two-barrier CG
 *         iteration instead of the single-reduction form; bit 2 renumbers the
 *         rows by recursive coordinate bisection so that every block's chunk
 *         is a compact patch of the mesh (smaller halos; b and x pass through
 *         a gather and a scatter launch; the renumbered system is built once
 *         per block count and boundary condition, about 12 nnz + 45 n_c
 *         bytes); bit 3 (the FP64 single-reduction form, and the FP32 inner
 *         iterations of MIXED) passes each grid-wide reduction through tagged
 *         slots that show by themselves when every block has stored its
 *         partial sum, polled while the barrier counter fills, instead of a
 *         read of the slots after the barrier (FP32: the same totals, bit for
 *         bit; FP64: 64-bit fixed-point partials, exact up to a truncation
 *         2^-54 below a warp's or block's largest term); bit 4 (FP64, rows in shared memory, at least 256
 *         threads per block and 1, 2 or 4 lanes per row; otherwise the
 *         single-reduction form runs) runs the pipelined iteration of
 *         Ghysels and Vanroose: four warps of every block complete the
 *         iteration's grid reduction and fetch the next halo while the others
 *         form the next product, at the price of three more FP64 vector
 *         operations per row and recurrences that drift sooner (a restart
 *         from the true residual near tight tolerances); bit 5 (FP64,
 *         meshes registered with cgp_mesh_set_ogrid, rows in shared memory)
 *         renumbers the rows into near-rectangular tiles of the O-grid's
 *         (angle, ring) index grid, one per block, and forms every product
 *         with the seven-point stencil on the block's padded box (no column
 *         indices; bit 2 is then ignored); with bit 4 as well and at least
 *         256 threads per block the tiles run the pipelined iteration
 *         without a grid barrier in the loop: three warps poll every block's
 *         tagged partial sums while the others form the next product, and
 *         each block publishes its w behind a flag (release) that the blocks
 *         reading its rows wait for (acquire, bounded; cgp_autotune does not
 *         try this form); other bits must be 0.
 *         SpMV: bit 0 uses the O-grid stencil form (cgp_mesh_set_ogrid) with
 *         one thread per row (lanes ignored).
 * Invalid shapes are rejected with INVALID_ARG.  cgp_autotune sets these.
 */
typedef enum {
  CGP_TUNE_SOLVE_FP64 = 0,
  CGP_TUNE_SOLVE_MIXED = 1,
  CGP_TUNE_SPMV_FP64 = 2,
  CGP_TUNE_SPMV_FP32 = 3
} cgp_tune_target;

int cgp_set_tuning(cgp_mesh m, int what, int block, int lanes, int blocks, int flags);
int cgp_get_tuning(cgp_mesh m, int what, int* block, int* lanes, int* blocks, int* flags);

/*
 * cgp_autotune - pick the solver's launch shape for this mesh by timing.
 *
 * Runs the solve (precision CGP_FP64 or CGP_MIXED, tol 1e-8, from x = 0) on
 * the caller's right-hand side b (device [n_c]) for every candidate of
 * threads per block {256, 512}, lanes per CSR row {1, 2, 4}, grid size (a
 * few counts around the SM count, and 1..16 blocks for small systems),
 * shared-memory residency, the row order (flag bit 2), the reduction form
 * (flag bit 3) and, for FP64, the iteration form (flag bits 1 and 4) and,
 * on meshes registered with cgp_mesh_set_ogrid, the O-grid tiles with the
 * stencil product (flag bit 5); only candidates that converge count,
 * and keeps the fastest with cgp_set_tuning.  Every candidate meets the
 * same tolerance on the true residual.  x
 * (device [n_c]) is overwritten.  cache_path (nullable) names a text file of
 * earlier results keyed by GPU name, n, nnz and target: a hit applies the
 * cached shape without timing (best_ms = -1), a miss appends the new
 * result.  Synchronous.
 */
int cgp_autotune(cgp_mesh m, int precision, const double* b, double* x, const char* cache_path, void* stream,
                 double* best_ms);

/*
 * cgp_last_launch - shape of the last persistent solver launch on this mesh.
 * precision CGP_FP64 or CGP_MIXED; outputs (any may be NULL): grid blocks,
 * threads per block, whether each block kept its rows in shared memory, and
 * the dynamic shared memory per block in bytes.  All zero before any solve.
 */
int cgp_last_launch(cgp_mesh m, int precision, int* blocks, int* block, int* resident, int* smem_bytes);

/*
 * cgp_barrier_selftest - exercise the persistent solver's grid barrier.
 * Launches nblk co-resident blocks (1 <= nblk <= 1024) of which the last
 * `absent` never arrive; the others give up after spin_ns nanoseconds and the
 * call returns CGP_ERR_TIMEOUT, or CGP_OK when absent == 0.  The GPU context
 * stays usable either way.  Synchronises the stream.
 */
int cgp_barrier_selftest(int nblk, int absent, long long spin_ns, void* stream);

/* Frees the mesh and its device memory (synchronises the device first). */
int cgp_mesh_destroy(cgp_mesh m);

/* Message of the last failed call on this thread ("" if none). */
const char* cgp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CGP_H */
